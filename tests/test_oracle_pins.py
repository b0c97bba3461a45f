"""Pins of the FP64 oracle against facts fixed outside it (CPU only).

The paper prints no formula or worked example for the domain-wall operator, so the oracle is
pinned by: dense brute-force matrices built independently (tests/_dense.py), the free-field
plane-wave closed form, gamma5- and gamma5*R5-hermiticity, adjoint identities, gauge
covariance, the closed-form inverse of the fifth-dimension matrix, the determinant of the
free zero-momentum operator (bare plus residual mass), exact dense solves, and central finite
differences of the action (the action |M psi|^2 and the pseudofermion action
phi^+ (Mpc^+ Mpc)^-1 phi, the latter against dense solves).
"""
import numpy as np
import pytest

from paper_2203_06777_gb300 import synth
from tests import _dense

BC = (1, 1, 1, -1)
M5, MASS = 1.8, 0.01


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def vdot(a, b):
    return np.vdot(a.ravel(), b.ravel())


# ---------------------------------------------------------------- gamma matrices


def test_gamma_clifford_and_basis(oracle_lib):
    g = oracle_lib.gamma()
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)
        for nu in range(4):
            anti = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(anti, 2.0 * (mu == nu) * np.eye(4))
    assert np.allclose(g[4], np.diag([1, 1, -1, -1]))
    assert np.allclose(g[:4], _dense.GAMMA)


# ---------------------------------------------------------------- dense brute force

DENSE_CASES = [((2, 2, 2, 2), 4), ((2, 2, 2, 4), 4), ((4, 2, 2, 2), 2)]


@pytest.mark.parametrize("dims,Ls", DENSE_CASES)
@pytest.mark.parametrize("dag", [False, True])
def test_dhop_matches_dense(oracle_lib, dims, Ls, dag):
    U = synth.random_gauge(dims, seed=11)
    psi = synth.random_spinor(dims, Ls, seed=12)
    D = _dense.dense_dhop(dims, Ls, BC, U, dag=dag)
    ref = (D @ psi.ravel()).reshape(psi.shape)
    full = oracle_lib.dhop(dims, Ls, BC, U, psi, out_parity=2, dag=dag)
    assert rel(full, ref) < 1e-14
    odd = oracle_lib.parity_mask(dims)
    for par in (0, 1):
        half = oracle_lib.dhop(dims, Ls, BC, U, psi, out_parity=par, dag=dag)
        mask = odd if par == 1 else ~odd
        assert rel(half[mask], ref[mask]) < 1e-14
        assert np.all(half[~mask] == 0)


@pytest.mark.parametrize("dims,Ls", DENSE_CASES)
def test_m_mooee_match_dense(oracle_lib, dims, Ls):
    U = synth.random_gauge(dims, seed=21)
    psi = synth.random_spinor(dims, Ls, seed=22)
    M = _dense.dense_m(dims, Ls, M5, MASS, BC, U)
    K = _dense.dense_mooee(dims, Ls, M5, MASS)
    v = psi.ravel()
    assert rel(oracle_lib.m(dims, Ls, M5, MASS, BC, U, psi).ravel(), M @ v) < 1e-14
    assert rel(oracle_lib.m(dims, Ls, M5, MASS, BC, U, psi, dag=True).ravel(), M.conj().T @ v) < 1e-14
    assert rel(oracle_lib.mooee(dims, Ls, M5, MASS, psi).ravel(), K @ v) < 1e-14
    assert rel(oracle_lib.mooee(dims, Ls, M5, MASS, psi, dag=True).ravel(), K.conj().T @ v) < 1e-14
    assert rel(oracle_lib.mooee(dims, Ls, M5, MASS, psi, inverse=True).ravel(), np.linalg.solve(K, v)) < 1e-13
    assert rel(oracle_lib.mooee(dims, Ls, M5, MASS, psi, dag=True, inverse=True).ravel(),
               np.linalg.solve(K.conj().T, v)) < 1e-13


@pytest.mark.parametrize("dims,Ls", DENSE_CASES[:2])
def test_schur_matches_dense_blocks(oracle_lib, dims, Ls):
    U = synth.random_gauge(dims, seed=31)
    psi = synth.random_spinor(dims, Ls, seed=32)
    Mpc, o = _dense.dense_schur_odd(dims, Ls, M5, MASS, BC, U)
    v = psi.ravel()[o]
    out = oracle_lib.mpc(dims, Ls, M5, MASS, BC, U, psi).ravel()
    assert rel(out[o], Mpc @ v) < 1e-13
    outd = oracle_lib.mpc(dims, Ls, M5, MASS, BC, U, psi, dag=True).ravel()
    assert rel(outd[o], Mpc.conj().T @ v) < 1e-13
    mdm = oracle_lib.mdagm(dims, Ls, M5, MASS, BC, U, psi).ravel()
    assert rel(mdm[o], Mpc.conj().T @ (Mpc @ v)) < 1e-13
    even = np.setdiff1d(np.arange(out.size), o)
    assert np.all(out[even] == 0) and np.all(mdm[even] == 0)


def test_schur_cg_solves_dense_system(oracle_lib):
    dims, Ls = (2, 2, 2, 4), 4
    U = synth.random_gauge(dims, seed=41)
    b = synth.random_spinor(dims, Ls, seed=42)
    x, it, res, ok = oracle_lib.schur_cg(dims, Ls, M5, MASS, BC, U, b, tol=1e-12, maxiter=2000)
    assert ok and res <= 1e-11
    M = _dense.dense_m(dims, Ls, M5, MASS, BC, U)
    xd = np.linalg.solve(M, b.ravel())
    assert rel(x.ravel(), xd) < 1e-9


# ---------------------------------------------------------------- closed forms


def plane_wave(dims, Ls, n, u):
    """psi(x, s) = exp(i p.x) u_s with p_mu = 2 pi n_mu / L_mu, antiperiodic in t."""
    lx, ly, lz, lt = dims
    p = [2 * np.pi * n[0] / lx, 2 * np.pi * n[1] / ly, 2 * np.pi * n[2] / lz, np.pi * (2 * n[3] + 1) / lt]
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    return ph[..., None, None, None] * u[None, None, None, None], p


@pytest.mark.parametrize("dims,Ls,n", [((4, 4, 4, 4), 2, (1, 0, 3, 0)), ((4, 6, 4, 8), 3, (1, 2, 3, 1)),
                                        ((8, 4, 4, 4), 1, (3, 1, 0, 2))])
def test_free_field_plane_wave(oracle_lib, dims, Ls, n):
    rng = np.random.default_rng(5)
    u = synth.complex_gaussian(rng, (Ls, 4, 3))
    psi, p = plane_wave(dims, Ls, n, u)
    U = synth.unit_gauge(dims)
    Dp = sum(2 * np.cos(p[m]) * np.eye(4) - 2j * np.sin(p[m]) * _dense.GAMMA[m] for m in range(4))
    expect_u = np.einsum("ab,sbc->sac", Dp, u)
    ref, _ = plane_wave(dims, Ls, n, expect_u)
    assert rel(oracle_lib.dhop(dims, Ls, BC, U, psi), ref) < 1e-13
    # the adjoint: Dhop^+ psi = [sum 2 cos p + 2 i gamma sin p] psi
    Dpd = sum(2 * np.cos(p[m]) * np.eye(4) + 2j * np.sin(p[m]) * _dense.GAMMA[m] for m in range(4))
    refd, _ = plane_wave(dims, Ls, n, np.einsum("ab,sbc->sac", Dpd, u))
    assert rel(oracle_lib.dhop(dims, Ls, BC, U, psi, dag=True), refd) < 1e-13


@pytest.mark.parametrize("Ls", [1, 2, 5, 8, 16])
@pytest.mark.parametrize("mass", [0.0, 0.01, 0.3])
def test_zero_momentum_determinant_bare_plus_residual_mass(oracle_lib, Ls, mass):
    """Free field at p = 0: per chirality the 5D operator is the Ls x Ls matrix
    (1 - M5) I - (shift) + m (corner); its determinant is (1 - M5)^Ls + m, the bare mass plus
    the residual mass of the domain-wall construction."""
    dims = (2, 2, 2, 2)
    U = synth.unit_gauge(dims)
    bc = (1, 1, 1, 1)
    cols = []
    for s in range(Ls):
        for sp in range(4):
            psi = np.zeros((2, 2, 2, 2, Ls, 4, 3), dtype=complex)
            psi[..., s, sp, 0] = 1.0
            out = oracle_lib.m(dims, Ls, M5, mass, bc, U, psi)
            cols.append(out[0, 0, 0, 0, :, :, 0].ravel())
    M0 = np.array(cols).T.reshape(Ls, 4, Ls, 4)
    for sp in range(4):
        block = M0[:, sp, :, sp]
        assert np.isclose(np.linalg.det(block), (1 - M5) ** Ls + mass, rtol=1e-12, atol=1e-14)
    assert np.allclose(M0[:, 0, :, 2], 0) and np.allclose(M0[:, 2, :, 0], 0)


@pytest.mark.parametrize("Ls", [1, 2, 7, 12, 16])
@pytest.mark.parametrize("dag", [False, True])
def test_mooee_inverse_closed_form(oracle_lib, Ls, dag):
    """Closed form of the inverse of the cyclic bidiagonal fifth-dimension matrix:
    for the chirality coupled to s-1 (upper spins), with d = 5 - M5,
      y_0 = (b_0 - m sum_{k=1}^{Ls-1} d^{-(Ls-k)} b_k) / (d + m d^{-(Ls-1)}),
      y_s = (b_s + y_{s-1}) / d;
    the other chirality is its mirror image in s; the adjoint swaps the two."""
    dims = (2, 2, 2, 2)
    b = synth.random_spinor(dims, Ls, seed=7)
    d = 5.0 - M5

    def lower_solve(bv):  # bv[s, ...]
        y = np.zeros_like(bv)
        acc = bv[0].copy()
        for k in range(1, Ls):
            acc = acc - MASS * d ** (-(Ls - k)) * bv[k]
        y[0] = acc / (d + MASS * d ** (-(Ls - 1)))
        for s in range(1, Ls):
            y[s] = (bv[s] + y[s - 1]) / d
        return y

    up, lo = slice(0, 2), slice(2, 4)
    if dag:
        up, lo = lo, up
    expect = np.empty_like(b)
    bb = np.moveaxis(b, 4, 0)
    ee = np.moveaxis(expect, 4, 0)
    ee[:, ..., up, :] = lower_solve(bb[:, ..., up, :])
    ee[:, ..., lo, :] = lower_solve(bb[::-1, ..., lo, :])[::-1]
    got = oracle_lib.mooee(dims, Ls, M5, MASS, b, dag=dag, inverse=True)
    assert rel(got, expect) < 1e-14
    back = oracle_lib.mooee(dims, Ls, M5, MASS, got, dag=dag)
    assert rel(back, b) < 1e-14


# ---------------------------------------------------------------- identities at larger volume


def test_gamma5_hermiticity_dhop(oracle_lib):
    dims, Ls = (4, 4, 4, 4), 4
    U = synth.random_gauge(dims, seed=51)
    psi = synth.random_spinor(dims, Ls, seed=52)
    chi = synth.random_spinor(dims, Ls, seed=53)
    g5 = np.diag([1, 1, -1, -1])
    g5x = lambda f: np.einsum("ab,...bc->...ac", g5, f)
    lhs = vdot(chi, oracle_lib.dhop(dims, Ls, BC, U, psi))
    rhs = vdot(g5x(oracle_lib.dhop(dims, Ls, BC, U, g5x(chi))), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    assert rel(oracle_lib.dhop(dims, Ls, BC, U, psi, dag=True), g5x(oracle_lib.dhop(dims, Ls, BC, U, g5x(psi)))) < 1e-14


def test_gamma5_r5_hermiticity_m(oracle_lib):
    dims, Ls = (4, 4, 4, 4), 6
    U = synth.random_gauge(dims, seed=61)
    psi = synth.random_spinor(dims, Ls, seed=62)
    g5 = np.diag([1, 1, -1, -1])
    gam = lambda f: np.einsum("ab,...bc->...ac", g5, f)[..., ::-1, :, :]
    lhs = oracle_lib.m(dims, Ls, M5, MASS, BC, U, psi, dag=True)
    rhs = gam(oracle_lib.m(dims, Ls, M5, MASS, BC, U, gam(psi)))
    assert rel(lhs, rhs) < 1e-14


def test_adjoint_pairs(oracle_lib):
    dims, Ls = (4, 4, 4, 4), 4
    U = synth.random_gauge(dims, seed=71)
    psi = synth.random_spinor(dims, Ls, seed=72)
    chi = synth.random_spinor(dims, Ls, seed=73)
    odd = oracle_lib.parity_mask(dims)
    ops = {
        "dhop": lambda f, d: oracle_lib.dhop(dims, Ls, BC, U, f, dag=d),
        "mooee": lambda f, d: oracle_lib.mooee(dims, Ls, M5, MASS, f, dag=d),
        "mooee_inv": lambda f, d: oracle_lib.mooee(dims, Ls, M5, MASS, f, dag=d, inverse=True),
        "m": lambda f, d: oracle_lib.m(dims, Ls, M5, MASS, BC, U, f, dag=d),
    }
    for name, op in ops.items():
        a = vdot(chi, op(psi, False))
        b = vdot(op(chi, True), psi)
        assert abs(a - b) < 1e-12 * abs(a), name
    po, co = psi * odd[..., None, None, None], chi * odd[..., None, None, None]
    a = vdot(co, oracle_lib.mpc(dims, Ls, M5, MASS, BC, U, po))
    b = vdot(oracle_lib.mpc(dims, Ls, M5, MASS, BC, U, co, dag=True), po)
    assert abs(a - b) < 1e-12 * abs(a)
    # EO / OE are adjoint blocks: <chi_e, D_eo psi_o> = <D^+_oe chi_e, psi_o>
    pe, ce = psi * ~odd[..., None, None, None], chi * ~odd[..., None, None, None]
    a = vdot(ce, oracle_lib.dhop(dims, Ls, BC, U, po, out_parity=0))
    b = vdot(oracle_lib.dhop(dims, Ls, BC, U, ce, out_parity=1, dag=True), po)
    assert abs(a - b) < 1e-12 * abs(a)


def test_gauge_covariance(oracle_lib):
    dims, Ls = (4, 4, 4, 6), 3
    U = synth.random_gauge(dims, seed=81)
    psi = synth.random_spinor(dims, Ls, seed=82)
    Om = synth.random_su3_transform(dims, seed=83)
    Up = np.empty_like(U)
    for mu in range(4):
        axis = 3 - mu  # canonical array axes are [t, z, y, x]
        Om_fwd = np.roll(Om, -1, axis=axis)
        Up[..., mu, :, :] = Om @ U[..., mu, :, :] @ np.conj(np.swapaxes(Om_fwd, -1, -2))
    rot = lambda f: np.einsum("tzyxab,tzyxspb->tzyxspa", Om, f)
    lhs = oracle_lib.dhop(dims, Ls, BC, Up, rot(psi))
    rhs = rot(oracle_lib.dhop(dims, Ls, BC, U, psi))
    assert rel(lhs, rhs) < 1e-14
    assert rel(oracle_lib.m(dims, Ls, M5, MASS, BC, Up, rot(psi)), rot(oracle_lib.m(dims, Ls, M5, MASS, BC, U, psi))) < 1e-14


def test_linearity(oracle_lib):
    dims, Ls = (4, 4, 2, 2), 3
    U = synth.random_gauge(dims, seed=91)
    a = synth.random_spinor(dims, Ls, seed=92)
    b = synth.random_spinor(dims, Ls, seed=93)
    z = 0.3 - 1.7j
    lhs = oracle_lib.m(dims, Ls, M5, MASS, BC, U, a + z * b)
    rhs = oracle_lib.m(dims, Ls, M5, MASS, BC, U, a) + z * oracle_lib.m(dims, Ls, M5, MASS, BC, U, b)
    assert rel(lhs, rhs) < 1e-14


# ---------------------------------------------------------------- derivatives


def _expm_su3(A):
    """exp of anti-Hermitian 3x3 matrices through the Hermitian eigendecomposition of -iA."""
    lam, v = np.linalg.eigh(-1j * A)
    return np.einsum("...ab,...b,...cb->...ac", v, np.exp(1j * lam), np.conj(v))


@pytest.mark.parametrize("dims,Ls,seed", [((4, 4, 4, 4), 4, 101), ((2, 4, 2, 4), 3, 111)])
def test_force_against_finite_differences(oracle_lib, dims, Ls, seed):
    U = synth.random_gauge(dims, seed=seed)
    psi = synth.random_spinor(dims, Ls, seed=seed + 1)
    S, F, G = oracle_lib.force(dims, Ls, M5, MASS, BC, U, psi)
    chi = oracle_lib.m(dims, Ls, M5, MASS, BC, U, psi)
    assert abs(S - np.vdot(chi, chi).real) < 1e-12 * S
    action = lambda UU: oracle_lib.norm2(oracle_lib.m(dims, Ls, M5, MASS, BC, UU, psi))
    h = 1e-5
    # F is traceless anti-Hermitian
    assert np.allclose(F, -np.conj(np.swapaxes(F, -1, -2)), atol=1e-12 * np.abs(F).max())
    assert np.allclose(np.trace(F, axis1=-2, axis2=-1), 0, atol=1e-12 * np.abs(F).max())
    # su(3) direction: U -> exp(eps A) U, dS/deps = sum Re tr(A^+ F)
    for k in range(3):
        A = synth.random_su3_algebra(U.shape[:-2], seed=seed + 10 + k)
        fd = (action(_expm_su3(h * A) @ U) - action(_expm_su3(-h * A) @ U)) / (2 * h)
        an = np.sum(np.einsum("...ba,...ba->...", np.conj(A), F).real)
        assert abs(fd - an) < 1e-6 * (abs(an) + 1e-3 * S), (fd, an)
    # single link, single component of the ambient gradient. M is real-linear in (Re U, Im U),
    # so S is quadratic along U + h E and the central difference is exact up to rounding
    # (about eps * S / h); a large step keeps that small.
    rng = np.random.default_rng(seed + 20)
    hl = 0.1
    for _ in range(3):
        idx = tuple(int(rng.integers(0, n)) for n in U.shape)
        for unit in (1.0, 1j):
            E = np.zeros_like(U)
            E[idx] = unit
            fd = (action(U + hl * E) - action(U - hl * E)) / (2 * hl)
            an = (np.conj(G[idx]) * unit).real
            assert abs(fd - an) < 1e-10 * abs(an) + 1e-13 * S / hl, (fd, an)
    # F = TA(G U^+)
    X = G @ np.conj(np.swapaxes(U, -1, -2))
    Xa = 0.5 * (X - np.conj(np.swapaxes(X, -1, -2)))
    Xa = Xa - (np.trace(Xa, axis1=-2, axis2=-1) / 3.0)[..., None, None] * np.eye(3)
    assert rel(Xa, F) < 1e-13


def _dense_pf_action(dims, Ls, U, phi):
    """S = phi_o^+ (Mpc^+ Mpc)^-1 phi_o with Mpc from the blocks of the dense M, and the solution X."""
    Mpc, o = _dense.dense_schur_odd(dims, Ls, M5, MASS, BC, U)
    po = phi.ravel()[o]
    xo = np.linalg.solve(Mpc.conj().T @ Mpc, po)
    X = np.zeros(phi.size, dtype=complex)
    X[o] = xo
    return float(np.vdot(po, xo).real), X.reshape(phi.shape)


@pytest.mark.parametrize("dims,Ls,seed", [((2, 2, 2, 4), 4, 501), ((4, 2, 2, 2), 3, 511)])
def test_pf_action_and_solution_match_dense(oracle_lib, dims, Ls, seed):
    U = synth.random_gauge(dims, seed=seed)
    phi = synth.random_spinor(dims, Ls, seed=seed + 1)  # even sites are ignored
    S, X, _, _, it = oracle_lib.pf_force(dims, Ls, M5, MASS, BC, U, phi, tol=1e-13, want_force=False)
    S_ref, X_ref = _dense_pf_action(dims, Ls, U, phi)
    assert it > 0
    assert abs(S - S_ref) < 1e-10 * S_ref
    assert rel(X, X_ref) < 1e-9
    assert np.all(X[~oracle_lib.parity_mask(dims)] == 0)


@pytest.mark.parametrize("dims,Ls,seed", [((2, 2, 2, 4), 4, 521), ((2, 4, 2, 2), 2, 531)])
def test_pf_force_against_finite_differences(oracle_lib, dims, Ls, seed):
    """F and G of S = phi^+ (Mpc^+ Mpc)^-1 phi against central differences of the dense action."""
    U = synth.random_gauge(dims, seed=seed)
    phi = synth.random_spinor(dims, Ls, seed=seed + 1)
    S, _, F, G, _ = oracle_lib.pf_force(dims, Ls, M5, MASS, BC, U, phi, tol=1e-13)
    action = lambda UU: _dense_pf_action(dims, Ls, UU, phi)[0]
    assert np.allclose(F, -np.conj(np.swapaxes(F, -1, -2)), atol=1e-12 * np.abs(F).max())
    assert np.allclose(np.trace(F, axis1=-2, axis2=-1), 0, atol=1e-12 * np.abs(F).max())
    h = 1e-4  # central differences: truncation O(h^2) relative
    for k in range(2):
        A = synth.random_su3_algebra(U.shape[:-2], seed=seed + 10 + k)
        fd = (action(_expm_su3(h * A) @ U) - action(_expm_su3(-h * A) @ U)) / (2 * h)
        an = np.sum(np.einsum("...ba,...ba->...", np.conj(A), F).real)
        assert abs(fd - an) < 1e-6 * (abs(an) + 1e-3 * S), (fd, an)
    rng = np.random.default_rng(seed + 20)
    for _ in range(2):
        idx = tuple(int(rng.integers(0, n)) for n in U.shape)
        for unit in (1.0, 1j):
            E = np.zeros_like(U)
            E[idx] = unit
            fd = (action(U + h * E) - action(U - h * E)) / (2 * h)
            an = (np.conj(G[idx]) * unit).real
            assert abs(fd - an) < 1e-6 * (abs(an) + 1e-3 * S), (fd, an)
    X = G @ np.conj(np.swapaxes(U, -1, -2))  # F = TA(G U^+)
    Xa = 0.5 * (X - np.conj(np.swapaxes(X, -1, -2)))
    Xa = Xa - (np.trace(Xa, axis1=-2, axis2=-1) / 3.0)[..., None, None] * np.eye(3)
    assert rel(Xa, F) < 1e-12


def test_psi_gradient_against_finite_differences(oracle_lib):
    dims, Ls = (4, 4, 2, 4), 4
    U = synth.random_gauge(dims, seed=121)
    psi = synth.random_spinor(dims, Ls, seed=122)
    chi = oracle_lib.m(dims, Ls, M5, MASS, BC, U, psi)
    grad = 2.0 * oracle_lib.m(dims, Ls, M5, MASS, BC, U, chi, dag=True)
    action = lambda p: oracle_lib.norm2(oracle_lib.m(dims, Ls, M5, MASS, BC, U, p))
    S = action(psi)
    h = 0.1  # S is quadratic in psi: the central difference is exact up to rounding
    for k in range(3):
        d = synth.random_spinor(dims, Ls, seed=130 + k)
        fd = (action(psi + h * d) - action(psi - h * d)) / (2 * h)
        an = np.vdot(grad, d).real
        assert abs(fd - an) < 1e-10 * abs(an) + 1e-13 * S / h, (fd, an)


def test_dhop_sites_matches_full_lattice(oracle_lib):
    dims, Ls = (4, 2, 6, 4), 3
    U = synth.random_gauge(dims, seed=141)
    psi = synth.random_spinor(dims, Ls, seed=142)
    sites = np.array([0, 5, 17, 63, 100, 191])
    for dag in (False, True):
        full = oracle_lib.dhop(dims, Ls, BC, U, psi, dag=dag).reshape(-1, Ls, 4, 3)
        assert np.array_equal(oracle_lib.dhop_sites(dims, Ls, BC, U, psi, sites, dag=dag), full[sites])
