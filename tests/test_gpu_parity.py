"""Parity of the CUDA library (through the C ABI) with the FP64 oracle, element by element.

Every comparison checks two measures against the same tolerance: the relative L2 norm over the
whole field, |y_gpu - y_ref| / |y_ref|, and the largest element error relative to the largest
reference element, max|y_gpu - y_ref| / max|y_ref| (a single wrong site, which moves the L2
measure by only about 1/sqrt(sites), fails the second). Tolerances:
  FP64 1e-12; FP32 1e-5 (both from the operator's specification), for Dhop, Mooee, M, Mpc and
  Mpc^+ Mpc alike: every launch computes in the storage precision and these operators have no
  cancellation that amplifies rounding (|Mpc x| is comparable to |Mooee x|);
  FP16 / BF16 storage with FP32 arithmetic, against the oracle applied to the same rounded
  inputs: the output is rounded once to the storage format (unit roundoff 2^-11 / 2^-8) after
  FP32 arithmetic, so 2e-3 (FP16) and 1.6e-2 (BF16) bound it with margin; the Schur operators
  store their intermediate fields in the storage format too (Mpc two launches, Mpc^+ Mpc four,
  each rounding its output once), so they get 4x and 8x that bound; against the exact inputs the
  error is reported and bounded loosely (input rounding of 24 + 18 reals per hop).
"""
import numpy as np
import pytest
import torch

from paper_2203_06777_gb300 import synth

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)
M5, MASS = 1.8, 0.01
TOL = {0: 1e-12, 1: 1e-5, 2: 2e-3, 3: 1.6e-2}


@pytest.fixture(scope="module")
def dwf():
    from paper_2203_06777_gb300 import dwf as mod

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mod.load()
    return mod


def rel(a, b):
    """The larger of the relative L2 error and the largest element error relative to the largest
    reference element."""
    a = np.asarray(a)
    b = np.asarray(b)
    d = np.abs(a - b)
    return float(max(np.linalg.norm(d) / np.linalg.norm(b), d.max() / np.abs(b).max()))


# Schur operators in 16-bit storage: one output rounding per launch (Mpc 2 launches, Mpc^+ Mpc 4)
SCHUR_FACTOR = {"mpc": {0: 1, 1: 1, 2: 4, 3: 4}, "mdagm": {0: 1, 1: 1, 2: 8, 3: 8}}


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def parity_fields(oracle, dims, psi):
    odd = oracle.parity_mask(dims)[..., None, None, None]
    return psi * ~odd, psi * odd


def round_spinor(x, prec):
    """The canonical field as the library stores it in `prec` (round to nearest), back in FP64."""
    if prec == 0:
        return x
    if prec == 1:
        f = lambda a: a.astype(np.float32).astype(np.float64)
    elif prec == 2:
        f = lambda a: a.astype(np.float16).astype(np.float64)
    else:  # bfloat16: 8 significant bits, round to nearest even, straight from FP64
        def f(a):
            m, e = np.frexp(a)
            return np.ldexp(np.rint(m * 256.0) / 256.0, e)
    return f(x.real) + 1j * f(x.imag)


def make(dwf, dims, Ls, seed, eps=None, compress12=False, bc=BC, mass=MASS):
    U = synth.random_gauge(dims, seed=seed, eps=eps)
    op = dwf.GridDWF(dims, Ls, M5, mass, bc=bc, compress12=compress12)
    op.set_gauge(dev(U))
    return op, U


# ---------------------------------------------------------------- layout


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_pack_unpack_roundtrip(dwf, oracle_lib, prec):
    dims, Ls = (4, 2, 6, 4), 3
    op, _ = make(dwf, dims, Ls, 1)
    psi = synth.random_spinor(dims, Ls, seed=2)
    f = op.pack(dev(psi), prec, dwf.FULL)
    back = host(op.unpack(f))
    assert np.array_equal(back, round_spinor(psi, prec))
    for sub in (dwf.EVEN, dwf.ODD):
        h = op.pack(dev(psi), prec, sub)
        b = host(op.unpack(h, subset=sub))
        mask = oracle_lib.parity_mask(dims)
        m = mask if sub == dwf.ODD else ~mask
        assert np.array_equal(b[m], round_spinor(psi, prec)[m])
        assert np.all(b[~m] == 0)


# ---------------------------------------------------------------- Dhop

DHOP_CASES = [((4, 4, 4, 4), 8, None), ((4, 4, 4, 4), 16, 0.3), ((2, 4, 6, 4), 3, None), ((6, 2, 4, 2), 12, None),
              ((4, 6, 2, 4), 1, None), ((2, 2, 2, 2), 2, None), ((8, 4, 4, 6), 4, 0.5)]


@pytest.mark.parametrize("dims,Ls,eps", DHOP_CASES)
@pytest.mark.parametrize("prec", [0, 1])
def test_dhop_parity(dwf, oracle_lib, dims, Ls, eps, prec):
    op, U = make(dwf, dims, Ls, 11, eps=eps)
    psi = synth.random_spinor(dims, Ls, seed=12)
    f = op.pack(dev(psi), prec, dwf.FULL)
    psi_r = round_spinor(psi, prec)
    U_r = round_spinor(U, prec)
    for dag in (False, True):
        ref = oracle_lib.dhop(dims, Ls, BC, U_r, psi_r, dag=dag)
        out = host(op.unpack(op.dhop(f, dwf.FULL, dag=dag)))
        assert rel(out, ref) < TOL[prec], (dag, rel(out, ref))
        # half-lattice forms: EO reads the odd half, OE the even half
        pe, po = parity_fields(oracle_lib, dims, psi)
        fo = op.pack(dev(po), prec, dwf.ODD)
        fe = op.pack(dev(pe), prec, dwf.EVEN)
        eo = host(op.unpack(op.dhop(fo, dwf.EVEN, dag=dag), subset=dwf.EVEN))
        oe = host(op.unpack(op.dhop(fe, dwf.ODD, dag=dag), subset=dwf.ODD))
        mask = oracle_lib.parity_mask(dims)
        assert rel(eo[~mask], ref[~mask]) < TOL[prec]
        assert rel(oe[mask], ref[mask]) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_dhop_largest_ls(dwf, oracle_lib, prec):
    """Ls = 128, the largest the handle accepts (FP64: one thread per slice fills a CTA)."""
    dims, Ls = (2, 2, 2, 4), 128
    op, U = make(dwf, dims, Ls, 13)
    psi = synth.random_spinor(dims, Ls, seed=14)
    f = op.pack(dev(psi), prec, dwf.FULL)
    for dag in (False, True):
        ref = oracle_lib.dhop(dims, Ls, BC, round_spinor(U, prec), round_spinor(psi, prec), dag=dag)
        assert rel(host(op.unpack(op.dhop(f, dwf.FULL, dag=dag))), ref) < TOL[prec]
    _, po = parity_fields(oracle_lib, dims, round_spinor(psi, prec))
    mask = oracle_lib.parity_mask(dims)
    out = host(op.unpack(op.mdagm(op.pack(dev(po), prec, dwf.ODD)), subset=dwf.ODD))
    ref = oracle_lib.mdagm(dims, Ls, M5, MASS, BC, round_spinor(U, prec), po)
    assert rel(out[mask], ref[mask]) < SCHUR_FACTOR["mdagm"][prec] * TOL[prec]


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("dims,Ls", [(d, ls) for d, ls, _ in DHOP_CASES] + [((4, 4, 2, 2), 16)])
def test_dhop_low_precision_storage(dwf, oracle_lib, prec, dims, Ls):
    op, U = make(dwf, dims, Ls, 21, eps=0.3)
    psi = synth.random_spinor(dims, Ls, seed=22)
    f = op.pack(dev(psi), prec, dwf.FULL)
    for dag in (False, True):
        out = host(op.unpack(op.dhop(f, dwf.FULL, dag=dag)))
        ref_same_inputs = oracle_lib.dhop(dims, Ls, BC, round_spinor(U, prec), round_spinor(psi, prec), dag=dag)
        assert rel(out, ref_same_inputs) < TOL[prec]
        ref_exact = oracle_lib.dhop(dims, Ls, BC, U, psi, dag=dag)
        assert rel(out, ref_exact) < 4 * TOL[prec]


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_dhop_compressed_links(dwf, oracle_lib, prec):
    dims, Ls = (4, 4, 6, 4), 6
    op, U = make(dwf, dims, Ls, 31, compress12=True)
    psi = synth.random_spinor(dims, Ls, seed=32)
    f = op.pack(dev(psi), prec, dwf.FULL)
    out = host(op.unpack(op.dhop(f, dwf.FULL)))
    ref = oracle_lib.dhop(dims, Ls, BC, U, psi)
    tol = {0: 1e-12, 1: 1e-5, 2: 4 * TOL[2], 3: 4 * TOL[3]}[prec]
    assert rel(out, ref) < tol


def test_dhop_boundary_conditions(dwf, oracle_lib):
    dims, Ls = (4, 2, 4, 6), 4
    for bc in [(1, 1, 1, 1), (-1, 1, 1, -1), (-1, -1, -1, -1), (1, -1, 1, 1)]:
        op, U = make(dwf, dims, Ls, 41, bc=bc)
        psi = synth.random_spinor(dims, Ls, seed=42)
        f = op.pack(dev(psi), 0, dwf.FULL)
        assert rel(host(op.unpack(op.dhop(f, dwf.FULL))), oracle_lib.dhop(dims, Ls, bc, U, psi)) < 1e-12


# ---------------------------------------------------------------- fifth dimension, M, Schur


@pytest.mark.parametrize("Ls", [1, 2, 7, 8, 16])
@pytest.mark.parametrize("prec", [0, 1])
def test_mooee_family(dwf, oracle_lib, Ls, prec):
    dims = (4, 2, 2, 4)
    op, _ = make(dwf, dims, Ls, 51)
    psi = synth.random_spinor(dims, Ls, seed=52)
    f = op.pack(dev(psi), prec, dwf.FULL)
    psi_r = round_spinor(psi, prec)
    for dag in (False, True):
        for inv in (False, True):
            out = host(op.unpack(op.mooee(f, dag=dag, inverse=inv)))
            ref = oracle_lib.mooee(dims, Ls, M5, MASS, psi_r, dag=dag, inverse=inv)
            assert rel(out, ref) < TOL[prec], (dag, inv)
    g = f.clone()
    op.mooee(g, inverse=True, out=g)  # in place
    assert rel(host(op.unpack(g)), oracle_lib.mooee(dims, Ls, M5, MASS, psi_r, inverse=True)) < TOL[prec]


# The packed kernels' CTA sizes: Ls 5-6 take 32 sites of 3 slice pairs (96 threads; 48 sites per
# parity here, so one end CTA), Ls 11-12 16 sites of 6, Ls 23-24 8 sites of 12, which also sets the
# Mooee^-1 lines' strides (28 and 696 floats at Ls = 24).
@pytest.mark.parametrize("dims,Ls", [((4, 4, 4, 4), 8), ((2, 4, 6, 4), 5), ((6, 4, 2, 2), 12), ((4, 2, 2, 6), 6),
                                     ((4, 4, 2, 2), 24)])
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_m_mpc_mdagm(dwf, oracle_lib, dims, Ls, prec):
    op, U = make(dwf, dims, Ls, 61)
    psi = synth.random_spinor(dims, Ls, seed=62)
    psi_r, U_r = round_spinor(psi, prec), round_spinor(U, prec)
    f = op.pack(dev(psi), prec, dwf.FULL)
    for dag in (False, True):
        out = host(op.unpack(op.m(f, dag=dag)))
        assert rel(out, oracle_lib.m(dims, Ls, M5, MASS, BC, U_r, psi_r, dag=dag)) < TOL[prec]
    _, po = parity_fields(oracle_lib, dims, psi_r)
    fo = op.pack(dev(po), prec, dwf.ODD)
    mask = oracle_lib.parity_mask(dims)
    for dag in (False, True):
        out = host(op.unpack(op.mpc(fo, dag=dag), subset=dwf.ODD))
        ref = oracle_lib.mpc(dims, Ls, M5, MASS, BC, U_r, po, dag=dag)
        assert rel(out[mask], ref[mask]) < SCHUR_FACTOR["mpc"][prec] * TOL[prec], (dag, rel(out[mask], ref[mask]))
    out = host(op.unpack(op.mdagm(fo), subset=dwf.ODD))
    ref = oracle_lib.mdagm(dims, Ls, M5, MASS, BC, U_r, po)
    assert rel(out[mask], ref[mask]) < SCHUR_FACTOR["mdagm"][prec] * TOL[prec], rel(out[mask], ref[mask])


def test_mdagm_low_precision(dwf, oracle_lib):
    dims, Ls = (4, 4, 4, 4), 8
    for prec in (2, 3):
        op, U = make(dwf, dims, Ls, 71, eps=0.3)
        psi = synth.random_spinor(dims, Ls, seed=72)
        _, po = parity_fields(oracle_lib, dims, psi)
        fo = op.pack(dev(po), prec, dwf.ODD)
        out = host(op.unpack(op.mdagm(fo), subset=dwf.ODD))
        ref = oracle_lib.mdagm(dims, Ls, M5, MASS, BC, U, po)
        mask = oracle_lib.parity_mask(dims)
        assert rel(out[mask], ref[mask]) < 8 * TOL[prec]


# ---------------------------------------------------------------- reductions


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_norm_inner(dwf, prec):
    dims, Ls = (4, 4, 2, 6), 5
    op, _ = make(dwf, dims, Ls, 81)
    a = synth.random_spinor(dims, Ls, seed=82)
    b = synth.random_spinor(dims, Ls, seed=83)
    fa, fb = op.pack(dev(a), prec, dwf.FULL), op.pack(dev(b), prec, dwf.FULL)
    ar, br = round_spinor(a, prec), round_spinor(b, prec)
    tol = 1e-13 if prec == 0 else 1e-6
    n2 = op.norm2(fa)
    assert abs(n2 - np.vdot(ar, ar).real) < tol * n2
    z = op.inner(fa, fb)
    zr = np.vdot(ar, br)
    assert abs(z - zr) < tol * np.sqrt(n2 * np.vdot(br, br).real)
    assert op.norm2(fa) == n2  # bitwise reproducible


# ---------------------------------------------------------------- solvers


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_cg_solves_full_system(dwf, oracle_lib, mode):
    dims, Ls = (4, 4, 4, 4), 8
    op, U = make(dwf, dims, Ls, 91, eps=0.4)
    b = synth.random_spinor(dims, Ls, seed=92)
    fb = op.pack(dev(b), 0, dwf.FULL)
    x, st = op.cg(fb, tol=1e-10, maxiter=5000, mode=mode)
    assert st.converged and st.true_residual <= 1e-10
    xs = host(op.unpack(x))
    # the oracle recomputes the residual of the full system and the Schur normal equations
    r = b - oracle_lib.m(dims, Ls, M5, MASS, BC, U, xs)
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-8
    xo, it, res, ok = oracle_lib.schur_cg(dims, Ls, M5, MASS, BC, U, b, tol=1e-12, maxiter=20000)
    assert ok
    assert rel(xs, xo) < 1e-7


@pytest.mark.parametrize("mode,delta,lag", [(1, "0.1", "0"), (1, "1e-6", "1"), (2, "0.3", "1"), (3, "0.01", "1"),
                                            (2, None, "0")])
def test_mixed_cg_tuning_knobs(dwf, oracle_lib, monkeypatch, mode, delta, lag):
    """GRID_DWF_CG_DELTA and GRID_DWF_CG_LAG (read when the handle is created) change how often
    the mixed CG folds its inner solution into x and recomputes the FP64 residual, and when it
    decides to, not what it converges to: the solution still reaches the tolerance, and the
    oracle's recomputed residual of the full system agrees."""
    if delta is None:
        monkeypatch.delenv("GRID_DWF_CG_DELTA", raising=False)
    else:
        monkeypatch.setenv("GRID_DWF_CG_DELTA", delta)
    monkeypatch.setenv("GRID_DWF_CG_LAG", lag)
    dims, Ls = (4, 4, 4, 4), 8
    op, U = make(dwf, dims, Ls, 93, eps=0.4)
    b = synth.random_spinor(dims, Ls, seed=94)
    fb = op.pack(dev(b), 0, dwf.FULL)
    x, st = op.cg(fb, tol=1e-10, maxiter=5000, mode=mode)
    assert st.converged and st.true_residual <= 1e-10
    assert st.reliable_updates >= 1
    xs = host(op.unpack(x))
    r = b - oracle_lib.m(dims, Ls, M5, MASS, BC, U, xs)
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-8


@pytest.mark.parametrize("mode", [1, 2])
def test_mixed_cg_stopped_by_maxiter(dwf, oracle_lib, mode):
    """A mixed solve cut short by maxiter: not converged, and the returned x is the folded
    solution whose true residual the stats report (recomputed here by the oracle)."""
    dims, Ls = (4, 4, 4, 4), 8
    op, U = make(dwf, dims, Ls, 95, eps=0.4)
    b = synth.random_spinor(dims, Ls, seed=96)
    fb = op.pack(dev(b), 0, dwf.FULL)
    x, st = op.cg(fb, tol=1e-12, maxiter=7, mode=mode, raise_on_fail=False)
    assert not st.converged and st.iterations == 7
    xs = host(op.unpack(x))
    assert np.all(np.isfinite(xs))
    # the Schur normal-equation residual of x_o reported by the solver, against the oracle's
    mask = oracle_lib.parity_mask(dims)[..., None, None, None]
    be, bo = b * ~mask, b * mask
    bp = bo + 0.5 * oracle_lib.dhop(dims, Ls, BC, U, oracle_lib.mooee(dims, Ls, M5, MASS, be, inverse=True)) * mask
    rhs = oracle_lib.mpc(dims, Ls, M5, MASS, BC, U, bp, dag=True)
    r = rhs - oracle_lib.mdagm(dims, Ls, M5, MASS, BC, U, xs * mask)
    true_res = np.linalg.norm(r[mask[..., 0, 0, 0]]) / np.linalg.norm(rhs[mask[..., 0, 0, 0]])
    assert abs(true_res - st.true_residual) < 1e-6 * true_res + 1e-14


# ---------------------------------------------------------------- force


# (4, 4, 4, 6) x 10: 192 sites per parity in CTAs of 25, so the FP32 M launch that also sums the
# action has end CTAs (one per half) beside its full ones.
@pytest.mark.parametrize("dims,Ls", [((4, 4, 4, 4), 4), ((2, 4, 2, 6), 3), ((4, 2, 4, 2), 16), ((4, 4, 4, 6), 10)])
@pytest.mark.parametrize("prec", [0, 1])
def test_force_parity(dwf, oracle_lib, dims, Ls, prec):
    op, U = make(dwf, dims, Ls, 101)
    psi = synth.random_spinor(dims, Ls, seed=102)
    f = op.pack(dev(psi), prec, dwf.FULL)
    S, F, G = op.force(f)
    psi_r, U_r = round_spinor(psi, prec), round_spinor(U, prec)
    S_ref, F_ref, G_ref = oracle_lib.force(dims, Ls, M5, MASS, BC, U_r, psi_r)
    tol = 1e-12 if prec == 0 else 2e-5
    assert abs(S - S_ref) < tol * S_ref
    assert rel(host(F), F_ref) < tol
    assert rel(host(G), G_ref) < tol


def test_autograd_gradients_match_oracle(dwf, oracle_lib):
    dims, Ls = (4, 2, 2, 4), 4
    U = synth.random_gauge(dims, seed=111)
    psi = synth.random_spinor(dims, Ls, seed=112)
    op = dwf.GridDWF(dims, Ls, M5, MASS, bc=BC)
    pt = dev(psi).requires_grad_(True)
    Ut = dev(U).requires_grad_(True)
    S = dwf.dwf_action(pt, Ut, op)
    S.backward()
    S_ref, F_ref, G_ref = oracle_lib.force(dims, Ls, M5, MASS, BC, U, psi)
    chi = oracle_lib.m(dims, Ls, M5, MASS, BC, U, psi)
    gpsi_ref = 2.0 * oracle_lib.m(dims, Ls, M5, MASS, BC, U, chi, dag=True)
    assert abs(S.item() - S_ref) < 1e-12 * S_ref
    assert rel(host(pt.grad), gpsi_ref) < 1e-12
    assert rel(host(Ut.grad), G_ref) < 1e-12


def test_autograd_gradcheck(dwf):
    dims, Ls = (2, 2, 2, 2), 2
    U = dev(synth.random_gauge(dims, seed=121)).requires_grad_(True)
    psi = dev(synth.random_spinor(dims, Ls, seed=122)).requires_grad_(True)
    op = dwf.GridDWF(dims, Ls, M5, MASS, bc=BC)
    assert torch.autograd.gradcheck(lambda p, u: dwf.dwf_action(p, u, op), (psi, U), eps=1e-6, atol=1e-5, rtol=1e-6)


# ---------------------------------------------------------------- pseudofermion action and force
# S = phi^+ (Mpc^+ Mpc)^-1 phi: the library solves to a true residual tol and contracts the
# force; the oracle solves by plain CG to the same tol. Two solutions at residual tol differ by
# at most cond(Mpc^+ Mpc) * tol relative (about 1e3 here), so X, F and G agree to 1e-8 at
# tol = 1e-12, and S (quadratic in the error) much closer.


def _odd(oracle, dims, psi):
    return psi * oracle.parity_mask(dims)[..., None, None, None]


@pytest.mark.parametrize("dims,Ls", [((4, 4, 4, 4), 8), ((2, 4, 2, 6), 3), ((4, 2, 4, 2), 16)])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_pf_force_parity(dwf, oracle_lib, dims, Ls, mode):
    op, U = make(dwf, dims, Ls, 201)
    phi = _odd(oracle_lib, dims, synth.random_spinor(dims, Ls, seed=202))
    f = op.pack(dev(phi), 0, dwf.ODD)
    S, F, G, X, st = op.pf_force(f, tol=1e-12, mode=mode)
    assert st.converged and st.true_residual <= 1e-12
    S_ref, X_ref, F_ref, G_ref, it = oracle_lib.pf_force(dims, Ls, M5, MASS, BC, U, phi, tol=1e-12)
    assert it > 0
    assert abs(S - S_ref) < 1e-11 * S_ref
    assert rel(host(op.unpack(X, subset=dwf.ODD)), X_ref) < 1e-8
    assert rel(host(F), F_ref) < 1e-8
    assert rel(host(G), G_ref) < 1e-8


def test_pf_force_fp32_contraction(dwf, oracle_lib):
    """FP32 force contraction of the FP64 solve: fields rounded once to FP32, FP64 accumulation."""
    dims, Ls = (4, 4, 2, 4), 8
    op, U = make(dwf, dims, Ls, 211)
    phi = _odd(oracle_lib, dims, synth.random_spinor(dims, Ls, seed=212))
    f = op.pack(dev(phi), 0, dwf.ODD)
    S, F, G, X, st = op.pf_force(f, tol=1e-12, mode=dwf.CG_MIXED_FP32, precision=dwf.FP32)
    S_ref, _, F_ref, G_ref, _ = oracle_lib.pf_force(dims, Ls, M5, MASS, BC, U, phi, tol=1e-12)
    assert abs(S - S_ref) < 1e-11 * S_ref
    assert rel(host(F), F_ref) < 2e-5
    assert rel(host(G), G_ref) < 2e-5


def test_pf_force_finite_differences_on_gpu(dwf, oracle_lib):
    """The GPU force against central differences of the GPU action along su(3) directions."""
    dims, Ls = (4, 4, 4, 4), 4
    op, U = make(dwf, dims, Ls, 221)
    phi = _odd(oracle_lib, dims, synth.random_spinor(dims, Ls, seed=222))
    f = op.pack(dev(phi), 0, dwf.ODD)

    def action(UU):
        op.set_gauge(dev(UU))
        return op.pf_force(f, tol=1e-13, maxiter=100000, want_F=False, want_G=False)[0]

    S0 = action(U)
    op.set_gauge(dev(U))
    _, F, _, _, _ = op.pf_force(f, tol=1e-13, maxiter=100000, want_G=False)
    F = host(F)
    h = 1e-4
    for k in range(2):
        A = synth.random_su3_algebra(U.shape[:-2], seed=230 + k)
        lam, v = np.linalg.eigh(-1j * h * A)
        Ep = np.einsum("...ab,...b,...cb->...ac", v, np.exp(1j * lam), np.conj(v))
        fd = (action(Ep @ U) - action(np.conj(np.swapaxes(Ep, -1, -2)) @ U)) / (2 * h)
        an = np.sum(np.einsum("...ba,...ba->...", np.conj(A), F).real)
        assert abs(fd - an) < 1e-6 * (abs(an) + 1e-3 * S0), (fd, an)


def test_pf_autograd_matches_oracle(dwf, oracle_lib):
    dims, Ls = (4, 2, 2, 4), 4
    U = synth.random_gauge(dims, seed=241)
    phi = _odd(oracle_lib, dims, synth.random_spinor(dims, Ls, seed=242))
    op = dwf.GridDWF(dims, Ls, M5, MASS, bc=BC)
    pt = dev(phi).requires_grad_(True)
    Ut = dev(U).requires_grad_(True)
    S = dwf.pseudofermion_action(pt, Ut, op, tol=1e-13)
    S.backward()
    S_ref, X_ref, _, G_ref, _ = oracle_lib.pf_force(dims, Ls, M5, MASS, BC, U, phi, tol=1e-13)
    assert abs(S.item() - S_ref) < 1e-11 * S_ref
    assert rel(host(pt.grad), 2.0 * X_ref) < 1e-8
    assert rel(host(Ut.grad), G_ref) < 1e-8


# ---------------------------------------------------------------- errors are reported, not raised on the GPU


def test_argument_errors(dwf):
    dims, Ls = (4, 4, 4, 4), 4
    op, _ = make(dwf, dims, Ls, 131)
    f = op.field(0, dwf.FULL, zero=True)
    with pytest.raises(dwf.GridDWFError) as e:
        op.dhop(f, dwf.FULL, out=f)  # in == out
    assert e.value.code == -6
    with pytest.raises(dwf.GridDWFError) as e:
        op._call("grid_dwf_dhop", 0, dwf._ptr(f.data_ptr() + 8), dwf._ptr(f), 2, 0)  # misaligned
    assert e.value.code == -1
    op2 = dwf.GridDWF(dims, Ls, M5, MASS)
    with pytest.raises(dwf.GridDWFError) as e:
        op2.dhop(f, dwf.FULL)  # no gauge field yet
    assert e.value.code == -7
    b = op.field(0, dwf.FULL, zero=True)
    b[0] = float("nan")
    with pytest.raises(dwf.GridDWFError) as e:
        op.cg(b, tol=1e-10, maxiter=10)
    assert e.value.code == -5
    b = op.pack(dev(synth.random_spinor(dims, Ls, seed=132)), 0, dwf.FULL)
    x, st = op.cg(b, tol=1e-14, maxiter=3, raise_on_fail=False)
    assert not st.converged and st.iterations == 3


# ---------------------------------------------------------------- full-size workloads
# The benchmark's 16^4 x 16 lattice, compared over the whole field (the oracle takes a few
# seconds on the host cores), and the 32^4 x 16 lattice on sampled sites: the oracle's per-site
# hopping term at 256 random 4D sites (all slices) against the same sites of the GPU output.


def _workload(name):
    return synth.WORKLOADS[name]


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_full_size_dhop_16x16x16x16_ls16(dwf, oracle_lib, prec):
    w = _workload("dwf_16x16x16x16_ls16_exp0.3")
    dims, Ls = w["dims"], w["Ls"]
    U = synth.random_gauge(dims, seed=1000 * w["case"], eps=w["eps"])
    psi = synth.random_spinor(dims, Ls, seed=1000 * w["case"] + 1)
    op = dwf.GridDWF(dims, Ls, w["M5"], w["mass"], bc=BC)
    op.set_gauge(dev(U))
    f = op.pack(dev(psi), prec, dwf.FULL)
    ref = oracle_lib.dhop(dims, Ls, BC, round_spinor(U, prec), round_spinor(psi, prec))
    # the benchmark's launch: one full-lattice call (the packed precisions apply both halves in
    # one launch, the second half from the CTAs past the first half's grid)
    got = host(op.unpack(op.dhop(f, dwf.FULL)))
    assert rel(got, ref) < TOL[prec], rel(got, ref)
    # and the two half-lattice launches
    half = op.half_reals
    out = op.field(prec, dwf.FULL)
    op.dhop(f[half:], dwf.EVEN, out=out[:half])
    op.dhop(f[:half], dwf.ODD, out=out[half:])
    got = host(op.unpack(out))
    assert rel(got, ref) < TOL[prec], rel(got, ref)


@pytest.fixture(scope="module")
def fields_32():
    w = _workload("dwf_32x32x32x32_ls16_exp0.5")
    U = synth.random_gauge(w["dims"], seed=1000 * w["case"], eps=w["eps"])
    psi = synth.random_spinor(w["dims"], w["Ls"], seed=1000 * w["case"] + 1)
    return w, U, psi


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_full_size_dhop_32x32x32x32_ls16_sampled(dwf, oracle_lib, fields_32, prec):
    w, U, psi = fields_32
    dims, Ls = w["dims"], w["Ls"]
    op = dwf.GridDWF(dims, Ls, w["M5"], w["mass"], bc=BC)
    op.set_gauge(dev(U))
    f = op.pack(dev(psi), prec, dwf.FULL)
    got = host(op.unpack(op.dhop(f, dwf.FULL))).reshape(-1, Ls, 4, 3)
    op.close()
    rng = np.random.default_rng(77)
    sites = rng.choice(int(np.prod(dims)), size=256, replace=False)
    lx, ly, lz, lt = dims
    # include the lattice corners, where every hop wraps around
    sites = np.concatenate([sites, [0, lx - 1, lx * ly * lz * lt - 1]])
    # the oracle reads only the sampled sites and their 8 neighbours: round just those
    V = int(np.prod(dims))
    need = set(int(x) for x in sites)
    for x in sites:
        c = [int(x) % lx, int(x) // lx % ly, int(x) // (lx * ly) % lz, int(x) // (lx * ly * lz)]
        for mu in range(4):
            for d in (1, -1):
                cn = list(c)
                cn[mu] = (cn[mu] + d) % dims[mu]
                need.add(cn[0] + lx * (cn[1] + ly * (cn[2] + lz * cn[3])))
    idx = np.array(sorted(need))
    psi_r = psi.reshape(V, Ls, 4, 3).copy()
    U_r = U.reshape(V, 4, 3, 3).copy()
    psi_r[idx] = round_spinor(psi_r[idx], prec)
    U_r[idx] = round_spinor(U_r[idx], prec)
    ref = oracle_lib.dhop_sites(dims, Ls, BC, U_r.reshape(U.shape), psi_r.reshape(psi.shape), sites)
    assert rel(got[sites], ref) < TOL[prec]


def test_force_8x8x8x8_ls8_fd_and_oracle(dwf, oracle_lib):
    """The derivative workload's check case: 8^4 x Ls=8, Haar links, FP64. The GPU force and
    ambient gradient match the oracle's explicit formula, and central differences of the GPU's
    own action along single link components (exact up to rounding: S is quadratic there)."""
    w = synth.WORKLOADS["dwf_8x8x8x8_ls8_haar"]
    dims, Ls = w["dims"], w["Ls"]
    U = synth.random_gauge(dims, seed=1000 * w["case"])
    psi = synth.random_spinor(dims, Ls, seed=1000 * w["case"] + 1)
    op = dwf.GridDWF(dims, Ls, w["M5"], w["mass"], bc=BC)
    op.set_gauge(dev(U))
    f = op.pack(dev(psi), 0, dwf.FULL)
    S, F, G = op.force(f)
    S_ref, F_ref, G_ref = oracle_lib.force(dims, Ls, w["M5"], w["mass"], BC, U, psi)
    assert abs(S - S_ref) < 1e-12 * S_ref
    assert rel(host(F), F_ref) < 1e-12 and rel(host(G), G_ref) < 1e-12
    Gh = host(G)
    rng = np.random.default_rng(5)
    hstep = 0.1
    for _ in range(4):
        idx = tuple(int(rng.integers(0, n)) for n in U.shape)
        for unit in (1.0, 1j):
            vals = []
            for sgn in (1, -1):
                Up = U.copy()
                Up[idx] += sgn * hstep * unit
                op.set_gauge(dev(Up))
                vals.append(op.norm2(op.m(f)))
            fd = (vals[0] - vals[1]) / (2 * hstep)
            an = (np.conj(Gh[idx]) * unit).real
            assert abs(fd - an) < 1e-9 * abs(an) + 1e-12 * S / hstep, (fd, an)


# ---------------------------------------------------------------- random-shape sweep
# Seeded random lattice shapes (each extent 2, 4 or 6; Ls in 1..16) against the oracle: ragged
# half lattices, odd Ls (pad slice), tail launches and every Ls specialisation and the generic
# kernel, for the hopping term (both signs) and the full M.

def _random_shapes(n=12, seed=2203):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        dims = tuple(int(v) for v in rng.choice([2, 4, 6], size=4))
        Ls = int(rng.choice([1, 2, 3, 4, 5, 8, 12, 16]))
        out.append((dims, Ls))
    return out


@pytest.mark.parametrize("dims,Ls", _random_shapes())
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_random_shape_sweep(dwf, oracle_lib, dims, Ls, prec):
    op, U = make(dwf, dims, Ls, 301, eps=0.4)
    psi = synth.random_spinor(dims, Ls, seed=302)
    f = op.pack(dev(psi), prec, dwf.FULL)
    psi_r, U_r = round_spinor(psi, prec), round_spinor(U, prec)
    for dag in (False, True):
        ref = oracle_lib.dhop(dims, Ls, BC, U_r, psi_r, dag=dag)
        assert rel(host(op.unpack(op.dhop(f, dwf.FULL, dag=dag))), ref) < TOL[prec], ("dhop", dag)
    ref = oracle_lib.m(dims, Ls, M5, MASS, BC, U_r, psi_r)
    assert rel(host(op.unpack(op.m(f))), ref) < TOL[prec], ("m", rel(host(op.unpack(op.m(f))), ref))


# ---------------------------------------------------------------- walk order and solver paths


@pytest.mark.parametrize("zblk", [0, 2, 4])
@pytest.mark.parametrize("prec", [1, 2])
def test_dhop_z_blocked_walk(dwf, oracle_lib, monkeypatch, zblk, prec):
    """The z-blocked CTA walk (chosen automatically for FP32 fields larger than L2; forced here on
    a small lattice through GRID_DWF_ZBLOCK, read when the handle is created) visits every site
    once: Dhop, M and Mpc^+ Mpc equal the oracle's, and the walk does not change a single bit."""
    dims, Ls = (8, 4, 8, 6), 16
    monkeypatch.setenv("GRID_DWF_ZBLOCK", str(zblk))
    op, U = make(dwf, dims, Ls, 311, eps=0.3)
    monkeypatch.setenv("GRID_DWF_ZBLOCK", "0")
    ref_op, _ = make(dwf, dims, Ls, 311, eps=0.3)
    psi = synth.random_spinor(dims, Ls, seed=312)
    f = op.pack(dev(psi), prec, dwf.FULL)
    psi_r, U_r = round_spinor(psi, prec), round_spinor(U, prec)
    for dag in (False, True):
        out = op.dhop(f, dwf.FULL, dag=dag)
        assert rel(host(op.unpack(out)), oracle_lib.dhop(dims, Ls, BC, U_r, psi_r, dag=dag)) < TOL[prec]
        assert torch.equal(out, ref_op.dhop(f, dwf.FULL, dag=dag))
    assert torch.equal(op.m(f), ref_op.m(f))
    _, po = parity_fields(oracle_lib, dims, psi_r)
    fo = op.pack(dev(po), prec, dwf.ODD)
    assert torch.equal(op.mdagm(fo), ref_op.mdagm(fo))


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_mixed_cg_with_compressed_links(dwf, oracle_lib, mode):
    """12-real links take the unfused inner step (separate p^+ A p and r update passes); the
    solution still meets the tolerance, checked by the oracle."""
    dims, Ls = (4, 4, 4, 4), 8
    op, U = make(dwf, dims, Ls, 93, eps=0.4, compress12=True)
    b = synth.random_spinor(dims, Ls, seed=94)
    fb = op.pack(dev(b), 0, dwf.FULL)
    x, st = op.cg(fb, tol=1e-10, maxiter=5000, mode=mode)
    assert st.converged and st.true_residual <= 1e-10
    xs = host(op.unpack(x))
    r = b - oracle_lib.m(dims, Ls, M5, MASS, BC, U, xs)
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-8
