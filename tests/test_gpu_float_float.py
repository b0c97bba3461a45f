"""Parity of the FP64 hopping term in float-float arithmetic (grid_dwf_set_fp64_arith with
FP64_ARITH_FLOAT_FLOAT) with the FP64 oracle, through the C ABI.

Float-float carries about 46 significant bits (each stored real is split into two floats with a
relative error below 2^-46 ~ 1.4e-14, and every sum and product keeps a similar relative error),
so the operator keeps the FP64 bar of 1e-12 relative over the whole field with margin; the
solvers that use it keep their FP64 residual targets. The exponent range is float's: the tests
scale fields by 1e+-20 to show it is not the binding limit for physical fields.
"""
import numpy as np
import pytest
import torch

from paper_2203_06777_gb300 import synth

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)
M5, MASS = 1.8, 0.01
TOL = 1e-12


@pytest.fixture(scope="module")
def dwf():
    from paper_2203_06777_gb300 import dwf as mod

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mod.load()
    return mod


def rel(a, b):
    """The larger of the relative L2 error and the largest element error relative to the largest
    reference element (a single wrong site fails the second)."""
    a = np.asarray(a)
    b = np.asarray(b)
    d = np.abs(a - b)
    return float(max(np.linalg.norm(d) / np.linalg.norm(b), d.max() / np.abs(b).max()))


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def make(dwf, dims, Ls, seed, eps=None, compress12=False, bc=BC, mass=MASS):
    U = synth.random_gauge(dims, seed=seed, eps=eps)
    op = dwf.GridDWF(dims, Ls, M5, mass, bc=bc, compress12=compress12, fp64_arith=dwf.FP64_ARITH_FLOAT_FLOAT)
    op.set_gauge(dev(U))
    return op, U


CASES = [((4, 4, 4, 4), 8, None), ((4, 4, 4, 4), 16, 0.3), ((2, 4, 6, 4), 3, None), ((6, 2, 4, 2), 12, None),
         ((4, 6, 2, 4), 1, None), ((2, 2, 2, 2), 2, None), ((8, 4, 4, 6), 4, 0.5)]


@pytest.mark.parametrize("dims,Ls,eps", CASES)
def test_dhop_float_float(dwf, oracle_lib, dims, Ls, eps):
    op, U = make(dwf, dims, Ls, 11, eps=eps)
    psi = synth.random_spinor(dims, Ls, seed=12)
    f = op.pack(dev(psi), 0, dwf.FULL)
    mask = oracle_lib.parity_mask(dims)
    for dag in (False, True):
        ref = oracle_lib.dhop(dims, Ls, BC, U, psi, dag=dag)
        assert rel(host(op.unpack(op.dhop(f, dwf.FULL, dag=dag))), ref) < TOL
        po = psi * mask[..., None, None, None]
        pe = psi * ~mask[..., None, None, None]
        eo = host(op.unpack(op.dhop(op.pack(dev(po), 0, dwf.ODD), dwf.EVEN, dag=dag), subset=dwf.EVEN))
        oe = host(op.unpack(op.dhop(op.pack(dev(pe), 0, dwf.EVEN), dwf.ODD, dag=dag), subset=dwf.ODD))
        assert rel(eo[~mask], ref[~mask]) < TOL
        assert rel(oe[mask], ref[mask]) < TOL


def test_dhop_float_float_compressed_links_and_boundaries(dwf, oracle_lib):
    dims, Ls = (4, 4, 6, 4), 6
    op, U = make(dwf, dims, Ls, 31, compress12=True)
    psi = synth.random_spinor(dims, Ls, seed=32)
    f = op.pack(dev(psi), 0, dwf.FULL)
    assert rel(host(op.unpack(op.dhop(f, dwf.FULL))), oracle_lib.dhop(dims, Ls, BC, U, psi)) < TOL
    dims, Ls = (4, 2, 4, 6), 4
    for bc in [(1, 1, 1, 1), (-1, 1, 1, -1), (-1, -1, -1, -1), (1, -1, 1, 1)]:
        op, U = make(dwf, dims, Ls, 41, bc=bc)
        psi = synth.random_spinor(dims, Ls, seed=42)
        f = op.pack(dev(psi), 0, dwf.FULL)
        assert rel(host(op.unpack(op.dhop(f, dwf.FULL))), oracle_lib.dhop(dims, Ls, bc, U, psi)) < TOL


@pytest.mark.parametrize("scale", [1e-20, 1e20])
def test_dhop_float_float_magnitudes(dwf, oracle_lib, scale):
    """Far from 1 but inside float's range the relative accuracy is unchanged."""
    dims, Ls = (4, 4, 2, 4), 8
    op, U = make(dwf, dims, Ls, 45)
    psi = synth.random_spinor(dims, Ls, seed=46) * scale
    f = op.pack(dev(psi), 0, dwf.FULL)
    assert rel(host(op.unpack(op.dhop(f, dwf.FULL))), oracle_lib.dhop(dims, Ls, BC, U, psi)) < TOL


def test_float_float_largest_ls(dwf, oracle_lib):
    dims, Ls = (2, 2, 2, 4), 128
    op, U = make(dwf, dims, Ls, 15)
    psi = synth.random_spinor(dims, Ls, seed=16)
    f = op.pack(dev(psi), 0, dwf.FULL)
    assert rel(host(op.unpack(op.dhop(f, dwf.FULL))), oracle_lib.dhop(dims, Ls, BC, U, psi)) < TOL
    assert rel(host(op.unpack(op.m(f))), oracle_lib.m(dims, Ls, M5, MASS, BC, U, psi)) < TOL


def test_dhop_float_float_zero_field(dwf):
    dims, Ls = (4, 4, 2, 2), 5
    op, _ = make(dwf, dims, Ls, 47)
    f = op.field(0, dwf.FULL, zero=True)
    out = op.dhop(f, dwf.FULL)
    assert torch.count_nonzero(out).item() == 0


@pytest.mark.parametrize("dims,Ls", [((4, 4, 4, 4), 8), ((2, 4, 6, 4), 5), ((6, 4, 2, 2), 12)])
def test_m_mpc_mdagm_float_float(dwf, oracle_lib, dims, Ls):
    op, U = make(dwf, dims, Ls, 61)
    psi = synth.random_spinor(dims, Ls, seed=62)
    f = op.pack(dev(psi), 0, dwf.FULL)
    for dag in (False, True):
        assert rel(host(op.unpack(op.m(f, dag=dag))), oracle_lib.m(dims, Ls, M5, MASS, BC, U, psi, dag=dag)) < TOL
    mask = oracle_lib.parity_mask(dims)
    po = psi * mask[..., None, None, None]
    fo = op.pack(dev(po), 0, dwf.ODD)
    for dag in (False, True):
        out = host(op.unpack(op.mpc(fo, dag=dag), subset=dwf.ODD))
        ref = oracle_lib.mpc(dims, Ls, M5, MASS, BC, U, po, dag=dag)
        assert rel(out[mask], ref[mask]) < TOL, rel(out[mask], ref[mask])
    out = host(op.unpack(op.mdagm(fo), subset=dwf.ODD))
    assert rel(out[mask], oracle_lib.mdagm(dims, Ls, M5, MASS, BC, U, po)[mask]) < TOL


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_cg_float_float(dwf, oracle_lib, mode):
    """FP64 CG on the float-float operator, and the mixed CGs whose FP64 true residuals use it."""
    dims, Ls = (4, 4, 4, 4), 8
    op, U = make(dwf, dims, Ls, 91, eps=0.4)
    b = synth.random_spinor(dims, Ls, seed=92)
    fb = op.pack(dev(b), 0, dwf.FULL)
    x, st = op.cg(fb, tol=1e-10, maxiter=5000, mode=mode)
    assert st.converged and st.true_residual <= 1e-10
    xs = host(op.unpack(x))
    r = b - oracle_lib.m(dims, Ls, M5, MASS, BC, U, xs)
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-8
    xo, _, _, ok = oracle_lib.schur_cg(dims, Ls, M5, MASS, BC, U, b, tol=1e-12, maxiter=20000)
    assert ok
    assert rel(xs, xo) < 1e-7


@pytest.mark.parametrize("dims,Ls", [((4, 4, 4, 4), 4), ((2, 4, 2, 6), 3), ((4, 2, 4, 2), 16), ((2, 2, 2, 4), 128)])
def test_force_float_float(dwf, oracle_lib, dims, Ls):
    """S = |M psi|^2, its su(3) force and ambient gradient with FP64 fields in float-float."""
    op, U = make(dwf, dims, Ls, 101)
    psi = synth.random_spinor(dims, Ls, seed=102)
    S, F, G = op.force(op.pack(dev(psi), 0, dwf.FULL))
    S_ref, F_ref, G_ref = oracle_lib.force(dims, Ls, M5, MASS, BC, U, psi)
    assert abs(S - S_ref) < TOL * S_ref
    assert rel(host(F), F_ref) < TOL
    assert rel(host(G), G_ref) < TOL


def test_force_float_float_compressed_links(dwf, oracle_lib):
    dims, Ls = (4, 4, 2, 4), 6
    op, U = make(dwf, dims, Ls, 105, compress12=True)
    psi = synth.random_spinor(dims, Ls, seed=106)
    S, F, G = op.force(op.pack(dev(psi), 0, dwf.FULL))
    S_ref, F_ref, G_ref = oracle_lib.force(dims, Ls, M5, MASS, BC, U, psi)
    assert abs(S - S_ref) < TOL * S_ref
    assert rel(host(F), F_ref) < TOL and rel(host(G), G_ref) < TOL


def test_pf_force_float_float(dwf, oracle_lib):
    dims, Ls = (4, 4, 4, 4), 8
    op, U = make(dwf, dims, Ls, 201)
    phi = synth.random_spinor(dims, Ls, seed=202) * oracle_lib.parity_mask(dims)[..., None, None, None]
    S, F, G, X, st = op.pf_force(op.pack(dev(phi), 0, dwf.ODD), tol=1e-12, mode=dwf.CG_FP64)
    assert st.converged and st.true_residual <= 1e-12
    S_ref, X_ref, F_ref, G_ref, _ = oracle_lib.pf_force(dims, Ls, M5, MASS, BC, U, phi, tol=1e-12)
    assert abs(S - S_ref) < 1e-11 * S_ref
    assert rel(host(op.unpack(X, subset=dwf.ODD)), X_ref) < 1e-8
    assert rel(host(F), F_ref) < 1e-8
    assert rel(host(G), G_ref) < 1e-8


def test_full_size_dhop_16x16x16x16_ls16_float_float(dwf, oracle_lib):
    w = synth.WORKLOADS["dwf_16x16x16x16_ls16_exp0.3"]
    dims, Ls = w["dims"], w["Ls"]
    U = synth.random_gauge(dims, seed=1000 * w["case"], eps=w["eps"])
    psi = synth.random_spinor(dims, Ls, seed=1000 * w["case"] + 1)
    op = dwf.GridDWF(dims, Ls, w["M5"], w["mass"], bc=BC, fp64_arith=dwf.FP64_ARITH_FLOAT_FLOAT)
    op.set_gauge(dev(U))
    got = host(op.unpack(op.dhop(op.pack(dev(psi), 0, dwf.FULL), dwf.FULL)))
    assert rel(got, oracle_lib.dhop(dims, Ls, BC, U, psi)) < TOL


def test_mode_switch_and_errors(dwf, oracle_lib):
    dims, Ls = (4, 4, 2, 2), 4
    op, U = make(dwf, dims, Ls, 131)
    psi = synth.random_spinor(dims, Ls, seed=132)
    f = op.pack(dev(psi), 0, dwf.FULL)
    ref = oracle_lib.dhop(dims, Ls, BC, U, psi)
    a = host(op.unpack(op.dhop(f, dwf.FULL)))
    op.set_fp64_arith(dwf.FP64_ARITH_NATIVE)
    b = host(op.unpack(op.dhop(f, dwf.FULL)))
    assert rel(a, ref) < TOL and rel(b, ref) < TOL
    with pytest.raises(dwf.GridDWFError) as e:
        op.set_fp64_arith(7)
    assert e.value.code == -1
