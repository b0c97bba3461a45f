"""Guard bands around every output buffer: each call writes exactly its output field and nothing
before or after it (a kernel that strays past the end of a ragged lattice, a pad slice or a tail
launch would overwrite the guard), and its output is finite.

Each output is the middle of a larger byte buffer whose guards hold a fixed byte pattern; after
the call the pattern must be intact. Lattices include an odd Ls (a zero pad slice), a half
lattice that is not a multiple of the sites per CTA (the extra tail launch) and the largest Ls.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2203_06777_gb300 import synth

pytestmark = pytest.mark.gpu

GUARD = 4096  # bytes on each side, a multiple of 16 so the output stays 16-byte aligned
PATTERN = 0xA5
CASES = [((4, 2, 6, 4), 3), ((6, 4, 2, 2), 12), ((2, 2, 2, 4), 128)]


@pytest.fixture(scope="module")
def dwf():
    from paper_2203_06777_gb300 import dwf as mod

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mod.load()
    return mod


class Guarded:
    """An output tensor of `numel` elements of `dtype` inside guard bands."""

    def __init__(self, numel, dtype, shape=None):
        esz = torch.empty(0, dtype=dtype).element_size()
        self.nbytes = numel * esz
        self.buf = torch.full((2 * GUARD + self.nbytes,), PATTERN, dtype=torch.uint8, device="cuda")
        t = self.buf[GUARD:GUARD + self.nbytes].view(dtype)
        self.t = t.view(shape) if shape is not None else t

    def check(self, what):
        torch.cuda.synchronize()
        head = self.buf[:GUARD]
        tail = self.buf[GUARD + self.nbytes:]
        assert bool((head == PATTERN).all()), f"{what}: wrote before its output"
        assert bool((tail == PATTERN).all()), f"{what}: wrote past its output"
        v = self.t.view(torch.float64) if self.t.dtype == torch.complex128 else self.t
        assert bool(torch.isfinite(v.float()).all()), f"{what}: non-finite output"


def like(f):
    return Guarded(f.numel(), f.dtype)


@pytest.mark.parametrize("dims,Ls", CASES)
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_outputs_stay_in_bounds(dwf, dims, Ls, prec):
    U = synth.random_gauge(dims, seed=7, eps=0.3)
    psi = synth.random_spinor(dims, Ls, seed=8)
    for arith in ([dwf.FP64_ARITH_NATIVE, dwf.FP64_ARITH_FLOAT_FLOAT] if prec == 0 else [dwf.FP64_ARITH_NATIVE]):
        op = dwf.GridDWF(dims, Ls, 1.8, 0.01, fp64_arith=arith)
        op.set_gauge(torch.from_numpy(U).cuda())
        f = op.pack(torch.from_numpy(psi).cuda(), prec, dwf.FULL)
        half = op.half_reals
        fo, fe = f[half:].clone(), f[:half].clone()
        for dag in (False, True):
            g = like(f)
            op.dhop(f, dwf.FULL, dag=dag, out=g.t)
            g.check(f"dhop full dag={dag}")
            g = like(fo)
            op.dhop(fo, dwf.EVEN, dag=dag, out=g.t)
            g.check(f"dhop EO dag={dag}")
            g = like(fe)
            op.dhop(fe, dwf.ODD, dag=dag, out=g.t)
            g.check(f"dhop OE dag={dag}")
            g = like(f)
            op.m(f, dag=dag, out=g.t)
            g.check(f"m dag={dag}")
            g = like(fo)
            op.mpc(fo, dag=dag, out=g.t)
            g.check(f"mpc dag={dag}")
            for inv in (False, True):
                g = like(f)
                op.mooee(f, dag=dag, inverse=inv, out=g.t)
                g.check(f"mooee dag={dag} inverse={inv}")
        g = like(fo)
        op.mdagm(fo, out=g.t)
        g.check("mdagm")
        for dst in (0, 1, 2, 3):
            g = Guarded(f.numel(), op.field(dst, dwf.FULL).dtype)
            op.convert(f, dst, out=g.t)
            g.check(f"convert to {dst}")
        g = Guarded(int(np.prod(op.canonical_shape())), torch.complex128, op.canonical_shape())
        op.unpack(f, out=g.t)
        g.check("unpack")
        g = Guarded(f.numel(), f.dtype)
        op.pack(torch.from_numpy(psi).cuda(), prec, dwf.FULL, out=g.t)
        g.check("pack")
        if prec in (0, 1):
            lx, ly, lz, lt = dims
            shape = (lt, lz, ly, lx, 4, 3, 3)
            F = Guarded(int(np.prod(shape)), torch.complex128, shape)
            G = Guarded(int(np.prod(shape)), torch.complex128, shape)
            chi = like(f)
            S = ctypes.c_double()
            op._call("grid_dwf_force", prec, dwf._ptr(f), dwf._ptr(chi.t), dwf._ptr(F.t), dwf._ptr(G.t),
                     ctypes.byref(S))
            F.check("force F")
            G.check("force G")
            chi.check("force chi")
        op.close()


def test_cg_solution_stays_in_bounds(dwf):
    dims, Ls = (6, 4, 2, 2), 12
    op = dwf.GridDWF(dims, Ls, 1.8, 0.01)
    op.set_gauge(torch.from_numpy(synth.random_gauge(dims, seed=9, eps=0.3)).cuda())
    b = op.pack(torch.from_numpy(synth.random_spinor(dims, Ls, seed=10)).cuda(), 0, dwf.FULL)
    for mode in (0, 1, 2, 3):
        x = like(b)
        x.t.zero_()
        _, st = op.cg(b, x=x.t, tol=1e-10, maxiter=5000, mode=mode)
        assert st.converged
        x.check(f"cg mode {mode}")
