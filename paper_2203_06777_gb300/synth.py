"""Seeded synthetic inputs for the domain-wall operator: gauge links and spinor fields.

This module holds no part of the operator's arithmetic. It only draws random fields, and both
the CUDA path and the CPU oracle consume what it draws. Everything is NumPy FP64 in the
canonical site-major layout:

* spinor field ``psi[t, z, y, x, s, spin(4), colour(3)]`` (complex128), x fastest among the
  4D coordinates, the fifth-dimension index s inside each 4D site;
* gauge field ``U[t, z, y, x, mu(4), a(3), b(3)]`` (complex128), ``mu = 0, 1, 2, 3`` for
  the x, y, z, t directions; ``U[..., mu, a, b]`` is row a, column b of U_mu(x).

Lattice dimensions are passed as ``dims = (Lx, Ly, Lz, Lt)``.

Distributions (the paper measures on production gauge ensembles that are not available here;
these seeded synthetic fields stand in for them):

* Haar-random SU(3): QR of a complex Gaussian 3x3 matrix, the phases of R's diagonal moved
  into Q (Mezzadri 2007), then det fixed to 1 by dividing by the principal cube root of det Q.
* Weakly disordered links ``exp(i eps H)``, H a Gaussian traceless Hermitian 3x3 matrix,
  exponentiated through its eigendecomposition.
* Spinors: every complex component ``(N(0, 1/2) + i N(0, 1/2))`` so that ``E|z|^2 = 1``.

Seeds: ``numpy.random.default_rng(seed)``; the workloads use ``seed = 1000 * case + field``.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "complex_gaussian",
    "haar_su3",
    "exp_i_eps_h",
    "random_gauge",
    "random_spinor",
    "random_su3_transform",
    "random_su3_algebra",
    "random_spinor_device",
    "random_gauge_device",
    "unit_gauge",
    "WORKLOADS",
]


def _shape4(dims):
    lx, ly, lz, lt = (int(d) for d in dims)
    return (lt, lz, ly, lx)


def complex_gaussian(rng: np.random.Generator, shape, var: float = 1.0) -> np.ndarray:
    """Complex Gaussian with E|z|^2 = var (real and imaginary parts each of variance var/2)."""
    sd = np.sqrt(var / 2.0)
    return rng.normal(0.0, sd, size=shape) + 1j * rng.normal(0.0, sd, size=shape)


def haar_su3(rng: np.random.Generator, n: int) -> np.ndarray:
    """n Haar-distributed SU(3) matrices, shape (n, 3, 3)."""
    a = complex_gaussian(rng, (n, 3, 3))
    q, r = np.linalg.qr(a)
    d = np.diagonal(r, axis1=1, axis2=2)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    return q / (det ** (1.0 / 3.0))[:, None, None]


def exp_i_eps_h(rng: np.random.Generator, n: int, eps: float) -> np.ndarray:
    """n matrices exp(i eps H), H = traceless Hermitian part of a complex Gaussian 3x3."""
    a = complex_gaussian(rng, (n, 3, 3))
    h = 0.5 * (a + np.conj(np.swapaxes(a, 1, 2)))
    tr = np.trace(h, axis1=1, axis2=2).real
    h = h - (tr / 3.0)[:, None, None] * np.eye(3)[None]
    lam, v = np.linalg.eigh(h)
    ph = np.exp(1j * eps * lam)
    return np.einsum("nab,nb,ncb->nac", v, ph, np.conj(v))


def random_gauge(dims, seed: int, eps: float | None = None) -> np.ndarray:
    """Gauge field U[t,z,y,x,mu,a,b]: Haar SU(3) (eps None) or exp(i eps H) links."""
    rng = np.random.default_rng(seed)
    sh = _shape4(dims)
    n = int(np.prod(sh)) * 4
    links = haar_su3(rng, n) if eps is None else exp_i_eps_h(rng, n, eps)
    return np.ascontiguousarray(links.reshape(sh + (4, 3, 3)))


def unit_gauge(dims) -> np.ndarray:
    sh = _shape4(dims)
    u = np.zeros(sh + (4, 3, 3), dtype=np.complex128)
    u[..., :, :] = np.eye(3)
    return u


def random_spinor(dims, Ls: int, seed: int) -> np.ndarray:
    """Spinor field psi[t,z,y,x,s,spin,colour] with unit variance per complex component."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(complex_gaussian(rng, _shape4(dims) + (int(Ls), 4, 3)))


def random_su3_transform(dims, seed: int) -> np.ndarray:
    """One Haar SU(3) matrix per 4D site, shape [t,z,y,x,3,3] (a gauge transformation)."""
    rng = np.random.default_rng(seed)
    sh = _shape4(dims)
    return np.ascontiguousarray(haar_su3(rng, int(np.prod(sh))).reshape(sh + (3, 3)))


def random_su3_algebra(shape, seed: int) -> np.ndarray:
    """Random traceless anti-Hermitian 3x3 matrices (directions in su(3)), shape + (3, 3)."""
    rng = np.random.default_rng(seed)
    a = complex_gaussian(rng, tuple(shape) + (3, 3))
    x = 0.5 * (a - np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(x, axis1=-2, axis2=-1)
    return x - (tr / 3.0)[..., None, None] * np.eye(3)


def random_spinor_device(dims, Ls: int, seed: int, device):
    """Same distribution as random_spinor, drawn on a CUDA device by torch's seeded generator
    (a different stream of numbers than the NumPy one; for timing runs on large lattices)."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    shape = _shape4(dims) + (int(Ls), 4, 3, 2)
    x = torch.randn(shape, generator=g, device=device, dtype=torch.float64) * np.sqrt(0.5)
    return torch.view_as_complex(x)


def random_gauge_device(dims, seed: int, eps: float, device):
    """exp(i eps H) links as in random_gauge, drawn on a CUDA device by torch's seeded generator;
    H the traceless Hermitian part of a complex Gaussian matrix, the exponential by torch."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    shape = _shape4(dims) + (4, 3, 3, 2)
    a = torch.view_as_complex(torch.randn(shape, generator=g, device=device, dtype=torch.float64) * np.sqrt(0.5))
    h = 0.5 * (a + a.conj().transpose(-1, -2))
    tr = torch.diagonal(h, dim1=-2, dim2=-1).sum(-1).real
    h = h - (tr / 3.0)[..., None, None] * torch.eye(3, dtype=h.dtype, device=device)
    return torch.linalg.matrix_exp(1j * eps * h).contiguous()


# The benchmark and parity workloads. Each names its lattice, fifth-dimension extent,
# domain-wall height M5, quark mass, boundary conditions and link disorder.
WORKLOADS = {
    "dwf_4x4x4x4_ls8_haar": dict(dims=(4, 4, 4, 4), Ls=8, M5=1.8, mass=0.01, eps=None, case=0),
    "dwf_16x16x16x16_ls16_exp0.3": dict(dims=(16, 16, 16, 16), Ls=16, M5=1.8, mass=0.01, eps=0.3, case=1),
    "dwf_24x24x24x24_ls12_exp0.4": dict(dims=(24, 24, 24, 24), Ls=12, M5=1.8, mass=0.01, eps=0.4, case=2),
    "dwf_8x8x8x8_ls8_haar": dict(dims=(8, 8, 8, 8), Ls=8, M5=1.8, mass=0.01, eps=None, case=3),
    "dwf_16x16x16x16_ls16_haar": dict(dims=(16, 16, 16, 16), Ls=16, M5=1.8, mass=0.01, eps=None, case=3),
    "dwf_32x32x32x32_ls16_exp0.5": dict(dims=(32, 32, 32, 32), Ls=16, M5=1.8, mass=0.005, eps=0.5, case=4),
}

BC_DEFAULT = (1, 1, 1, -1)
