"""FP64 CPU oracle for the 5D Shamir domain-wall fermion operator (test infrastructure).

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may import this
package. It wraps ``dwf_oracle.c`` (plain C99, FP64, OpenMP over 4D sites) through ctypes and
shares nothing with the CUDA library. Fields are NumPy complex128 arrays in the canonical
layout ``psi[t, z, y, x, s, spin, colour]`` and ``U[t, z, y, x, mu, a, b]``; dims are
``(Lx, Ly, Lz, Lt)``. Half-lattice fields are full-size arrays whose other-parity sites the
oracle ignores on input and zeroes on output.

The operator conventions are stated in the header of ``dwf_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dwf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libdwf_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP). Returns the shared-library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c99", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.dwf_oracle_gamma.argtypes = [_dp]
            lib.dwf_oracle_dhop.argtypes = [_ip, ctypes.c_int, _ip, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int]
            lib.dwf_oracle_dhop_sites.argtypes = [_ip, ctypes.c_int, _ip, _dp, _dp, ctypes.POINTER(ctypes.c_long),
                                                  ctypes.c_long, _dp, ctypes.c_int, ctypes.c_int]
            lib.dwf_oracle_mooee.argtypes = [_ip, ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _dp,
                                             ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.dwf_oracle_mooee.restype = ctypes.c_int
            for name in ("dwf_oracle_m", "dwf_oracle_mpc"):
                getattr(lib, name).argtypes = [_ip, ctypes.c_int, ctypes.c_double, ctypes.c_double, _ip, _dp, _dp,
                                               _dp, ctypes.c_int, ctypes.c_int]
            lib.dwf_oracle_mdagm.argtypes = [_ip, ctypes.c_int, ctypes.c_double, ctypes.c_double, _ip, _dp, _dp,
                                             _dp, ctypes.c_int]
            lib.dwf_oracle_schur_cg.argtypes = [_ip, ctypes.c_int, ctypes.c_double, ctypes.c_double, _ip, _dp,
                                                _dp, _dp, ctypes.c_double, ctypes.c_int, _ip, _dp, ctypes.c_int]
            lib.dwf_oracle_schur_cg.restype = ctypes.c_int
            lib.dwf_oracle_force.argtypes = [_ip, ctypes.c_int, ctypes.c_double, ctypes.c_double, _ip, _dp, _dp,
                                             _dp, _dp, ctypes.c_int]
            lib.dwf_oracle_force.restype = ctypes.c_double
            lib.dwf_oracle_pf_force.argtypes = [_ip, ctypes.c_int, ctypes.c_double, ctypes.c_double, _ip, _dp, _dp,
                                                _dp, _dp, _dp, ctypes.c_double, ctypes.c_int, _dp, ctypes.c_int]
            lib.dwf_oracle_pf_force.restype = ctypes.c_int
            lib.dwf_oracle_norm2.argtypes = [ctypes.c_long, _dp]
            lib.dwf_oracle_norm2.restype = ctypes.c_double
            _lib = lib
    return _lib


def default_threads() -> int:
    return int(os.environ.get("DWF_ORACLE_THREADS", os.cpu_count() or 1))


def _ints(v):
    return (ctypes.c_int * len(v))(*[int(a) for a in v])


def _ptr(a: np.ndarray):
    assert a.dtype == np.complex128 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _check_spinor(dims, Ls, psi):
    lx, ly, lz, lt = dims
    if psi.shape != (lt, lz, ly, lx, Ls, 4, 3):
        raise ValueError(f"spinor shape {psi.shape} does not match dims {dims} and Ls {Ls}")


def gamma() -> np.ndarray:
    """gamma_x, gamma_y, gamma_z, gamma_t, gamma5 as a (5, 4, 4) complex array."""
    out = np.zeros((5, 4, 4), dtype=np.complex128)
    _load().dwf_oracle_gamma(_ptr(out))
    return out


def dhop(dims, Ls, bc, U, psi, out_parity=2, dag=False, nthreads=None):
    """Wilson hopping term per s-slice; out_parity 0 = DhopEO, 1 = DhopOE, 2 = both."""
    U, psi = _c128(U), _c128(psi)
    _check_spinor(dims, Ls, psi)
    out = np.empty_like(psi)
    _load().dwf_oracle_dhop(_ints(dims), Ls, _ints(bc), _ptr(U), _ptr(psi), _ptr(out), int(out_parity), int(dag),
                            nthreads or default_threads())
    return out


def dhop_sites(dims, Ls, bc, U, psi, sites, dag=False, nthreads=None):
    """Dhop at the listed lexicographic 4D sites only: returns [len(sites), Ls, 4, 3]."""
    U, psi = _c128(U), _c128(psi)
    _check_spinor(dims, Ls, psi)
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    if sites.size and (sites.min() < 0 or sites.max() >= int(np.prod(dims))):
        raise ValueError("site index out of range")
    out = np.empty((sites.size, Ls, 4, 3), dtype=np.complex128)
    _load().dwf_oracle_dhop_sites(_ints(dims), Ls, _ints(bc), _ptr(U), _ptr(psi),
                                  sites.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), sites.size, _ptr(out),
                                  int(dag), nthreads or default_threads())
    return out


def mooee(dims, Ls, M5, mass, psi, dag=False, inverse=False, nthreads=None):
    """Mooee, Mooee^+, Mooee^-1 or (Mooee^+)^-1 on every 4D site."""
    psi = _c128(psi)
    _check_spinor(dims, Ls, psi)
    out = np.empty_like(psi)
    rc = _load().dwf_oracle_mooee(_ints(dims), Ls, M5, mass, _ptr(psi), _ptr(out), int(dag), int(inverse),
                                  nthreads or default_threads())
    if rc != 0:
        raise ArithmeticError("Mooee matrix is singular")
    return out


def m(dims, Ls, M5, mass, bc, U, psi, dag=False, nthreads=None):
    """Full operator M = Mooee - Dhop/2 (dag: M^+)."""
    U, psi = _c128(U), _c128(psi)
    _check_spinor(dims, Ls, psi)
    out = np.empty_like(psi)
    _load().dwf_oracle_m(_ints(dims), Ls, M5, mass, _ints(bc), _ptr(U), _ptr(psi), _ptr(out), int(dag),
                         nthreads or default_threads())
    return out


def mpc(dims, Ls, M5, mass, bc, U, psi, dag=False, nthreads=None):
    """Odd-site Schur complement Mpc (dag: Mpc^+); reads odd sites, zero on even sites."""
    U, psi = _c128(U), _c128(psi)
    _check_spinor(dims, Ls, psi)
    out = np.empty_like(psi)
    _load().dwf_oracle_mpc(_ints(dims), Ls, M5, mass, _ints(bc), _ptr(U), _ptr(psi), _ptr(out), int(dag),
                           nthreads or default_threads())
    return out


def mdagm(dims, Ls, M5, mass, bc, U, psi, nthreads=None):
    """Mpc^+ Mpc on odd sites."""
    U, psi = _c128(U), _c128(psi)
    _check_spinor(dims, Ls, psi)
    out = np.empty_like(psi)
    _load().dwf_oracle_mdagm(_ints(dims), Ls, M5, mass, _ints(bc), _ptr(U), _ptr(psi), _ptr(out),
                             nthreads or default_threads())
    return out


def schur_cg(dims, Ls, M5, mass, bc, U, b, x0=None, tol=1e-10, maxiter=10000, nthreads=None):
    """Solve M x = b by CG on the odd-site Schur system. Returns (x, iterations, true_resid, converged)."""
    U, b = _c128(U), _c128(b)
    _check_spinor(dims, Ls, b)
    x = np.zeros_like(b) if x0 is None else _c128(x0).copy()
    it = ctypes.c_int(0)
    res = ctypes.c_double(0.0)
    rc = _load().dwf_oracle_schur_cg(_ints(dims), Ls, M5, mass, _ints(bc), _ptr(U), _ptr(b), _ptr(x), tol,
                                     int(maxiter), ctypes.byref(it), ctypes.byref(res), nthreads or default_threads())
    return x, it.value, res.value, rc == 0


def force(dims, Ls, M5, mass, bc, U, psi, nthreads=None):
    """S = |M psi|^2, su(3) force F[t,z,y,x,mu,3,3] and ambient gradient G = dS/dReU + i dS/dImU."""
    U, psi = _c128(U), _c128(psi)
    _check_spinor(dims, Ls, psi)
    F = np.empty_like(U)
    G = np.empty_like(U)
    S = _load().dwf_oracle_force(_ints(dims), Ls, M5, mass, _ints(bc), _ptr(U), _ptr(psi), _ptr(F), _ptr(G),
                                 nthreads or default_threads())
    return S, F, G


def pf_force(dims, Ls, M5, mass, bc, U, phi, tol=1e-12, maxiter=100000, want_force=True, nthreads=None):
    """Pseudofermion action S = phi^+ (Mpc^+ Mpc)^-1 phi (odd sites of phi) and its link derivatives.

    Returns (S, X, F, G, iterations): X = (Mpc^+ Mpc)^-1 phi on odd sites (zero on even), F the su(3)
    force and G = dS/dRe U + i dS/dIm U in the gauge layout (None unless want_force); iterations
    is -1 if CG did not reach tol within maxiter.
    """
    U, phi = _c128(U), _c128(phi)
    _check_spinor(dims, Ls, phi)
    X = np.zeros_like(phi)
    F = np.empty_like(U) if want_force else None
    G = np.empty_like(U) if want_force else None
    S = ctypes.c_double(0.0)
    null = ctypes.POINTER(ctypes.c_double)()
    it = _load().dwf_oracle_pf_force(_ints(dims), Ls, M5, mass, _ints(bc), _ptr(U), _ptr(phi), _ptr(X),
                                     _ptr(F) if want_force else null, _ptr(G) if want_force else null, tol,
                                     int(maxiter), ctypes.byref(S), nthreads or default_threads())
    return S.value, X, F, G, it


def norm2(v) -> float:
    v = _c128(v)
    return float(_load().dwf_oracle_norm2(v.size, _ptr(v)))


def parity_mask(dims) -> np.ndarray:
    """Boolean [t,z,y,x] mask of odd sites, parity = (x+y+z+t) mod 2."""
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return ((x + y + z + t) % 2) == 1
