"""Python binding of libgrid_dwf.so: argument marshalling only.

Every step of the operator runs in the CUDA library; this module passes torch device pointers
and sizes through the C ABI declared in ``include/grid_dwf.h``, on torch's current CUDA stream.
There is no CPU fallback: :func:`load` raises if the library cannot be built or loaded, and
:class:`GridDWF` raises if no CUDA device is present.

Fields on the device are flat real tensors in the library's device layout (one checkerboard half
holds V/2 * Lsp * 24 reals with Lsp = Ls rounded up to even, a full field twice that); their
torch dtype selects the storage
precision: float64 -> FP64, float32 -> FP32, float16 -> FP16, bfloat16 -> BF16. Canonical
fields are complex128 tensors ``psi[t, z, y, x, s, spin, colour]`` and ``U[t, z, y, x, mu, a, b]``.
"""
from __future__ import annotations

import ctypes
import threading
from dataclasses import dataclass

import numpy as np
import torch

from . import _build

FP64, FP32, FP16, BF16 = 0, 1, 2, 3
EVEN, ODD, FULL = 0, 1, 2
CG_FP64, CG_MIXED_FP32, CG_MIXED_FP16, CG_MIXED_BF16 = 0, 1, 2, 3
# arithmetic of the FP64 hopping term: IEEE double, or float-float (pairs of FP32 numbers)
FP64_ARITH_NATIVE, FP64_ARITH_FLOAT_FLOAT = 0, 1

STATUS = {
    0: "ok",
    -1: "invalid argument",
    -2: "CUDA error",
    -3: "out of device memory",
    -4: "solver did not converge",
    -5: "non-finite value",
    -6: "output overlaps an input",
    -7: "no gauge field set",
}

_DTYPE_OF_PREC = {FP64: torch.float64, FP32: torch.float32, FP16: torch.float16, BF16: torch.bfloat16}
_PREC_OF_DTYPE = {v: k for k, v in _DTYPE_OF_PREC.items()}

_lock = threading.Lock()
_lib = None


class GridDWFError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)} ({code}): {msg}")
        self.code = code


class _CgStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("reliable_updates", ctypes.c_int), ("converged", ctypes.c_int),
                ("true_residual", ctypes.c_double), ("seconds", ctypes.c_double), ("flops", ctypes.c_double)]


class _CacheStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_ulonglong) for n in ("hits", "misses", "evictions", "cpu_opens", "copies_to_device",
                                                   "copies_to_host", "bytes_to_device", "bytes_to_host")] + \
               [("peak_resident", ctypes.c_size_t), ("resident_bytes", ctypes.c_size_t)]


class CacheBackend(ctypes.Structure):
    """Data motion of a FieldCache (grid_dwf_cache_backend): device allocation, free and the two
    copies as C callbacks returning 0 on success."""
    _ALLOC = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p))
    _FREE = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)
    _COPY = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t)
    _fields_ = [("ctx", ctypes.c_void_p), ("alloc", _ALLOC), ("free", _FREE), ("to_device", _COPY),
                ("to_host", _COPY)]


@dataclass
class CgStats:
    iterations: int
    reliable_updates: int
    converged: bool
    true_residual: float
    seconds: float
    flops: float


def library_path() -> str:
    return _build.LIB


def load(build: bool = True):
    """Load libgrid_dwf.so (building it first if it is missing or stale). Raises on failure."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build else _build.LIB
        lib = ctypes.CDLL(path)
        vp, ip, dp, i, d = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double
        sig = {
            "grid_dwf_create": [ip, i, d, d, ip, i, vp, ctypes.POINTER(vp)],
            "grid_dwf_destroy": [vp],
            "grid_dwf_set_stream": [vp, vp],
            "grid_dwf_set_fp64_arith": [vp, i],
            "grid_dwf_field_bytes": [vp, i, i, ctypes.POINTER(ctypes.c_size_t)],
            "grid_dwf_set_gauge": [vp, vp],
            "grid_dwf_pack": [vp, i, i, vp, vp],
            "grid_dwf_unpack": [vp, i, i, vp, vp],
            "grid_dwf_convert": [vp, i, i, i, vp, vp, d],
            "grid_dwf_dhop": [vp, i, vp, vp, i, i],
            "grid_dwf_mooee": [vp, i, i, vp, vp, i, i],
            "grid_dwf_m": [vp, i, vp, vp, i],
            "grid_dwf_mpc": [vp, i, vp, vp, i, vp],
            "grid_dwf_mdagm": [vp, i, vp, vp, vp, vp],
            "grid_dwf_norm2": [vp, i, i, vp, dp],
            "grid_dwf_inner": [vp, i, i, vp, vp, dp],
            "grid_dwf_cg": [vp, vp, vp, d, i, i, ctypes.POINTER(_CgStats)],
            "grid_dwf_force": [vp, i, vp, vp, vp, vp, dp],
            "grid_dwf_pf_force": [vp, vp, vp, d, i, i, i, vp, vp, dp, ctypes.POINTER(_CgStats)],
            "grid_dwf_pipe_peak": [i, vp, dp],
            "grid_dwf_face_bytes": [vp, i, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)],
            "grid_dwf_face_project": [vp, i, vp, i, i, i, vp, vp],
            "grid_dwf_face_links": [vp, i, i, vp],
            "grid_dwf_dhop_region": [vp, i, vp, vp, i, i, i, vp, vp, vp],
            "grid_dwf_cache_create": [ctypes.c_size_t, vp, vp, ctypes.POINTER(vp)],
            "grid_dwf_cache_destroy": [vp],
            "grid_dwf_cache_advise": [vp, vp, ctypes.c_size_t, i],
            "grid_dwf_cache_open": [vp, vp, ctypes.c_size_t, i, ctypes.POINTER(vp)],
            "grid_dwf_cache_close": [vp, vp],
            "grid_dwf_cache_flush": [vp],
            "grid_dwf_cache_forget": [vp, vp],
            "grid_dwf_cache_query": [vp, vp, ip, ip, ctypes.POINTER(vp)],
            "grid_dwf_cache_get_stats": [vp, ctypes.POINTER(_CacheStats)],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        lib.grid_dwf_last_error.argtypes = [vp]
        lib.grid_dwf_last_error.restype = ctypes.c_char_p
        lib.grid_dwf_status_string.argtypes = [i]
        lib.grid_dwf_status_string.restype = ctypes.c_char_p
        lib.grid_dwf_cache_last_error.argtypes = [vp]
        lib.grid_dwf_cache_last_error.restype = ctypes.c_char_p
        _lib = lib
        return lib


PEAK_FP64_FMA, PEAK_FP32_FMA, PEAK_FP32X2_FMA = 0, 1, 2


def pipe_peak(kind: int) -> float:
    """Measured FMA throughput of the current device in GFLOP/s (grid_dwf_pipe_peak): FP64,
    scalar FP32 or packed FP32x2 fused multiply-adds over all SMs, on torch's current stream."""
    lib = load()
    out = ctypes.c_double(0.0)
    rc = lib.grid_dwf_pipe_peak(int(kind), _ptr(torch.cuda.current_stream().cuda_stream), ctypes.byref(out))
    if rc != 0:
        raise GridDWFError(rc, "grid_dwf_pipe_peak failed")
    return out.value


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(int(t))


def _ints(v):
    return (ctypes.c_int * len(v))(*[int(a) for a in v])


def prec_of(t: torch.Tensor) -> int:
    try:
        return _PREC_OF_DTYPE[t.dtype]
    except KeyError:
        raise TypeError(f"unsupported field dtype {t.dtype}") from None


class GridDWF:
    """A 5D Shamir domain-wall operator on one GPU (the handle of the C ABI)."""

    def __init__(self, dims, Ls, M5=1.8, mass=0.01, bc=(1, 1, 1, -1), compress12=False, device=None,
                 fp64_arith=FP64_ARITH_NATIVE):
        if not torch.cuda.is_available():
            raise RuntimeError("GridDWF needs a CUDA device; there is no CPU fallback")
        self.lib = load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.dims = tuple(int(d) for d in dims)
        self.Ls = int(Ls)
        self.M5, self.mass = float(M5), float(mass)
        self.bc = tuple(int(b) for b in bc)
        self.compress12 = bool(compress12)
        self.half_sites = int(np.prod(self.dims)) // 2
        # device layout: Ls padded to even (slice pairs), so a half field holds V/2 * Lsp * 24 reals
        self.Ls_padded = self.Ls + (self.Ls & 1)
        self.half_reals = self.half_sites * self.Ls_padded * 24
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = self.lib.grid_dwf_create(_ints(self.dims), self.Ls, self.M5, self.mass, _ints(self.bc),
                                          int(self.compress12), _ptr(torch.cuda.current_stream().cuda_stream),
                                          ctypes.byref(h))
        if rc != 0:
            raise GridDWFError(rc, "grid_dwf_create rejected the parameters")
        self._h = h
        self.fp64_arith = FP64_ARITH_NATIVE
        if fp64_arith != FP64_ARITH_NATIVE:
            self.set_fp64_arith(fp64_arith)

    # -------------------------------------------------------------- plumbing
    def close(self):
        if getattr(self, "_h", None):
            self.lib.grid_dwf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _call(self, name, *args):
        self.lib.grid_dwf_set_stream(self._h, _ptr(torch.cuda.current_stream(self.device).cuda_stream))
        rc = getattr(self.lib, name)(self._h, *args)
        if rc != 0:
            raise GridDWFError(rc, f"{name}: {self.lib.grid_dwf_last_error(self._h).decode()}")
        return rc

    def set_fp64_arith(self, mode: int):
        """Arithmetic of every FP64 hopping-term application on this handle (grid_dwf_set_fp64_arith):
        FP64_ARITH_NATIVE (IEEE double) or FP64_ARITH_FLOAT_FLOAT (float-float, ~46 bits)."""
        rc = self.lib.grid_dwf_set_fp64_arith(self._h, int(mode))
        if rc != 0:
            raise GridDWFError(rc, f"grid_dwf_set_fp64_arith: {self.lib.grid_dwf_last_error(self._h).decode()}")
        self.fp64_arith = int(mode)

    def _subset_of(self, t: torch.Tensor) -> int:
        if t.numel() == self.half_reals:
            return EVEN
        if t.numel() == 2 * self.half_reals:
            return FULL
        raise ValueError(f"field of {t.numel()} reals is neither a half ({self.half_reals}) nor a full field")

    def _check_field(self, t: torch.Tensor):
        if not isinstance(t, torch.Tensor) or t.device != self.device or not t.is_contiguous():
            raise ValueError("fields must be contiguous tensors on the operator's CUDA device")
        return prec_of(t)

    def field(self, prec=FP64, subset=ODD, zero=False) -> torch.Tensor:
        n = self.half_reals * (2 if subset == FULL else 1)
        alloc = torch.zeros if zero else torch.empty
        return alloc(n, dtype=_DTYPE_OF_PREC[prec], device=self.device)

    def canonical_shape(self):
        lx, ly, lz, lt = self.dims
        return (lt, lz, ly, lx, self.Ls, 4, 3)

    # -------------------------------------------------------------- data movement
    def set_gauge(self, U):
        """U: canonical complex128 gauge field (torch tensor on host or device, or numpy)."""
        if isinstance(U, np.ndarray):
            U = torch.from_numpy(np.ascontiguousarray(U, dtype=np.complex128))
        lx, ly, lz, lt = self.dims
        if U.dtype != torch.complex128 or tuple(U.shape) != (lt, lz, ly, lx, 4, 3, 3):
            raise ValueError("U must be complex128 with shape [t, z, y, x, 4, 3, 3]")
        U = U.contiguous()
        self._call("grid_dwf_set_gauge", _ptr(U))
        if U.device.type == "cpu":
            torch.cuda.current_stream(self.device).synchronize()

    def pack(self, psi: torch.Tensor, prec=FP64, subset=FULL, out=None) -> torch.Tensor:
        """Canonical complex128 spinor (device) -> device-layout field of prec/subset."""
        if psi.dtype != torch.complex128 or tuple(psi.shape) != self.canonical_shape():
            raise ValueError("psi must be complex128 with shape [t, z, y, x, Ls, 4, 3]")
        psi = psi.to(self.device).contiguous()
        out = self.field(prec, subset) if out is None else out
        self._call("grid_dwf_pack", prec, subset, _ptr(psi), _ptr(out))
        return out

    def unpack(self, f: torch.Tensor, subset=None, out=None) -> torch.Tensor:
        """Device-layout field -> canonical complex128 tensor (sites outside the subset are zero)."""
        prec = self._check_field(f)
        if subset is None:
            if self._subset_of(f) != FULL:
                raise ValueError("unpacking a half field needs subset=EVEN or subset=ODD")
            subset = FULL
        if out is None:
            out = torch.zeros(self.canonical_shape(), dtype=torch.complex128, device=self.device)
        self._call("grid_dwf_unpack", prec, subset, _ptr(f), _ptr(out))
        return out

    def convert(self, f: torch.Tensor, prec, scale=1.0, out=None) -> torch.Tensor:
        src = self._check_field(f)
        subset = self._subset_of(f)
        out = self.field(prec, subset) if out is None else out
        self._call("grid_dwf_convert", src, prec, subset, _ptr(f), _ptr(out), float(scale))
        return out

    # -------------------------------------------------------------- operators
    def dhop(self, f: torch.Tensor, parity=FULL, dag=False, out=None) -> torch.Tensor:
        """parity EVEN: DhopEO (odd half in -> even half out); ODD: DhopOE; FULL: full fields."""
        prec = self._check_field(f)
        out = torch.empty_like(f) if out is None else out
        self._call("grid_dwf_dhop", prec, _ptr(f), _ptr(out), int(parity), int(dag))
        return out

    # ---- a block of a lattice split in t (see grid_dwf_face_project / grid_dwf_dhop_region)

    def face_buffers(self, prec):
        """Empty (face, link face) device buffers of this block's sizes, as uint8 tensors."""
        fb, lb = ctypes.c_size_t(), ctypes.c_size_t()
        rc = self.lib.grid_dwf_face_bytes(self._h, prec, ctypes.byref(fb), ctypes.byref(lb))
        if rc != 0:
            raise GridDWFError(rc, "grid_dwf_face_bytes")
        return (torch.empty(fb.value, dtype=torch.uint8, device=self.device),
                torch.empty(lb.value, dtype=torch.uint8, device=self.device))

    def face_project(self, f_half: torch.Tensor, dag=False, phase_first=1, phase_last=1):
        """(send_first, send_last): this block's first and last t-planes of the input half field,
        projected for the previous and the next block's hops."""
        prec = self._check_field(f_half)
        a, _ = self.face_buffers(prec)
        b = torch.empty_like(a)
        self._call("grid_dwf_face_project", prec, _ptr(f_half), int(dag), int(phase_first), int(phase_last), _ptr(a),
                   _ptr(b))
        return a, b

    def face_links(self, prec, out_parity):
        """The links U_t of this block's last t-plane read by the next block's hops of out_parity."""
        _, links = self.face_buffers(prec)
        self._call("grid_dwf_face_links", prec, int(out_parity), _ptr(links))
        return links

    def dhop_region(self, f_half: torch.Tensor, out_parity, region, dag=False, out=None, recv_fwd=None,
                    recv_bwd=None, links_bwd=None) -> torch.Tensor:
        """The hop on this block's interior (REGION_INTERIOR) or its two face planes (REGION_FACES,
        with the neighbours' faces and link face)."""
        prec = self._check_field(f_half)
        out = torch.empty_like(f_half) if out is None else out
        self._call("grid_dwf_dhop_region", prec, _ptr(f_half), _ptr(out), int(out_parity), int(dag), int(region),
                   _ptr(recv_fwd), _ptr(recv_bwd), _ptr(links_bwd))
        return out

    def mooee(self, f: torch.Tensor, dag=False, inverse=False, out=None) -> torch.Tensor:
        prec = self._check_field(f)
        subset = self._subset_of(f)
        out = torch.empty_like(f) if out is None else out
        self._call("grid_dwf_mooee", prec, subset, _ptr(f), _ptr(out), int(dag), int(inverse))
        return out

    def m(self, f: torch.Tensor, dag=False, out=None) -> torch.Tensor:
        prec = self._check_field(f)
        out = torch.empty_like(f) if out is None else out
        self._call("grid_dwf_m", prec, _ptr(f), _ptr(out), int(dag))
        return out

    def mpc(self, f: torch.Tensor, dag=False, out=None, tmp_even=None) -> torch.Tensor:
        prec = self._check_field(f)
        out = torch.empty_like(f) if out is None else out
        self._call("grid_dwf_mpc", prec, _ptr(f), _ptr(out), int(dag), _ptr(tmp_even))
        return out

    def mdagm(self, f: torch.Tensor, out=None, tmp_odd=None, tmp_even=None) -> torch.Tensor:
        prec = self._check_field(f)
        out = torch.empty_like(f) if out is None else out
        self._call("grid_dwf_mdagm", prec, _ptr(f), _ptr(out), _ptr(tmp_odd), _ptr(tmp_even))
        return out

    def norm2(self, f: torch.Tensor) -> float:
        prec = self._check_field(f)
        r = ctypes.c_double()
        self._call("grid_dwf_norm2", prec, self._subset_of(f), _ptr(f), ctypes.byref(r))
        return r.value

    def inner(self, a: torch.Tensor, b: torch.Tensor) -> complex:
        prec = self._check_field(a)
        r = (ctypes.c_double * 2)()
        self._call("grid_dwf_inner", prec, self._subset_of(a), _ptr(a), _ptr(b), r)
        return complex(r[0], r[1])

    def cg(self, b: torch.Tensor, x: torch.Tensor | None = None, tol=1e-10, maxiter=10000, mode=CG_FP64,
           raise_on_fail=True):
        """Solve M x = b (full FP64 fields) via the odd-site Schur complement. Returns (x, CgStats)."""
        if self._check_field(b) != FP64 or self._subset_of(b) != FULL:
            raise ValueError("cg needs a full FP64 right-hand side")
        x = torch.zeros_like(b) if x is None else x
        st = _CgStats()
        self.lib.grid_dwf_set_stream(self._h, _ptr(torch.cuda.current_stream(self.device).cuda_stream))
        rc = self.lib.grid_dwf_cg(self._h, _ptr(b), _ptr(x), float(tol), int(maxiter), int(mode), ctypes.byref(st))
        stats = CgStats(st.iterations, st.reliable_updates, bool(st.converged), st.true_residual, st.seconds, st.flops)
        if rc != 0 and (raise_on_fail or rc != -4):
            raise GridDWFError(rc, f"grid_dwf_cg: {self.lib.grid_dwf_last_error(self._h).decode()}")
        return x, stats

    def force(self, psi_field: torch.Tensor, want_F=True, want_G=True, chi=None):
        """S = |M psi|^2, su(3) force F and ambient gradient G (canonical complex128, device)."""
        prec = self._check_field(psi_field)
        lx, ly, lz, lt = self.dims
        shape = (lt, lz, ly, lx, 4, 3, 3)
        F = torch.empty(shape, dtype=torch.complex128, device=self.device) if want_F else None
        G = torch.empty(shape, dtype=torch.complex128, device=self.device) if want_G else None
        S = ctypes.c_double()
        self._call("grid_dwf_force", prec, _ptr(psi_field), _ptr(chi), _ptr(F), _ptr(G), ctypes.byref(S))
        return S.value, F, G


    def pf_force(self, phi: torch.Tensor, x: torch.Tensor | None = None, tol=1e-10, maxiter=10000, mode=CG_FP64,
                 precision=FP64, want_F=True, want_G=True, raise_on_fail=True):
        """Pseudofermion action S = phi^+ (Mpc^+ Mpc)^-1 phi of an odd FP64 half field phi, with
        its su(3) force F and ambient gradient G (canonical complex128, device) and the solution
        X = (Mpc^+ Mpc)^-1 phi (odd FP64 half field). Returns (S, F, G, X, CgStats)."""
        if self._check_field(phi) != FP64 or self._subset_of(phi) == FULL:
            raise ValueError("pf_force needs an odd FP64 half field phi")
        x = torch.zeros_like(phi) if x is None else x
        lx, ly, lz, lt = self.dims
        shape = (lt, lz, ly, lx, 4, 3, 3)
        F = torch.empty(shape, dtype=torch.complex128, device=self.device) if want_F else None
        G = torch.empty(shape, dtype=torch.complex128, device=self.device) if want_G else None
        S = ctypes.c_double()
        st = _CgStats()
        self.lib.grid_dwf_set_stream(self._h, _ptr(torch.cuda.current_stream(self.device).cuda_stream))
        rc = self.lib.grid_dwf_pf_force(self._h, _ptr(phi), _ptr(x), float(tol), int(maxiter), int(mode),
                                        int(precision), _ptr(F), _ptr(G), ctypes.byref(S), ctypes.byref(st))
        stats = CgStats(st.iterations, st.reliable_updates, bool(st.converged), st.true_residual, st.seconds, st.flops)
        if rc != 0 and (raise_on_fail or rc != -4):
            raise GridDWFError(rc, f"grid_dwf_pf_force: {self.lib.grid_dwf_last_error(self._h).decode()}")
        return S.value, F, G, x, stats


class DWFAction(torch.autograd.Function):
    """S = |M[U] psi|^2 with hand-written adjoints: dS/dpsi via M^+ (the library's dag kernels)
    and dS/dU via the force kernel. psi and U are canonical complex128 CUDA tensors; gradients
    follow torch's convention for real losses, dS/dRe z + i dS/dIm z."""

    @staticmethod
    def forward(ctx, psi, U, op: GridDWF, prec=FP64):
        op.set_gauge(U.detach())
        f = op.pack(psi.detach(), prec, FULL)
        chi = op.m(f)
        S = op.norm2(chi)
        ctx.op, ctx.prec = op, prec
        ctx.save_for_backward(f, chi, U.detach())
        return torch.tensor(S, dtype=torch.float64, device=psi.device)

    @staticmethod
    def backward(ctx, gS):
        f, chi, U = ctx.saved_tensors
        op = ctx.op
        g = gS.to(torch.float64)
        grad_psi = grad_U = None
        # the handle may hold other links by now (any forward call since this one re-uploads)
        op.set_gauge(U)
        if ctx.needs_input_grad[0]:
            grad_psi = op.unpack(op.m(chi, dag=True)) * (2.0 * g)
        if ctx.needs_input_grad[1]:
            _, _, G = op.force(f, want_F=False, want_G=True)
            grad_U = G * g
        return grad_psi, grad_U, None, None


def dwf_action(psi, U, op: GridDWF, prec=FP64):
    return DWFAction.apply(psi, U, op, prec)


class PseudofermionAction(torch.autograd.Function):
    """S = phi^+ (Mpc[U]^+ Mpc[U])^-1 phi for the odd sites of phi, differentiated through the
    solve: dS/dU from the library's pseudofermion force (G), dS/dphi = 2 (Mpc^+ Mpc)^-1 phi
    (odd sites). phi and U are canonical complex128 CUDA tensors; torch's convention for real
    losses, dS/dRe z + i dS/dIm z."""

    @staticmethod
    def forward(ctx, phi, U, op: GridDWF, tol=1e-12, mode=CG_FP64):
        op.set_gauge(U.detach())
        f = op.pack(phi.detach(), FP64, ODD)
        S, _, G, X, _ = op.pf_force(f, tol=tol, mode=mode, want_F=False, want_G=True)
        ctx.save_for_backward(op.unpack(X, subset=ODD), G)
        return torch.tensor(S, dtype=torch.float64, device=phi.device)

    @staticmethod
    def backward(ctx, gS):
        X, G = ctx.saved_tensors
        g = gS.to(torch.float64)
        grad_phi = 2.0 * g * X if ctx.needs_input_grad[0] else None
        grad_U = G * g if ctx.needs_input_grad[1] else None
        return grad_phi, grad_U, None, None, None


def pseudofermion_action(phi, U, op: GridDWF, tol=1e-12, mode=CG_FP64):
    return PseudofermionAction.apply(phi, U, op, tol, mode)


# ---------------------------------------------------------------- software-managed device cache

REGION_INTERIOR, REGION_FACES = 0, 1
CPU_READ, CPU_WRITE, ACC_READ, ACC_WRITE, ACC_WRITE_DISCARD = 0, 1, 2, 3, 4
ADVISE_NORMAL, ADVISE_INFREQUENT = 0, 1
CACHE_EMPTY, CACHE_CONSISTENT, CACHE_HOST_NEWER, CACHE_DEVICE_NEWER = 0, 1, 2, 3


class _DeviceArray:
    """A raw device buffer presented to torch through the CUDA array interface (no copy)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None, "stream": None}


_TYPESTR = {torch.float64: "<f8", torch.float32: "<f4", torch.float16: "<f2"}


class FieldCache:
    """Host fields paged through a bounded device footprint (grid_dwf_cache_*): views with an
    access intent move whole fields between host and device; least recently used fields are
    evicted, infrequently used (advised) ones first. Host fields are CPU tensors (pinned for
    asynchronous copies) or NumPy arrays. The copies run on `stream` (default: torch's current
    stream when the cache is created); kernels that use a view on another stream must be ordered
    after the open on that stream. With a CacheBackend the data motion is the caller's (no GPU
    needed)."""

    def __init__(self, high_watermark: int, backend: CacheBackend | None = None, stream=None):
        self.lib = load()
        self._backend = backend  # keeps the callbacks alive
        h = ctypes.c_void_p()
        if stream is None and backend is None:
            stream = torch.cuda.current_stream().cuda_stream
        rc = self.lib.grid_dwf_cache_create(int(high_watermark), _ptr(stream) if stream else None,
                                            ctypes.byref(backend) if backend is not None else None, ctypes.byref(h))
        if rc != 0:
            raise GridDWFError(rc, "grid_dwf_cache_create failed")
        self._h = h

    def close_cache(self):
        if getattr(self, "_h", None):
            self.lib.grid_dwf_cache_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close_cache()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != 0:
            raise GridDWFError(rc, f"{what}: {self.lib.grid_dwf_cache_last_error(self._h).decode()}")

    @staticmethod
    def _host(t):
        if isinstance(t, torch.Tensor):
            assert t.device.type == "cpu" and t.is_contiguous()
            return t.data_ptr(), t.numel() * t.element_size()
        return t.ctypes.data, t.nbytes  # numpy

    def advise(self, host, advice):
        p, n = self._host(host)
        self._check(self.lib.grid_dwf_cache_advise(self._h, _ptr(p), n, advice), "advise")

    def open(self, host, intent) -> int:
        """Open a view; returns the device pointer (accelerator intents) or the host pointer."""
        p, n = self._host(host)
        out = ctypes.c_void_p()
        self._check(self.lib.grid_dwf_cache_open(self._h, _ptr(p), n, intent, ctypes.byref(out)), "open")
        return out.value

    def device_view(self, host: torch.Tensor, intent) -> torch.Tensor:
        """Open an accelerator view and wrap it as a CUDA tensor of the host tensor's shape."""
        ptr = self.open(host, intent)
        return torch.as_tensor(_DeviceArray(ptr, host.shape, _TYPESTR[host.dtype]), device="cuda")

    def close(self, host):
        p, _ = self._host(host)
        self._check(self.lib.grid_dwf_cache_close(self._h, _ptr(p)), "close")

    def flush(self):
        self._check(self.lib.grid_dwf_cache_flush(self._h), "flush")

    def forget(self, host):
        p, _ = self._host(host)
        self._check(self.lib.grid_dwf_cache_forget(self._h, _ptr(p)), "forget")

    def query(self, host):
        p, _ = self._host(host)
        st, views, dev = ctypes.c_int(), ctypes.c_int(), ctypes.c_void_p()
        self._check(self.lib.grid_dwf_cache_query(self._h, _ptr(p), ctypes.byref(st), ctypes.byref(views),
                                                  ctypes.byref(dev)), "query")
        return st.value, views.value, dev.value

    def stats(self) -> dict:
        st = _CacheStats()
        self._check(self.lib.grid_dwf_cache_get_stats(self._h, ctypes.byref(st)), "stats")
        return {n: getattr(st, n) for n, _ in _CacheStats._fields_}
