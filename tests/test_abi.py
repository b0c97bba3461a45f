"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/grid_dwf.h declares.

No compute call is made here (there is no GPU on the build machine)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "grid_dwf.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(grid_dwf_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2203_06777_gb300 import _build

    return ctypes.CDLL(_build.build())


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("grid_dwf_create", "grid_dwf_set_gauge", "grid_dwf_dhop", "grid_dwf_mooee", "grid_dwf_m",
                 "grid_dwf_mpc", "grid_dwf_mdagm", "grid_dwf_cg", "grid_dwf_force", "grid_dwf_pack",
                 "grid_dwf_unpack", "grid_dwf_destroy", "grid_dwf_last_error", "grid_dwf_norm2"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_status_strings_are_host_only(lib):
    lib.grid_dwf_status_string.restype = ctypes.c_char_p
    lib.grid_dwf_status_string.argtypes = [ctypes.c_int]
    assert lib.grid_dwf_status_string(0) == b"ok"
    assert lib.grid_dwf_status_string(-4) == b"solver did not converge"


def test_invalid_create_rejected_before_any_device_work(lib):
    """Argument checks run on the host before any CUDA call: odd or tiny dims, Ls out of range,
    non-finite M5, bad boundary phases are refused with GRID_DWF_ERR_INVALID_ARG (-1)."""
    h = ctypes.c_void_p()
    f = lib.grid_dwf_create
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                  ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    dims = lambda *d: (ctypes.c_int * 4)(*d)
    bc = (ctypes.c_int * 4)(1, 1, 1, -1)
    assert f(dims(4, 4, 4, 3), 8, 1.8, 0.01, bc, 0, None, ctypes.byref(h)) == -1
    assert f(dims(4, 4, 4, 0), 8, 1.8, 0.01, bc, 0, None, ctypes.byref(h)) == -1
    assert f(dims(4, 4, 4, 4), 0, 1.8, 0.01, bc, 0, None, ctypes.byref(h)) == -1
    assert f(dims(4, 4, 4, 4), 129, 1.8, 0.01, bc, 0, None, ctypes.byref(h)) == -1
    assert f(dims(4, 4, 4, 4), 8, float("nan"), 0.01, bc, 0, None, ctypes.byref(h)) == -1
    assert f(dims(4, 4, 4, 4), 8, 5.0, 0.01, bc, 0, None, ctypes.byref(h)) == -1  # 5 - M5 = 0
    assert f(dims(4, 4, 4, 4), 8, 1.8, 0.01, (ctypes.c_int * 4)(1, 1, 1, 2), 0, None, ctypes.byref(h)) == -1
    assert h.value is None


def test_build_uses_sm103a_only():
    from paper_2203_06777_gb300 import _build

    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.NVCC_FLAGS)


def test_noalloc_rejects_partial_site_blocks_on_the_host(lib):
    """grid_dwf_inner_noalloc refuses an nsites that is not whole blocks of 4 sites before any CUDA
    call (the pointers below are never dereferenced): a partial block would be read past the end
    of a buffer sized for nsites sites."""
    f = lib.grid_dwf_inner_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_long, ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t]
    err = ctypes.create_string_buffer(256)
    fake = ctypes.c_void_p(1 << 20)  # aligned, never read
    for nsites in (1, 2, 3, 5, 6, 7, 4097):
        assert f(1, fake, None, nsites, 16, None, fake, err, 256) == -1
        assert b"multiple of 4" in err.value
    assert f(1, fake, None, -4, 16, None, fake, err, 256) == -1
    assert f(7, fake, None, 4, 16, None, fake, err, 256) == -1  # bad precision
