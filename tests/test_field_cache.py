"""The software-managed device cache (grid_dwf_cache_*) on the CPU: a host backend stands in for
the device (its "device" buffers are host buffers, its copies memmove), so the state machine, the
LRU replacement with its high watermark, the advise priority, pinning by open views and the
write-back of newer device copies are checked without a GPU. The paper's Section 2.3 describes the
cache these follow (intents, states, watermark, least-recently-used victims, advise)."""
import ctypes

import numpy as np
import pytest

from paper_2203_06777_gb300 import dwf

N = 1024  # bytes per field


class HostBackend:
    def __init__(self):
        self.bufs = {}
        self.log = []
        B = dwf.CacheBackend

        def alloc(ctx, n, out):
            b = ctypes.create_string_buffer(n)
            addr = ctypes.addressof(b)
            self.bufs[addr] = b
            out[0] = addr
            self.log.append(("alloc", addr))
            return 0

        def free(ctx, p):
            self.log.append(("free", p))
            del self.bufs[p]
            return 0

        def to_device(ctx, d, h, n):
            ctypes.memmove(d, h, n)
            self.log.append(("h2d", d))
            return 0

        def to_host(ctx, h, d, n):
            ctypes.memmove(h, d, n)
            self.log.append(("d2h", d))
            return 0

        self._keep = (B._ALLOC(alloc), B._FREE(free), B._COPY(to_device), B._COPY(to_host))
        self.backend = B(None, *self._keep)

    def read(self, p):
        return bytes(self.bufs[p].raw)

    def write(self, p, data):
        ctypes.memmove(p, data, len(data))


@pytest.fixture()
def cache():
    be = HostBackend()
    c = dwf.FieldCache(3 * N, backend=be.backend)  # room for three fields
    yield c, be
    c.close_cache()


def fields(k):
    return [np.full(N, i + 1, dtype=np.uint8) for i in range(k)]


def test_states_and_data_motion(cache):
    c, be = cache
    (a,) = fields(1)
    d = c.open(a, dwf.ACC_READ)  # miss: allocate, copy in
    assert be.read(d) == a.tobytes()
    assert c.query(a) == (dwf.CACHE_CONSISTENT, 1, d)
    c.close(a)
    assert c.open(a, dwf.ACC_READ) == d and c.stats()["hits"] == 1  # no copy on a hit
    c.close(a)
    assert sum(1 for op, _ in be.log if op == "h2d") == 1
    d = c.open(a, dwf.ACC_WRITE)  # the kernel writes the device copy
    be.write(d, b"\x07" * N)
    c.close(a)
    assert c.query(a)[0] == dwf.CACHE_DEVICE_NEWER and a[0] == 1  # host stale until a CPU view
    assert c.open(a, dwf.CPU_READ) == a.ctypes.data and a[0] == 7 and c.query(a)[0] == dwf.CACHE_CONSISTENT
    c.open(a, dwf.CPU_WRITE)  # the host writes: the device copy becomes stale
    a[:] = 9
    assert c.query(a)[0] == dwf.CACHE_HOST_NEWER
    d = c.open(a, dwf.ACC_READ)  # stale device copy refreshed
    assert be.read(d) == b"\x09" * N
    c.close(a)
    d2 = c.open(a, dwf.ACC_WRITE_DISCARD)  # no copy in
    h2d = sum(1 for op, _ in be.log if op == "h2d")
    c.close(a)
    assert d2 == d and h2d == 2


def test_lru_eviction_writes_back_and_respects_the_watermark(cache):
    c, be = cache
    f = fields(5)
    devs = []
    for x in f[:3]:
        devs.append(c.open(x, dwf.ACC_WRITE))
        c.close(x)
    be.write(devs[0], b"\x55" * N)  # field 0 is newer on the device
    c.open(f[1], dwf.ACC_READ)  # touch 1: the LRU order is now 1, 2, 0 (0 least recent)
    c.close(f[1])
    c.open(f[3], dwf.ACC_READ)  # needs room: evicts field 0 (written back first)
    c.close(f[3])
    assert c.query(f[0])[0] == dwf.CACHE_EMPTY and f[0][0] == 0x55
    assert c.stats()["evictions"] == 1 and c.stats()["resident_bytes"] == 3 * N
    c.open(f[4], dwf.ACC_READ)  # next victim: field 2
    c.close(f[4])
    assert c.query(f[2])[0] == dwf.CACHE_EMPTY and c.query(f[1])[0] != dwf.CACHE_EMPTY
    assert c.stats()["peak_resident"] <= 3 * N


def test_open_views_pin_and_infrequent_fields_go_first(cache):
    c, be = cache
    f = fields(5)
    c.advise(f[2], dwf.ADVISE_INFREQUENT)
    for x in f[:3]:
        c.open(x, dwf.ACC_READ)
    c.close(f[1])
    c.close(f[2])
    # f[0] is pinned (open view); the infrequent f[2] goes before the LRU f[1]
    c.open(f[3], dwf.ACC_READ)
    assert c.query(f[2])[0] == dwf.CACHE_EMPTY and c.query(f[1])[0] != dwf.CACHE_EMPTY
    # f[0] and f[3] pinned, f[1] evictable: room for one more
    c.open(f[4], dwf.ACC_READ)
    assert c.query(f[1])[0] == dwf.CACHE_EMPTY
    # now f[0], f[3], f[4] are all pinned: a fourth field cannot fit
    with pytest.raises(dwf.GridDWFError) as e:
        c.open(f[1], dwf.ACC_READ)
    assert e.value.code == -3
    with pytest.raises(dwf.GridDWFError) as e:  # no CPU view of a field with open device views
        c.open(f[0], dwf.CPU_READ)
    assert e.value.code == -6


def test_flush_forget_and_sizes(cache):
    c, be = cache
    a, b = fields(2)
    d = c.open(a, dwf.ACC_WRITE)
    be.write(d, b"\x11" * N)
    c.close(a)
    c.flush()
    assert a[0] == 0x11 and c.query(a)[0] == dwf.CACHE_CONSISTENT
    d = c.open(b, dwf.ACC_WRITE)
    be.write(d, b"\x22" * N)
    c.close(b)
    c.forget(b)  # written back, entry and device buffer gone
    assert b[0] == 0x22 and c.stats()["resident_bytes"] == N
    with pytest.raises(dwf.GridDWFError):
        c.query(b)
    with pytest.raises(dwf.GridDWFError) as e:
        rc = c.lib.grid_dwf_cache_open(c._h, dwf._ptr(a.ctypes.data), N // 2, dwf.ACC_READ,
                                       ctypes.byref(ctypes.c_void_p()))
        c._check(rc, "open")
    assert e.value.code == -1  # a registered field reopened with another size
