"""The software-managed device cache on the GPU (CUDA backend): more fields than the watermark
holds are paged through the device while the hopping term runs on them; every result equals the
same operator applied to device-resident fields, bit for bit, and the cache never holds more than
its watermark."""
import numpy as np
import pytest
import torch

from paper_2203_06777_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dwf():
    from paper_2203_06777_gb300 import dwf as mod

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mod.load()
    return mod


@pytest.mark.parametrize("prec", [0, 1])
def test_dhop_through_the_cache(dwf, prec):
    dims, Ls, nf = (8, 8, 4, 8), 8, 6
    op = dwf.GridDWF(dims, Ls, 1.8, 0.01)
    op.set_gauge(torch.from_numpy(synth.random_gauge(dims, seed=401, eps=0.3)).cuda())
    src = [op.pack(torch.from_numpy(synth.random_spinor(dims, Ls, seed=410 + k)).cuda(), prec, dwf.FULL)
           for k in range(nf)]
    ref = [op.dhop(s, dwf.FULL) for s in src]
    hin = [s.cpu().pin_memory() for s in src]
    hin_orig = [h.clone() for h in hin]
    hout = [torch.zeros_like(h).pin_memory() for h in hin]
    fbytes = hin[0].numel() * hin[0].element_size()
    cache = dwf.FieldCache(4 * fbytes)  # four of the twelve fields at a time
    del src
    torch.cuda.synchronize()
    for sweep in range(2):  # the second sweep in reverse order
        order = range(nf) if sweep == 0 else reversed(range(nf))
        for k in order:
            din = cache.device_view(hin[k], dwf.ACC_READ)
            dout = cache.device_view(hout[k], dwf.ACC_WRITE_DISCARD)
            op.dhop(din, dwf.FULL, out=dout)
            cache.close(hin[k])
            cache.close(hout[k])
    for k in range(nf):
        cache.open(hout[k], dwf.CPU_READ)
        assert torch.equal(hout[k], ref[k].cpu()), k
        cache.open(hin[k], dwf.CPU_READ)
    st = cache.stats()
    assert st["evictions"] > 0 and st["peak_resident"] <= 4 * fbytes and st["misses"] > nf
    # outputs were written back (on eviction or on the CPU view); inputs, only read, are unchanged
    assert st["copies_to_host"] >= nf
    assert all(torch.equal(hin[k], hin_orig[k]) for k in range(nf))
    cache.close_cache()
    op.close()
