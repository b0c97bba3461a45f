"""A lattice split into blocks along t, run on one GPU as separate operator handles: each block
projects its face planes (grid_dwf_face_project), the faces and the link faces are copied into the
neighbours' own buffers (the exchange of a multi-GPU run), and each block computes its interior
on one stream while the copies run on another, then its face planes from the received faces.
The result equals the hopping term of the whole lattice bit for bit (same FP32 operations), for
every block count, both parities and both signs, with the antiperiodic t boundary crossing the
global edge between the last and the first block."""
import numpy as np
import pytest
import torch

from paper_2203_06777_gb300 import halo, synth

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)


@pytest.fixture(scope="module")
def dwf():
    from paper_2203_06777_gb300 import dwf as mod

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mod.load()
    return mod


@pytest.mark.parametrize("nblk,Ls", [(2, 16), (3, 16), (2, 8), (4, 7)])
@pytest.mark.parametrize("prec", [1, 2, 3])
def test_t_split_blocks_match_the_whole_lattice(dwf, oracle_lib, nblk, Ls, prec):
    dims = (8, 4, 4, 4 * nblk)
    U = synth.random_gauge(dims, seed=601, eps=0.4)
    psi = synth.random_spinor(dims, Ls, seed=602)
    whole = dwf.GridDWF(dims, Ls, 1.8, 0.01, bc=BC)
    whole.set_gauge(torch.from_numpy(U).cuda())
    parts = [halo.Partition(dims, (1, 1, 1, nblk), k) for k in range(nblk)]
    ops = []
    for part in parts:
        op = dwf.GridDWF(part.local, Ls, 1.8, 0.01, bc=BC)
        op.set_gauge(torch.from_numpy(np.ascontiguousarray(part.local_block(U))).cuda())
        ops.append(op)
    comm, comp = torch.cuda.Stream(), torch.cuda.Stream()
    for p in (dwf.EVEN, dwf.ODD):
        links = [op.face_links(prec, p) for op in ops]  # once per gauge field and parity
        for dag in (False, True):
            ref = whole.unpack(whole.dhop(whole.pack(torch.from_numpy(psi).cuda(), prec, 1 - p), p, dag=dag),
                               subset=p).cpu().numpy()
            ins = [op.pack(torch.from_numpy(np.ascontiguousarray(part.local_block(psi))).cuda(), prec, 1 - p)
                   for op, part in zip(ops, parts)]
            outs = [op.field(prec, p, zero=True) for op in ops]
            torch.cuda.synchronize()
            with torch.cuda.stream(comm):  # face assembly and exchange into local receive buffers
                sends = [op.face_project(f, dag=dag, phase_first=part.send_phase(3, False, BC),
                                         phase_last=part.send_phase(3, True, BC))
                         for op, f, part in zip(ops, ins, parts)]
                recv_fwd = [sends[(k + 1) % nblk][0].clone() for k in range(nblk)]
                recv_bwd = [sends[(k - 1) % nblk][1].clone() for k in range(nblk)]
                link_bwd = [links[(k - 1) % nblk].clone() for k in range(nblk)]
                arrived = torch.cuda.Event()
                arrived.record(comm)
            with torch.cuda.stream(comp):  # interior while the faces travel, then the face planes
                for op, f, o in zip(ops, ins, outs):
                    op.dhop_region(f, p, dwf.REGION_INTERIOR, dag=dag, out=o)
                comp.wait_event(arrived)
                for k, (op, f, o) in enumerate(zip(ops, ins, outs)):
                    op.dhop_region(f, p, dwf.REGION_FACES, dag=dag, out=o, recv_fwd=recv_fwd[k],
                                   recv_bwd=recv_bwd[k], links_bwd=link_bwd[k])
            torch.cuda.synchronize()
            for op, o, part in zip(ops, outs, parts):
                got = op.unpack(o, subset=p).cpu().numpy()
                want = part.local_block(ref)
                mask = part.local_block(oracle_lib.parity_mask(dims)) == (p == dwf.ODD)
                assert np.array_equal(got[mask], want[mask]), (nblk, Ls, prec, p, dag)
    for op in ops:
        op.close()
    whole.close()


def test_region_calls_reject_bad_arguments(dwf):
    op = dwf.GridDWF((8, 4, 4, 4), 16, 1.8, 0.01)
    op.set_gauge(torch.from_numpy(synth.random_gauge((8, 4, 4, 4), seed=611)).cuda())
    f64 = op.field(dwf.FP64, dwf.ODD, zero=True)
    with pytest.raises(dwf.GridDWFError) as e:
        op.face_project(f64)
    assert e.value.code == -1  # FP64 fields have no block path
    f = op.field(dwf.FP32, dwf.ODD, zero=True)
    with pytest.raises(dwf.GridDWFError) as e:
        op.dhop_region(f, dwf.EVEN, dwf.REGION_FACES)  # faces without receive buffers
    assert e.value.code == -1
    with pytest.raises(dwf.GridDWFError) as e:
        op.face_project(f, phase_first=2)
    assert e.value.code == -1
    op.close()


@pytest.mark.parametrize("prec", [1, 2])
def test_interior_and_face_launches_write_only_their_sites(dwf, prec):
    """The interior launch writes every site off the two face planes and no other; the face launch
    writes the two planes and no other (sentinel bytes elsewhere survive)."""
    dims, Ls = (8, 4, 4, 6), 16
    op = dwf.GridDWF(dims, Ls, 1.8, 0.01, bc=BC)
    op.set_gauge(torch.from_numpy(synth.random_gauge(dims, seed=621, eps=0.4)).cuda())
    f = op.pack(torch.from_numpy(synth.random_spinor(dims, Ls, seed=622)).cuda(), prec, dwf.ODD)
    a, b = op.face_project(f)
    links = op.face_links(prec, dwf.EVEN)
    site_reals = op.half_reals // op.half_sites
    plane = dims[0] // 2 * dims[1] * dims[2]
    nplanes = dims[3]
    sentinel = torch.tensor(12345.0, dtype=f.dtype, device="cuda")
    for region in (dwf.REGION_INTERIOR, dwf.REGION_FACES):
        out = torch.full_like(f, float(sentinel))
        op.dhop_region(f, dwf.EVEN, region, out=out, recv_fwd=a, recv_bwd=b, links_bwd=links)
        torch.cuda.synchronize()
        # sites are stored in blocks of 4; a t-plane holds whole blocks here (plane = 64 sites)
        per_site = out.view(op.half_sites, site_reals)
        face = torch.zeros(op.half_sites, dtype=torch.bool, device="cuda")
        face[:plane] = True
        face[(nplanes - 1) * plane:] = True
        written = (per_site != sentinel).any(dim=1)
        untouched = (per_site == sentinel).all(dim=1)
        mine = face if region == dwf.REGION_FACES else ~face
        assert bool(written[mine].all()) and bool(untouched[~mine].all()), region
    op.close()
