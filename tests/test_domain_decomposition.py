"""Domain decomposition of the hopping term over two CPU ranks (gloo): the face protocol of
paper_2203_06777_gb300.halo reproduces the single-rank operator.

Each rank holds one half of the lattice (split in t, or in x), projects its two face planes to
half spinors (12 reals per site and slice: the rank-2 projector of the hop they serve, in an
orthonormal basis of its range), multiplies in the boundary phase where the hop crosses the global
edge, and exchanges them with torch.distributed point-to-point messages; the links of the backward
neighbour's last plane are exchanged once the same way. The rank then rebuilds the projected
neighbour spinors in two halo planes and applies the FP64 oracle's hopping term to its block plus
halos. Its block must equal the same block of the oracle's single-rank result to FP64 rounding.
With the halos filled with NaN (faces not yet arrived), the interior sites that
Partition.interior_mask names must already be exact, and only the face planes may be undefined:
the split that lets the interior compute overlap the exchange.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

BC = (1, 1, 1, -1)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _range_basis(gam, mu, sign):
    """4 x 2 orthonormal basis of the range of (1 + sign gamma_mu) / 2."""
    P = 0.5 * (np.eye(4) + sign * gam[mu])
    w, v = np.linalg.eigh(P)
    assert np.allclose(w, [0, 0, 1, 1], atol=1e-14)
    return v[:, w > 0.5]


def _halo_dhop(rank, dims, Ls, mu, dag, with_faces):
    import torch

    import oracle
    from paper_2203_06777_gb300 import halo, synth

    procs = [1, 1, 1, 1]
    procs[mu] = 2
    part = halo.Partition(dims, procs, rank)
    U = synth.random_gauge(dims, seed=501)  # every rank draws the global field and keeps its block
    psi = synth.random_spinor(dims, Ls, seed=502)
    Uloc, ploc = part.local_block(U), part.local_block(psi)
    gam = oracle.gamma()
    fwd_sign = +1 if dag else -1  # projector (1 + fwd_sign gamma_mu) of the forward hop
    Bf, Bb = _range_basis(gam, mu, fwd_sign), _range_basis(gam, mu, -fwd_sign)
    # faces: half spinors [.., Ls, 2, 3]
    h_first = np.einsum("ab,...bc->...ac", Bf.conj().T, part.face(ploc, mu, last=False)) * part.send_phase(mu, False, BC)
    h_last = np.einsum("ab,...bc->...ac", Bb.conj().T, part.face(ploc, mu, last=True)) * part.send_phase(mu, True, BC)
    assert h_first.shape[-3:] == (Ls, 2, 3) and h_first[..., 0, :, :].size * 2 == part.face_sites(mu) * 12
    tr = lambda a: torch.view_as_real(torch.from_numpy(np.ascontiguousarray(a)))
    from_fwd, from_bwd = halo.exchange_faces(part, mu, tr(h_first), tr(h_last))
    from_fwd = torch.view_as_complex(from_fwd).numpy()
    from_bwd = torch.view_as_complex(from_bwd).numpy()
    # links U_mu of the backward neighbour's last plane (once per gauge field)
    u_last = np.ascontiguousarray(part.face(Uloc, mu, last=True)[..., mu, :, :])
    _, u_from_bwd = halo.exchange_faces(part, mu, tr(np.zeros_like(u_last)), tr(u_last))
    u_from_bwd = torch.view_as_complex(u_from_bwd).numpy()

    # the block with one halo plane on each side of direction mu
    ax = halo.AXIS[mu]
    L = part.local[mu]
    hdims = list(part.local)
    hdims[mu] = L + 2
    psi_h = np.full(tuple(hdims[m] for m in (3, 2, 1, 0)) + (Ls, 4, 3), np.nan + 0j)
    U_h = np.zeros(tuple(hdims[m] for m in (3, 2, 1, 0)) + (4, 3, 3), dtype=complex)
    U_h[...] = np.eye(3)
    real = [slice(None)] * 4
    real[ax] = slice(1, L + 1)
    psi_h[tuple(real)] = ploc
    U_h[tuple(real)] = Uloc
    lo, hi = [slice(None)] * 4, [slice(None)] * 4
    lo[ax], hi[ax] = 0, L + 1
    U_lo = U_h[tuple(lo)]
    U_lo[..., mu, :, :] = u_from_bwd
    if with_faces:  # the rebuilt projected spinors Pi psi of the neighbours' planes
        psi_h[tuple(lo)] = np.einsum("ab,...bc->...ac", Bb, from_bwd)
        psi_h[tuple(hi)] = np.einsum("ab,...bc->...ac", Bf, from_fwd)
    bc_h = list(BC)
    bc_h[mu] = 1  # the halo planes' own wrap-around is never read by the block's sites
    out = oracle.dhop(tuple(hdims), Ls, tuple(bc_h), U_h, psi_h, dag=dag)[tuple(real)]
    ref = part.local_block(oracle.dhop(dims, Ls, BC, U, psi, dag=dag))
    return part, out, ref


def _worker(rank, world, port, mu, dag, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      DWF_ORACLE_THREADS="1")
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dims, Ls = ((4, 4, 2, 8) if mu == 3 else (8, 2, 4, 4)), 4
        part, out, ref = _halo_dhop(rank, dims, Ls, mu, dag, with_faces=True)
        err = float(np.abs(out - ref).max() / np.abs(ref).max())
        part, out_nan, _ = _halo_dhop(rank, dims, Ls, mu, dag, with_faces=False)
        inner = part.interior_mask()
        inner_err = float(np.abs(out_nan[inner] - ref[inner]).max() / np.abs(ref).max())
        faces_undefined = bool(np.all(np.isnan(out_nan[~inner])))
        q.put((rank, err, inner_err, faces_undefined, int(inner.sum()), int((~inner).sum())))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("mu,dag", [(3, False), (3, True), (0, False)])
def test_two_rank_halo_dhop_matches_single_rank_oracle(oracle_lib, mu, dag):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, mu, dag, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, err, inner_err, faces_undefined, n_in, n_face in res:
        assert err < 1e-13, (rank, err)
        assert inner_err < 1e-13, (rank, inner_err)
        assert faces_undefined
        assert n_in > 0 and n_face > 0


def test_partition_geometry():
    from paper_2203_06777_gb300 import halo

    p = halo.Partition((8, 4, 4, 12), (2, 1, 1, 3), rank=3)
    assert p.size == 6 and p.local == (4, 4, 4, 4) and p.coords == (1, 0, 0, 1) and p.origin == (4, 0, 0, 4)
    assert p.neighbour(0, True) == 2 and p.neighbour(0, False) == 2  # two ranks in x
    assert p.neighbour(3, True) == 5 and p.neighbour(3, False) == 1
    assert p.send_phase(3, False, BC) == 1 and p.send_phase(3, True, BC) == 1
    top = halo.Partition((8, 4, 4, 12), (2, 1, 1, 3), rank=5)
    assert top.send_phase(3, True, BC) == -1 and top.send_phase(3, False, BC) == 1
    bottom = halo.Partition((8, 4, 4, 12), (2, 1, 1, 3), rank=0)
    assert bottom.send_phase(3, False, BC) == -1
    m = p.interior_mask()
    assert m.shape == (4, 4, 4, 4) and m.sum() == 4 * 4 * 2 * 2  # x and t each lose two planes
    assert p.face_sites(3) == 64
    with pytest.raises(ValueError):
        halo.Partition((6, 4, 4, 4), (2, 1, 1, 1), rank=0)  # local extent 3 is odd
