"""Domain decomposition of the 4D lattice over ranks: the host side of a multi-GPU hopping term.

The paper runs the domain wall operator on many GPUs (Section 3: weak scaling on 4-GPU nodes, an
Nsight-Systems profile in which face assembly kernels and the halo exchange overlap with the
interior compute). This module holds what that needs on the host, and no operator arithmetic:

* :class:`Partition`: a processor grid over the four dimensions, each rank's local block (origin
  and extents; every local extent even, so that local and global checkerboard parity agree), its
  forward and backward neighbour ranks, the face planes it sends, the boundary phase a face picks
  up when its hop crosses the global lattice edge, and the interior sites whose eight neighbours
  are all local (computable while the faces are in flight).
* :func:`exchange_faces`: the point-to-point exchange of the faces in one direction through
  ``torch.distributed`` (NCCL between GPUs, gloo on CPU ranks).

Face protocol (what each rank sends, per partitioned direction mu): its first plane
(x_mu = 0), projected to half spinors by the forward-hop projector, goes to the backward
neighbour, for whose last plane it is psi(x + mu); its last plane, projected by the backward-hop
projector, goes to the forward neighbour. A projected half spinor has 2 spins x 3 colours
complex = 12 reals per site and fifth-dimension slice, half of a full spinor. The links a
rank needs for its backward hops out of its first plane, U_mu(x - mu), belong to the backward
neighbour's last plane; they change only when the gauge field does, so they are exchanged once
with it (:meth:`Partition.gauge_face_sites`), not with every hopping application.

No GPU path exists yet (the library runs on one GPU with the wrap-around inside the kernel);
a GPU version gathers each face with a kernel into a contiguous local send buffer, exchanges it
by copies into the receiving GPU's own local buffers, and applies the received half spinors in
an exterior kernel after the interior kernel. Canonical fields are laid out
``[t, z, y, x, ...]`` with dims ``(Lx, Ly, Lz, Lt)``.
"""
from __future__ import annotations

import numpy as np

# canonical array axis of each direction mu (x, y, z, t) in [t, z, y, x, ...]
AXIS = (3, 2, 1, 0)


class Partition:
    """Rank `rank` of a processor grid procs = (Px, Py, Pz, Pt) over a lattice dims = (Lx, Ly, Lz, Lt).

    Ranks are numbered with x fastest. Each dims[mu] must be a multiple of procs[mu] with an even
    local extent."""

    def __init__(self, dims, procs, rank: int):
        self.dims = tuple(int(d) for d in dims)
        self.procs = tuple(int(p) for p in procs)
        if len(self.dims) != 4 or len(self.procs) != 4:
            raise ValueError("dims and procs have four entries (x, y, z, t)")
        for d, p in zip(self.dims, self.procs):
            if p < 1 or d % p or (d // p) % 2:
                raise ValueError(f"extent {d} does not split into {p} even blocks")
        self.size = int(np.prod(self.procs))
        if not 0 <= rank < self.size:
            raise ValueError("rank out of range")
        self.rank = rank
        self.local = tuple(d // p for d, p in zip(self.dims, self.procs))
        c, r = [], rank
        for p in self.procs:
            c.append(r % p)
            r //= p
        self.coords = tuple(c)
        self.origin = tuple(ci * li for ci, li in zip(self.coords, self.local))

    def rank_of(self, coords) -> int:
        r, stride = 0, 1
        for ci, p in zip(coords, self.procs):
            r += (ci % p) * stride
            stride *= p
        return r

    def neighbour(self, mu: int, fwd: bool) -> int:
        c = list(self.coords)
        c[mu] += 1 if fwd else -1
        return self.rank_of(c)

    def partitioned(self, mu: int) -> bool:
        return self.procs[mu] > 1

    def local_block(self, field: np.ndarray) -> np.ndarray:
        """This rank's block of a global canonical field [t, z, y, x, ...]."""
        sl = [slice(None)] * field.ndim
        for mu in range(4):
            sl[AXIS[mu]] = slice(self.origin[mu], self.origin[mu] + self.local[mu])
        return field[tuple(sl)]

    def face(self, local_field: np.ndarray, mu: int, last: bool) -> np.ndarray:
        """The plane x_mu = local extent - 1 (last) or x_mu = 0 of a local canonical field."""
        idx = self.local[mu] - 1 if last else 0
        return np.take(local_field, idx, axis=AXIS[mu])

    def send_phase(self, mu: int, last: bool, bc) -> int:
        """Boundary phase of the hop a face serves: bc[mu] if it crosses the global lattice edge.

        The first plane (sent backward) serves the forward hop out of the backward neighbour's last
        plane, which crosses the edge when this rank holds global x_mu = 0; the last plane (sent
        forward) crosses it when this rank holds global x_mu = L_mu - 1."""
        at_edge = self.coords[mu] == (self.procs[mu] - 1 if last else 0)
        return int(bc[mu]) if at_edge else 1

    def gauge_face_sites(self, mu: int):
        """(rank that sends, plane it sends): the links U_mu of the backward neighbour's last plane,
        which this rank's backward hops out of its first plane read."""
        return self.neighbour(mu, False), self.local[mu] - 1

    def interior_mask(self) -> np.ndarray:
        """Boolean [t, z, y, x] mask of local sites whose eight neighbours are all on this rank."""
        m = np.ones(tuple(self.local[mu] for mu in (3, 2, 1, 0)), dtype=bool)
        for mu in range(4):
            if self.partitioned(mu):
                sl = [slice(None)] * 4
                sl[AXIS[mu]] = 0
                m[tuple(sl)] = False
                sl[AXIS[mu]] = self.local[mu] - 1
                m[tuple(sl)] = False
        return m

    def face_sites(self, mu: int) -> int:
        """4D sites of one face plane in direction mu."""
        return int(np.prod(self.local)) // self.local[mu]


def exchange_faces(part: Partition, mu: int, first_plane, last_plane, group=None):
    """Send this rank's projected first plane backward and last plane forward in direction mu and
    receive the neighbours' (torch tensors, contiguous, the same shape on every rank).

    Returns (from_forward, from_backward): the forward neighbour's first plane (this rank's
    psi(x + mu) beyond its last plane) and the backward neighbour's last plane (psi(x - mu)
    before its first plane)."""
    import torch
    import torch.distributed as dist

    fwd, bwd = part.neighbour(mu, True), part.neighbour(mu, False)
    from_fwd = torch.empty_like(first_plane)
    from_bwd = torch.empty_like(last_plane)
    # tags: 2 mu for faces travelling backward, 2 mu + 1 forward (with two ranks in mu the forward
    # and backward neighbours are the same rank, and the tags keep the two messages apart)
    reqs = [dist.isend(first_plane.contiguous(), bwd, group=group, tag=2 * mu),
            dist.isend(last_plane.contiguous(), fwd, group=group, tag=2 * mu + 1),
            dist.irecv(from_fwd, fwd, group=group, tag=2 * mu),
            dist.irecv(from_bwd, bwd, group=group, tag=2 * mu + 1)]
    for r in reqs:
        r.wait()
    return from_fwd, from_bwd
