"""Domain decomposition of one periodic lattice (Sec. V-A).

The paper's code splits the lattice into processor domains that exchange
their boundary points with the neighbouring domains after each step.  Here
each sub-domain is an ordinary ``qla.Grid`` on its block of the lattice plus
a halo of ``halo`` ghost cells on every side.  The grid steps as a periodic
lattice of its own; the wrap-around corrupts only the halo, at most four
cells deeper per step (U_x and U_y each reach four cells), plus one ring whose
potential angles (Eq. 2e13) see a wrapped neighbour of n.  So the interior
stays exact for ``k`` steps when ``halo >= 4 k + 1``, after which the halos
are refilled from the neighbours' interiors.

The refill runs in two phases: strips along x over the interior rows, then
strips along y over the full extended width (carrying the x halos just
received), so the corner cells come along without diagonal messages.  Strips
leave and enter a grid through ``qla_pack_box`` / ``qla_unpack_box``
(contiguous device buffers, the library's own kernels); between sub-domains
they travel by a transport:

* ``LocalTransport``: every sub-domain in this process (several on one GPU);
  a strip is unpacked straight from the sender's buffer.
* ``DistTransport``: one sub-domain per rank of a ``torch.distributed``
  process group; strips go by point-to-point send/recv (NCCL for device
  buffers), and the energy is an FP64 all-reduce of the interior sums.

``Partition`` is pure host logic (block sizes, neighbours, the strips of each
phase) and the exchange is written against any sub-domain object with
``pack(box)``, ``unpack(box, buf)`` and ``step(k)``, so it also runs with
host-side sub-domains.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def halo_for(steps_per_exchange: int) -> int:
    """Ghost cells per side for k steps between exchanges: 4k + 1 suffice;
    rounded up to a multiple of 4 so that widths stay multiples of 4 (the
    packed marching kernel's row chunks)."""
    need = 4 * int(steps_per_exchange) + 1
    return (need + 3) // 4 * 4


def _splits(n, parts):
    """Block sizes of n sites over `parts` blocks, as even as possible."""
    base, extra = divmod(n, parts)
    return [base + (1 if b < extra else 0) for b in range(parts)]


@dataclass(frozen=True)
class Box:
    """A rectangle of sites in a sub-domain's extended (haloed) lattice."""
    i0: int
    j0: int
    w: int
    h: int


@dataclass(frozen=True)
class Transfer:
    """One strip of one exchange phase: this rank's `send` box goes to
    `peer`, whose halo box `recv` (in the peer's coordinates) it fills.
    `tag` orders the messages between a pair of ranks."""
    peer: int
    send: Box
    recv: Box
    tag: int


class Partition:
    """A periodic nx x ny lattice split into px x py blocks with `halo`
    ghost cells per side.  Rank r owns block (r % px, r // px)."""

    def __init__(self, nx, ny, px, py, halo):
        self.nx, self.ny, self.px, self.py, self.halo = int(nx), int(ny), int(px), int(py), \
            int(halo)
        if min(self.px, self.py) < 1 or self.halo < 1:
            raise ValueError("need px, py >= 1 and halo >= 1")
        self.ws = _splits(self.nx, self.px)
        self.hs = _splits(self.ny, self.py)
        if min(self.ws) < self.halo or min(self.hs) < self.halo:
            raise ValueError("blocks (%d x %d at least) must be at least the halo (%d) wide"
                             % (min(self.ws), min(self.hs), self.halo))
        self.x0 = np.concatenate([[0], np.cumsum(self.ws)[:-1]]).astype(int).tolist()
        self.y0 = np.concatenate([[0], np.cumsum(self.hs)[:-1]]).astype(int).tolist()

    @property
    def size(self):
        return self.px * self.py

    def coords(self, rank):
        return rank % self.px, rank // self.px

    def rank_of(self, bx, by):
        return (by % self.py) * self.px + (bx % self.px)

    def block(self, rank):
        """Interior (i0, j0, w, h) of `rank` in global coordinates."""
        bx, by = self.coords(rank)
        return self.x0[bx], self.y0[by], self.ws[bx], self.hs[by]

    def extended(self, rank):
        """(nx, ny) of the rank's haloed lattice."""
        _, _, w, h = self.block(rank)
        return w + 2 * self.halo, h + 2 * self.halo

    def origin(self, rank):
        """Global site of the extended lattice's site (0, 0)."""
        i0, j0, _, _ = self.block(rank)
        return (i0 - self.halo) % self.nx, (j0 - self.halo) % self.ny

    def interior(self, rank):
        _, _, w, h = self.block(rank)
        return Box(self.halo, self.halo, w, h)

    def phases(self, rank):
        """The transfers this rank sends, phase by phase: [x strips, y strips]."""
        g = self.halo
        bx, by = self.coords(rank)
        _, _, w, h = self.block(rank)
        east, west = self.rank_of(bx + 1, by), self.rank_of(bx - 1, by)
        north, south = self.rank_of(bx, by + 1), self.rank_of(bx, by - 1)
        w_west = self.ws[(bx - 1) % self.px]
        h_south = self.hs[(by - 1) % self.py]
        x = [
            # the last g interior columns fill the east neighbour's west halo
            Transfer(east, Box(w, g, g, h), Box(0, g, g, h), 0),
            # the first g interior columns fill the west neighbour's east halo
            Transfer(west, Box(g, g, g, h), Box(g + w_west, g, g, h), 1),
        ]
        y = [
            Transfer(north, Box(0, h, w + 2 * g, g), Box(0, 0, w + 2 * g, g), 2),
            Transfer(south, Box(0, g, w + 2 * g, g), Box(0, g + h_south, w + 2 * g, g), 3),
        ]
        return [x, y]

    def receives(self, rank, phase):
        """The (peer, box, tag) this rank receives in `phase`, in the order
        its peers send them."""
        out = []
        for peer in range(self.size):
            for t in self.phases(peer)[phase]:
                if t.peer == rank:
                    out.append((peer, t.recv, t.tag))
        return out


class LocalTransport:
    """All sub-domains live in this process (``subs``: rank -> sub-domain)."""

    def exchange(self, part, subs):
        for phase in (0, 1):
            for rank in sorted(subs):
                for t in part.phases(rank)[phase]:
                    buf = subs[rank].pack(t.send)
                    subs[t.peer].unpack(t.recv, buf)

    def allreduce_sum(self, value):
        return float(value)


class DistTransport:
    """One sub-domain per rank of the default torch.distributed group.
    ``device``: where strip buffers live (a CUDA device for NCCL, "cpu" for
    gloo)."""

    def __init__(self, device=None):
        import torch.distributed as dist
        self.dist = dist
        self.rank = dist.get_rank()
        self.device = device

    def exchange(self, part, subs):
        dist = self.dist
        me = subs[self.rank]
        for phase in (0, 1):
            sends = part.phases(self.rank)[phase]
            recvs = part.receives(self.rank, phase)
            ops, bufs, local = [], [], []
            for t in sends:
                buf = me.pack(t.send)
                if t.peer == self.rank:
                    local.append((t, buf))
                else:
                    ops.append(dist.P2POp(dist.isend, buf, t.peer, tag=t.tag))
                    bufs.append(buf)
            incoming = []
            for peer, box, tag in recvs:
                if peer == self.rank:
                    continue
                buf = me.empty_box(box)
                ops.append(dist.P2POp(dist.irecv, buf, peer, tag=tag))
                incoming.append((box, buf))
            if ops:
                for req in dist.batch_isend_irecv(ops):
                    req.wait()
            for t, buf in local:
                me.unpack(t.recv, buf)
            for box, buf in incoming:
                me.unpack(box, buf)

    def allreduce_sum(self, value):
        import torch
        t = torch.tensor([float(value)], dtype=torch.float64,
                         device=self.device if self.device is not None else "cpu")
        self.dist.all_reduce(t)
        return float(t.item())


class GridSub:
    """A sub-domain backed by a ``qla.Grid`` on the rank's extended block."""

    def __init__(self, part, rank, delta=1.0, precision="fp64", te_only=False, **grid_kw):
        from . import qla
        self.part, self.rank = part, rank
        nx, ny = part.extended(rank)
        self.grid = qla.Grid(nx, ny, delta, precision, te_only=te_only, **grid_kw)
        self.planes = 3 if te_only else 6

    def set_medium(self, n_global):
        """The rank's extended window of the global medium (periodic)."""
        nx, ny = self.part.extended(self.rank)
        oi, oj = self.part.origin(self.rank)
        ii = (oi + np.arange(nx)) % self.part.nx
        jj = (oj + np.arange(ny)) % self.part.ny
        self.grid.set_medium(np.ascontiguousarray(n_global[np.ix_(jj, ii)]))

    def set_packet(self, **packet):
        oi, oj = self.part.origin(self.rank)
        self.grid.set_packet_window(oi, oj, self.part.nx, self.part.ny, **packet)

    def step(self, k):
        self.grid.step(k)

    def pack(self, box):
        return self.grid.pack_box(box.i0, box.j0, box.w, box.h)

    def empty_box(self, box):
        import torch
        return torch.empty((self.planes, box.h, box.w), dtype=self.grid.box_dtype(),
                           device=self.grid.device)

    def unpack(self, box, buf):
        self.grid.unpack_box(box.i0, box.j0, box.w, box.h, buf)

    def interior_energy(self):
        b = self.part.interior(self.rank)
        return self.grid.energy_box(b.i0, b.j0, b.w, b.h)

    def interior_state(self):
        b = self.part.interior(self.rank)
        return self.grid.get_state()[:, b.j0:b.j0 + b.h, b.i0:b.i0 + b.w]

    def close(self):
        self.grid.close()


class Domain:
    """One lattice advanced as sub-domains with halo exchange.

    ``subs`` maps ranks to sub-domain objects (all of them for a
    ``LocalTransport``, this rank's for a ``DistTransport``); ``k`` steps run
    between exchanges (the partition's halo must be at least 4k + 1)."""

    def __init__(self, part, subs, transport, k=1):
        if part.halo < 4 * k + 1:
            raise ValueError("halo %d too thin for %d steps between exchanges" % (part.halo, k))
        self.part, self.subs, self.transport, self.k = part, subs, transport, int(k)

    def step(self, n_steps):
        left = int(n_steps)
        while left > 0:
            k = min(self.k, left)
            for s in self.subs.values():
                s.step(k)
            self.transport.exchange(self.part, self.subs)
            left -= k

    def energy(self):
        """FP64 energy of the whole lattice: the interior sums, added over
        the sub-domains (all-reduced across ranks)."""
        local = sum(s.interior_energy() for s in self.subs.values())
        return self.transport.allreduce_sum(local)

    def gather(self):
        """The global state (6, ny, nx) from the sub-domains of this process."""
        out = np.zeros((6, self.part.ny, self.part.nx))
        for rank, s in self.subs.items():
            i0, j0, w, h = self.part.block(rank)
            out[:, j0:j0 + h, i0:i0 + w] = s.interior_state()
        return out
