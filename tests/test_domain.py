"""Domain decomposition on the CPU: the partition's blocks, halos and
exchange plan, and the halo exchange itself with sub-domains stepped by the
oracle (in one process, and over two gloo ranks), against the oracle run on
the whole lattice.  The GPU sub-domains are checked in test_gpu_domain.py."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2604_21128_gb300 import domain, inputs  # noqa: E402


class OracleSub:
    """A sub-domain whose extended block is stepped by the oracle (periodic
    on the block, as the GPU sub-domains are)."""

    def __init__(self, part, rank, n_global, packet, delta, q_global=None):
        self.part, self.rank, self.delta = part, rank, delta
        nx, ny = part.extended(rank)
        oi, oj = part.origin(rank)
        ii = (oi + np.arange(nx)) % part.nx
        jj = (oj + np.arange(ny)) % part.ny
        self.n = np.ascontiguousarray(n_global[np.ix_(jj, ii)])
        if q_global is not None:
            self.q = np.ascontiguousarray(q_global[:, jj][:, :, ii])
        else:
            self.q = oracle.packet(self.n, delta, window=(oi, oj),
                                   global_shape=(part.ny, part.nx), **packet)

    def step(self, k):
        self.q = oracle.run(self.q, self.n, self.delta, k)

    def pack(self, b):
        return torch.from_numpy(np.ascontiguousarray(self.q[:, b.j0:b.j0 + b.h, b.i0:b.i0 + b.w]))

    def empty_box(self, b):
        return torch.empty((6, b.h, b.w), dtype=torch.float64)

    def unpack(self, b, buf):
        self.q[:, b.j0:b.j0 + b.h, b.i0:b.i0 + b.w] = buf.numpy()

    def interior_energy(self):
        b = self.part.interior(self.rank)
        return oracle.energy(np.ascontiguousarray(self.q[:, b.j0:b.j0 + b.h, b.i0:b.i0 + b.w]))

    def interior_state(self):
        b = self.part.interior(self.rank)
        return self.q[:, b.j0:b.j0 + b.h, b.i0:b.i0 + b.w]


def _workload(nx=72, ny=60):
    w = inputs.scaled(inputs.ellipse_256(), nx, ny, 0)
    return w.medium(), w.packet.as_dict(), w.delta


def test_halo_for_covers_the_reach():
    for k in (1, 2, 3, 5):
        h = domain.halo_for(k)
        assert h >= 4 * k + 1 and h % 4 == 0


@pytest.mark.parametrize("nx,ny,px,py", [(72, 60, 2, 2), (73, 61, 3, 2), (64, 40, 1, 2),
                                         (50, 50, 2, 1)])
def test_partition_tiles_the_lattice_and_plans_match(nx, ny, px, py):
    part = domain.Partition(nx, ny, px, py, halo=8)
    cover = np.zeros((ny, nx), dtype=int)
    for r in range(part.size):
        i0, j0, w, h = part.block(r)
        cover[j0:j0 + h, i0:i0 + w] += 1
        ex, ey = part.extended(r)
        assert (ex, ey) == (w + 16, h + 16)
        assert part.origin(r) == ((i0 - 8) % nx, (j0 - 8) % ny)
    assert np.all(cover == 1)
    for phase in (0, 1):
        for r in range(part.size):
            for t in part.phases(r)[phase]:
                # sends come from the interior (phase 0) or interior rows
                # (phase 1), and the receiving halo box has the same shape
                assert (t.send.w, t.send.h) == (t.recv.w, t.recv.h)
                pnx, pny = part.extended(t.peer)
                assert 0 <= t.recv.i0 and t.recv.i0 + t.recv.w <= pnx
                assert 0 <= t.recv.j0 and t.recv.j0 + t.recv.h <= pny
            # every halo cell is written exactly once per phase
            got = part.receives(r, phase)
            ex, ey = part.extended(r)
            mark = np.zeros((ey, ex), dtype=int)
            for _, b, _ in got:
                mark[b.j0:b.j0 + b.h, b.i0:b.i0 + b.w] += 1
            assert mark.max() == 1
            g = part.halo
            if phase == 0:
                assert np.all(mark[g:ey - g, :g] == 1) and np.all(mark[g:ey - g, ex - g:] == 1)
            else:
                assert np.all(mark[:g, :] == 1) and np.all(mark[ey - g:, :] == 1)


def test_partition_rejects_blocks_thinner_than_the_halo():
    with pytest.raises(ValueError):
        domain.Partition(40, 40, 4, 1, halo=12)


@pytest.mark.parametrize("k", [1, 2])
def test_local_exchange_reproduces_the_whole_lattice(k):
    n, pk, delta = _workload()
    steps = 7
    want = oracle.run(oracle.packet(n, delta, **pk), n, delta, steps)
    part = domain.Partition(72, 60, 2, 2, domain.halo_for(k))
    subs = {r: OracleSub(part, r, n, pk, delta) for r in range(part.size)}
    dom = domain.Domain(part, subs, domain.LocalTransport(), k=k)
    dom.step(steps)
    got = dom.gather()
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))
    assert dom.energy() == pytest.approx(oracle.energy(want), rel=1e-13)


def test_a_halo_thinner_than_the_reach_is_refused_and_would_be_wrong():
    """Two steps between exchanges reach eight cells: a 4-cell halo is
    refused, and stepping with it anyway corrupts the interior (random
    fields and medium, so every boundary carries signal)."""
    nx, ny = 72, 60
    n = inputs.random_medium(nx, ny, seed=3, lo=1.0, hi=2.5)
    q0 = inputs.random_state(nx, ny, seed=4)
    part = domain.Partition(nx, ny, 2, 2, 4)
    subs = {r: OracleSub(part, r, n, None, 1.0, q_global=q0) for r in range(part.size)}
    with pytest.raises(ValueError):
        domain.Domain(part, subs, domain.LocalTransport(), k=2)
    want = oracle.run(q0, n, 1.0, 4)
    for _ in range(2):
        for s in subs.values():
            s.step(2)
        domain.LocalTransport().exchange(part, subs)
    got = np.zeros_like(want)
    for r, s in subs.items():
        i0, j0, w, h = part.block(r)
        got[:, j0:j0 + h, i0:i0 + w] = s.interior_state()
    assert np.max(np.abs(got - want)) > 1e-3
    # with halo_for(2) the same run is exact
    part = domain.Partition(nx, ny, 2, 2, domain.halo_for(2))
    subs = {r: OracleSub(part, r, n, None, 1.0, q_global=q0) for r in range(part.size)}
    dom = domain.Domain(part, subs, domain.LocalTransport(), k=2)
    dom.step(4)
    assert np.max(np.abs(dom.gather() - want)) <= 1e-13 * np.max(np.abs(want))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n, pk, delta = _workload()
        part = domain.Partition(72, 60, 2, 1, domain.halo_for(1))
        sub = OracleSub(part, rank, n, pk, delta)
        dom = domain.Domain(part, {rank: sub}, domain.DistTransport("cpu"), k=1)
        dom.step(5)
        e = dom.energy()
        i0, j0, w, h = part.block(rank)
        q.put((rank, (i0, j0, w, h), sub.interior_state().copy(), e))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_exchange_halos():
    """World size 2: one sub-domain per rank, strips sent over gloo, energy
    all-reduced; the assembled lattice equals the oracle's whole-lattice run."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    n, pk, delta = _workload()
    want = oracle.run(oracle.packet(n, delta, **pk), n, delta, 5)
    full = np.zeros_like(want)
    for rank, (i0, j0, w, h), block, e in got:
        full[:, j0:j0 + h, i0:i0 + w] = block
        assert e == pytest.approx(oracle.energy(want), rel=1e-13)
    assert np.max(np.abs(full - want)) <= 1e-13 * np.max(np.abs(want))
