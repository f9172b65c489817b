"""Domain decomposition on one GPU: a lattice split into sub-domain contexts
with halos (Sec. V-A), stepped by the library's kernels and refilled by its
pack / unpack kernels, against the oracle run on the whole lattice; the
global energy as the sum of the sub-domains' interior energies; and the
box and window-packet calls on their own."""
import os

import numpy as np
import pytest

import oracle
from paper_2604_21128_gb300 import build as qbuild
from paper_2604_21128_gb300 import domain, inputs, qla

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    qbuild.build()
    oracle.set_threads(os.cpu_count() or 1)


def _rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _run(nx, ny, px, py, k, steps, precision, te, n, pk=None, q0=None):
    part = domain.Partition(nx, ny, px, py, domain.halo_for(k))
    subs = {}
    for r in range(part.size):
        s = domain.GridSub(part, r, 1.0, precision, te_only=te)
        s.set_medium(n)
        if q0 is not None:
            nxe, nye = part.extended(r)
            oi, oj = part.origin(r)
            ii = (oi + np.arange(nxe)) % nx
            jj = (oj + np.arange(nye)) % ny
            s.grid.set_state(np.ascontiguousarray(q0[:, jj][:, :, ii]))
        else:
            s.set_packet(**pk)
        subs[r] = s
    dom = domain.Domain(part, subs, domain.LocalTransport(), k=k)
    dom.step(steps)
    out = dom.gather(), dom.energy()
    for s in subs.values():
        s.close()
    return out


@pytest.mark.parametrize("px,py,k", [(2, 2, 1), (2, 2, 2), (3, 2, 1), (1, 3, 3)])
def test_fp64_subdomains_match_the_whole_lattice(px, py, k):
    w = inputs.scaled(inputs.ellipse_256(), 200, 136, 0)
    n = w.medium()
    pk = w.packet.as_dict()
    steps = 23
    want = oracle.run(oracle.packet(n, w.delta, **pk), n, w.delta, steps)
    got, e = _run(w.nx, w.ny, px, py, k, steps, "fp64", False, n, pk=pk)
    assert _rel_l2(got, want) <= 1e-12
    assert abs(e / oracle.energy(want) - 1) <= 1e-12


def test_fp64_random_state_and_medium_2x2():
    nx, ny = 150, 118
    n = inputs.random_medium(nx, ny, seed=91, lo=1.0, hi=3.0)
    q0 = inputs.random_state(nx, ny, seed=92)
    want = oracle.run(q0, n, 1.0, 11)
    got, e = _run(nx, ny, 2, 2, 1, 11, "fp64", False, n, q0=q0)
    assert _rel_l2(got, want) <= 1e-12
    assert abs(e / oracle.energy(want) - 1) <= 1e-12


def test_fp32_ez_subdomains_2x2():
    """FP32 E_z sub-domains (the packed marching kernel on 16-aligned
    blocks) against the oracle: the single-lattice FP32 bound."""
    w = inputs.scaled(inputs.ellipse_256(), 256, 192, 0)
    n = w.medium()
    pk = w.packet.as_dict()
    steps = 40
    want = oracle.run(oracle.packet(n, w.delta, **pk), n, w.delta, steps)
    got, e = _run(w.nx, w.ny, 2, 2, 1, steps, "fp32", True, n, pk=pk)
    assert _rel_l2(got, want) <= 1e-6
    assert abs(e / oracle.energy(want) - 1) <= 1e-6
    assert np.all(got[[0, 1, 5]] == 0)


def test_box_calls_and_window_packet():
    import torch
    nx, ny = 96, 70
    n = inputs.random_medium(nx, ny, seed=5, lo=1.0, hi=2.0)
    q0 = inputs.random_state(nx, ny, seed=6)
    with qla.Grid(nx, ny, 1.0, "fp64") as g:
        g.set_medium(n)
        g.set_state(q0)
        box = g.pack_box(10, 20, 30, 15)
        assert box.shape == (6, 15, 30) and box.dtype == torch.float64
        assert np.array_equal(box.cpu().numpy(), q0[:, 20:35, 10:40])
        e = g.energy_box(10, 20, 30, 15)
        assert e == pytest.approx(float((q0[:, 20:35, 10:40] ** 2).sum()), rel=1e-13)
        # write the box elsewhere and read the state back
        g.unpack_box(50, 40, 30, 15, box)
        q1 = g.get_state()
        want = q0.copy()
        want[:, 40:55, 50:80] = q0[:, 20:35, 10:40]
        assert np.array_equal(q1, want)
        with pytest.raises(qla.QLAError) as err:
            g.pack_box(80, 0, 30, 5)
        assert err.value.status == 1
    # a window packet equals the same sites of the whole lattice's packet
    w = inputs.scaled(inputs.ellipse_256(), 200, 136, 0)
    nw = w.medium()
    pk = w.packet.as_dict()
    with qla.Grid(w.nx, w.ny, 1.0, "fp64") as g:
        g.set_medium(nw)
        g.set_packet(**pk)
        full = g.get_state()
    ii = (150 + np.arange(80)) % w.nx
    jj = (100 + np.arange(64)) % w.ny
    with qla.Grid(80, 64, 1.0, "fp64") as g:
        g.set_medium(np.ascontiguousarray(nw[np.ix_(jj, ii)]))
        g.set_packet_window(150, 100, w.nx, w.ny, **pk)
        part = g.get_state()
    assert np.max(np.abs(part - full[:, jj][:, :, ii])) <= 1e-15
