"""Batched persistent launch: many uneven lattices in one cooperative
kernel per chunk, against the same lattices advanced one by one."""
import math

import numpy as np
import pytest

from paper_2604_21128_gb300 import build as qbuild
from paper_2604_21128_gb300 import inputs, qla

pytestmark = pytest.mark.gpu

SIZES = [(128, 64), (192, 100), (256, 128), (320, 72)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    qbuild.build()


def _setup(g, k, nx, ny):
    n = inputs.ellipse_medium(nx, ny, 1.0, a=0.2 * nx, b=0.15 * ny, n_in=1.5 + 0.5 * k,
                              n_out=1.0, edge=3.0, angle=0.3 * k)
    g.set_medium(n)
    g.set_packet(x0=0.25 * nx, y0=0.5 * ny, angle=0.4 * k, k0=0.3, width=nx / 16,
                 transverse_width=nx / 8)
    return n


def _singles(precision, te, steps):
    out = []
    for k, (nx, ny) in enumerate(SIZES):
        with qla.Grid(nx, ny, 1.0, precision, te_only=te) as g:
            _setup(g, k, nx, ny)
            g.step(steps)
            out.append((g.get_state(), g.energy()))
    return out


@pytest.mark.parametrize("precision,te", [("fp32", True), ("fp64", False)])
def test_batch_step_equals_single_runs_bitwise(precision, te):
    want = _singles(precision, te, 23)
    with qla.Batch(SIZES, 1.0, precision, te_only=te) as b:
        for k, (nx, ny) in enumerate(SIZES):
            _setup(b.instance(k), k, nx, ny)
        b.step(10)
        b.step(13)
        e = b.energy()
        for k in range(len(SIZES)):
            got = b.instance(k).get_state()
            assert np.array_equal(got, want[k][0]), k
            assert e[k] == want[k][1]


def test_batch_run_graph_energies():
    steps, every = 24, 6
    rows = []
    for k, (nx, ny) in enumerate(SIZES):
        with qla.Grid(nx, ny, 1.0, "fp32", te_only=True) as g:
            _setup(g, k, nx, ny)
            col = []
            for r in range(steps // every):
                g.step(every)
                col.append(g.energy())
            rows.append(col)
    want = np.array(rows).T
    with qla.Batch(SIZES, 1.0, "fp32", te_only=True) as b:
        for k, (nx, ny) in enumerate(SIZES):
            _setup(b.instance(k), k, nx, ny)
        e = b.run(steps, every)
        assert e.shape == (steps // every, len(SIZES))
        assert np.allclose(e, want, rtol=1e-12, atol=0)
        # the states after the graph run equal the step-by-step ones
        got = b.instance(2).get_state()
    with qla.Grid(*SIZES[2], 1.0, "fp32", te_only=True) as g:
        _setup(g, 2, *SIZES[2])
        g.step(steps)
        assert np.array_equal(got, g.get_state())


def test_batch_autotune_keeps_results():
    with qla.Batch(SIZES, 1.0, "fp32", te_only=True) as b:
        for k, (nx, ny) in enumerate(SIZES):
            _setup(b.instance(k), k, nx, ny)
        lx, rows = b.autotune(trial_steps=2)
        assert lx in (1, 2) and rows in (64, 128, 256)
        b.step(5)
        got = [b.instance(k).get_state() for k in range(len(SIZES))]
    want = _singles("fp32", True, 6 * 2 + 5)
    for k in range(len(SIZES)):
        assert np.array_equal(got[k], want[k][0]), k


def test_batch_barrier_wait_times_out_and_batch_recovers():
    """A block that never arrives: every other block's bounded wait runs out
    and the step reports QLA_ETIMEOUT; no fault, and the batch works after."""
    with qla.Batch(SIZES, 1.0, "fp32", te_only=True) as b:
        for k, (nx, ny) in enumerate(SIZES):
            _setup(b.instance(k), k, nx, ny)
        b.step(1)  # every instance now has a pending potential step
        b.debug_barrier(budget_cycles=2_000_000, skip_block=0)
        with pytest.raises(qla.QLAError) as e:
            b.step(3)
        assert e.value.status == 5  # QLA_ETIMEOUT
        b.debug_barrier(0, -1)
        for k, (nx, ny) in enumerate(SIZES):
            _setup(b.instance(k), k, nx, ny)
        b.step(4)
        e4 = b.energy()
    want = _singles("fp32", True, 4)
    assert np.array_equal(e4, np.array([w[1] for w in want]))
