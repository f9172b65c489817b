"""Dataflow steps of the plateau split (FP32 E_z): every step of a qla_step
call in one persistent launch, each work unit waiting for the items it
depends on (those whose stored sites it reads within the four-site reach of
Eqs. 2e6 and 2e9, and those that read what it stores) instead of a launch
per step.  The schedule changes, the arithmetic does not: states and
energies must equal those of one launch per step bit for bit, on ragged
lattices, every potential reading, several segment heights and across
calls.  A wait that runs out (a unit made to withhold its completion)
reports QLA_ETIMEOUT at the next read, without a fault, and the context
works again once its state is set."""
import time

import numpy as np
import pytest
import torch

from paper_2604_21128_gb300 import build as qbuild
from paper_2604_21128_gb300 import inputs, qla

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    qbuild.build()


def plateau_medium(nx, ny):
    """n = 2 background, on wide lattices n = 3 in a band and n = 1 in an
    ellipse, and a patch of random n (rows 5/8 to 7/8 of the lattice, from
    column nx / 2): plateau items and general items next to each other, on
    small lattices too."""
    y, x = np.mgrid[0:ny, 0:nx]
    n = np.full((ny, nx), 2.0)
    if nx >= 600:
        n[:, : nx // 3] = 3.0
        n[((x - nx / 2) / (nx / 6)) ** 2 + ((y - ny / 2) / (ny / 4)) ** 2 < 1.0] = 1.0
    r0, r1, c0 = ny * 5 // 8, ny * 7 // 8, nx // 2
    w = min(70, nx // 4)
    n[r0:r1, c0:c0 + w] = np.random.default_rng(3).uniform(1.2, 2.8, (r1 - r0, w))
    return n


def run(n, calls, q0, kernel, rows, potential="rotation"):
    """State, energy, flow segment and launches after qla_step calls of the
    given step counts."""
    ny, nx = n.shape
    with qla.Grid(nx, ny, 1.0, "fp32", te_only=True, potential=potential) as g:
        g.set_step_kernel(kernel)
        g.set_march_tuning(0, rows)
        g.set_medium(n)
        g.set_state(q0)
        l0 = g.launches
        for k in calls:
            g.step(k)
        launches = g.launches - l0
        return g.get_state(), g.energy(), g.flow_plan, launches


@pytest.mark.parametrize("nx,ny,rows,potential,calls", [
    (1024, 384, 32, "rotation", (11,)),
    (1024, 384, 64, "literal", (8,)),
    (1024, 384, 48, "none", (9,)),
    (1000, 200, 32, "rotation", (7,)),       # last window 40 columns, last segment 8 rows
    (1000, 200, 32, "rotation", (1, 1, 2, 5)),
    (128, 64, 32, "rotation", (6,)),         # two windows (120 + 8 columns), two segments
    (248, 100, 40, "literal", (3, 4)),       # nx = 2 windows + 8 columns, ragged segments
    (512, 36, 32, "rotation", (5,)),         # second segment of 4 rows
])
def test_flow_steps_agree_bitwise(nx, ny, rows, potential, calls):
    n = plateau_medium(nx, ny)
    q0 = inputs.random_state(nx, ny, seed=41, planes=3)
    step = run(n, calls, q0, "march_step", rows, potential)
    flow = run(n, calls, q0, "march_flow", rows, potential)
    seg = (rows + 3) // 4 * 4
    assert step[2] == 0 and flow[2] == seg, (step[2], flow[2])
    # one launch per call, plus the first step of a call with no pending
    # potential step (the first call with a potential)
    first = 1 if potential != "none" else 0
    assert flow[3] == len(calls) + first - (1 if calls[0] == 1 and first else 0), flow[3]
    assert step[3] == sum(calls)
    assert np.array_equal(step[0], flow[0])
    assert step[1] == flow[1]


def test_flow_is_the_default_on_large_lattices():
    """The 8192^2 ellipse workload takes dataflow steps by default (64-row
    segments: at least three items per resident warp); 12 steps equal 12
    launches of the per-step kernel bit for bit, compared on the device."""
    w = inputs.ellipse_8192()
    n = w.medium()
    pk = w.packet.as_dict()
    out = {}
    for kernel in ("auto", "march_step"):
        with qla.Grid(w.nx, w.ny, w.delta, "fp32", te_only=True) as g:
            g.set_step_kernel(kernel)
            g.set_medium(n)
            g.set_packet(**pk)
            l0 = g.launches
            g.step(5)
            g.step(7)
            launches = g.launches - l0
            out[kernel] = (g.pack_box(0, 0, w.nx, w.ny), g.energy(), g.flow_plan, launches)
    assert out["auto"][2] > 0 and out["march_step"][2] == 0
    assert out["auto"][3] == 3 and out["march_step"][3] == 12
    assert torch.equal(out["auto"][0], out["march_step"][0])
    assert out["auto"][1] == out["march_step"][1]


def test_flow_wait_runs_out_without_fault():
    """A unit that finishes without counting itself: the units that depend
    on its item wait out a short limit, the launch drains, the next read
    returns QLA_ETIMEOUT; with the hook off and the state set again the
    context steps exactly as before."""
    nx, ny = 1024, 384
    n = plateau_medium(nx, ny)
    q0 = inputs.random_state(nx, ny, seed=42, planes=3)
    with qla.Grid(nx, ny, 1.0, "fp32", te_only=True) as g:
        g.set_step_kernel("march_flow")
        g.set_march_tuning(0, 32)
        g.set_medium(n)
        g.set_state(q0)
        g.step(1)                      # the potential step is now pending
        g.debug_flow(budget_cycles=2_000_000, withhold_unit=5)
        t0 = time.perf_counter()
        g.step(6)
        with pytest.raises(qla.QLAError) as e:
            g.energy()
        assert e.value.status == 5     # QLA_ETIMEOUT
        assert time.perf_counter() - t0 < 30.0
        g.step(2)                      # runs again, on an undefined state
        g.debug_flow()
        g.set_state(q0)
        g.step(7)
        got, e7 = g.get_state(), g.energy()
    want = run(n, (7,), q0, "march_step", 32)
    assert np.array_equal(got, want[0]) and e7 == want[1]


def test_debug_flow_arguments():
    with qla.Grid(256, 64, 1.0, "fp32", te_only=True) as g:
        with pytest.raises(qla.QLAError):
            g.debug_flow(budget_cycles=-1)
        with pytest.raises(qla.QLAError):
            g.debug_flow(withhold_unit=-2)
        g.debug_flow(0, -1)
