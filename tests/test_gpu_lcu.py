"""The LCU form of the potential operators (QLA_POTENTIAL_LCU, Eqs. 2f1-2f7,
emulated branch by branch) on the GPU against the oracle's branch-by-branch
emulation: scalar and tensor media, six planes and E_z, FP64 and FP32; and
the instability it carries (the printed q3 row of V_y) reproduced."""
import os

import numpy as np
import pytest

import oracle
from paper_2604_21128_gb300 import build as qbuild
from paper_2604_21128_gb300 import inputs, qla

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    qbuild.build()
    oracle.set_threads(os.cpu_count() or 1)


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def gpu(n, delta, q0, steps, precision="fp64", te=False, tensor=False):
    ny, nx = n.shape[-2:]
    with qla.Grid(nx, ny, delta, precision, te_only=te, potential="lcu", tensor=tensor) as g:
        g.set_medium(n)
        g.set_state(q0)
        g.step(steps)
        return g.get_state(), g.energy()


@pytest.mark.parametrize("te", [False, True])
@pytest.mark.parametrize("shape", [(67, 45), (9, 9), (130, 70)])
def test_fp64_matches_oracle(shape, te):
    nx, ny = shape
    n = inputs.random_medium(nx, ny, seed=nx + ny, lo=1.0, hi=3.0)
    q0 = inputs.random_state(nx, ny, seed=3 * nx + ny, planes=3 if te else 6)
    want = oracle.run(q0, n, 0.8, 5, "lcu")
    got, e = gpu(n, 0.8, q0, 5, te=te)
    assert rel_l2(got, want) <= 1e-11, rel_l2(got, want)
    assert e == pytest.approx(oracle.energy(want), rel=1e-11)


def test_tensor_medium_matches_oracle():
    nx, ny = 96, 50
    nt = np.stack([inputs.random_medium(nx, ny, seed=60 + k, lo=1.0, hi=3.0) for k in range(3)])
    q0 = inputs.random_state(nx, ny, seed=64)
    want = oracle.run(q0, nt, 0.9, 4, "lcu")
    got, _ = gpu(nt, 0.9, q0, 4, tensor=True)
    assert rel_l2(got, want) <= 1e-11, rel_l2(got, want)


def test_fp32_matches_oracle():
    nx, ny = 128, 64
    n = inputs.random_medium(nx, ny, seed=70, lo=1.0, hi=3.0)
    q0 = inputs.random_state(nx, ny, seed=71, planes=3)
    want = oracle.run(q0, n, 1.0, 5, "lcu")
    got, _ = gpu(n, 1.0, q0, 5, precision="fp32", te=True)
    assert rel_l2(got, want) <= 1e-5, rel_l2(got, want)


def test_energy_growth_of_the_printed_potential():
    """The 256^2 ellipse workload for 125 steps: the GPU reproduces the
    oracle's energy, which the printed V drives up: x1.5 at once (the q3 row
    of V_y overwrites B_x with n E_z), then exponentially from step ~90 on,
    when the packet reaches the ellipse (x4e9 by step 125)."""
    w = inputs.ellipse_256()
    n = w.medium()
    q0 = oracle.packet(n, w.delta, **w.packet.as_dict())
    e0 = oracle.energy(q0)
    want = oracle.energy(oracle.run(q0, n, w.delta, 125, "lcu"))
    _, e = gpu(n, w.delta, q0, 125)
    assert e == pytest.approx(want, rel=1e-6)
    assert e / e0 > 1e8
    print("energy after 125 steps: x%.3g (LCU as printed)" % (e / e0))


def test_lcu_contexts_step_with_the_tile_kernel():
    with qla.Grid(64, 16, 1.0, "fp64", potential="lcu") as g:
        with pytest.raises(qla.QLAError) as e:
            g.set_step_kernel("march")
        assert e.value.status == 1
