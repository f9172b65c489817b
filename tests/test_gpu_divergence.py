"""GPU Gauss-law monitors (qla_divergence, Eqs. 3.1 and 3.2) against the
oracle's orc_divergence on the same states, through the C ABI: random
states and media, all three potential readings, TE and six-plane contexts,
pending potential steps, ragged and pitched shapes; and the closed form on
a plane wave."""
import math
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


def _gpu(n, delta, q0, steps, precision="fp64", te=False, potential="rotation"):
    ny, nx = n.shape
    with qla.Grid(nx, ny, delta, precision, te_only=te, potential=potential) as g:
        g.set_medium(n)
        g.set_state(q0)
        g.step(steps)
        return g.divergence()


def _check(got, want, rel):
    for k in qla.DIV_KEYS:
        if want[k] == 0.0:
            assert got[k] == 0.0, k
        else:
            assert got[k] == pytest.approx(want[k], rel=rel), (k, got[k], want[k])


@pytest.mark.parametrize("te", [False, True])
@pytest.mark.parametrize("potential", ["rotation", "literal", "none"])
@pytest.mark.parametrize("shape,steps", [((67, 45), 5), ((128, 37), 0), ((9, 9), 3), ((300, 70), 4)])
def test_fp64_matches_oracle(shape, steps, potential, te):
    nx, ny = shape
    delta = 0.6
    n = inputs.random_medium(nx, ny, seed=nx * 13 + ny, lo=1.0, hi=3.5)
    q0 = inputs.random_state(nx, ny, seed=nx + 5 * ny)
    if te:
        q0[[0, 1, 5]] = 0.0
    want = oracle.divergence(oracle.run(q0, n, delta, steps, potential), n, delta)
    got = _gpu(n, delta, q0, steps, te=te, potential=potential)
    _check(got, want, 1e-10)


def test_fp32_te_matches_oracle():
    """FP32 E_z state (values rounded to 24 bits, rotations in FP32): the
    sums agree with the FP64 oracle to ~1e-6 relative."""
    nx, ny = 160, 96
    n = inputs.random_medium(nx, ny, seed=3, lo=1.0, hi=3.0)
    q0 = inputs.random_state(nx, ny, seed=4)
    q0[[0, 1, 5]] = 0.0
    want = oracle.divergence(oracle.run(q0, n, 1.0, 6), n, 1.0)
    got = _gpu(n, 1.0, q0, 6, precision="fp32", te=True)
    _check(got, want, 2e-5)


def test_plane_wave_closed_form_through_the_abi():
    """B = D = (s, s), s = sin(kx i + ky j): sums N/2 (sin kx + sin ky)^2 /
    delta^2 and N/2 (sin^2 kx + sin^2 ky) / delta^2 (no steps: the state as
    set).  nx = 100 exercises the padded row pitch."""
    nx, ny, delta = 100, 60, 0.5
    kx, ky = 2 * math.pi * 7 / nx, 2 * math.pi * 4 / ny
    i = np.arange(nx)[None, :]
    j = np.arange(ny)[:, None]
    s = np.sin(kx * i + ky * j)
    n = 1.0 + 0.5 * np.cos(2 * math.pi * i / nx) * np.ones((ny, 1))
    q = np.zeros((6, ny, nx))
    q[3] = q[4] = s
    q[0] = q[1] = s / n
    got = _gpu(n, delta, q, 0)
    N = nx * ny
    assert got["div_b_sq"] == pytest.approx(N / 2 * (math.sin(kx) + math.sin(ky)) ** 2 / delta ** 2,
                                            rel=1e-12)
    assert got["grad_b_sq"] == pytest.approx(N / 2 * (math.sin(kx) ** 2 + math.sin(ky) ** 2)
                                             / delta ** 2, rel=1e-12)
    assert got["div_d_sq"] == pytest.approx(got["div_b_sq"], rel=1e-12)


def test_needs_medium_and_state():
    with qla.Grid(64, 32, 1.0, "fp64") as g:
        with pytest.raises(qla.QLAError) as e:
            g.divergence()
        assert e.value.status == 2  # QLA_ESTATE
