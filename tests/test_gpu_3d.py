"""Three-dimensional QLA on the GPU (qla3_*, through the C ABI) against the
oracle's 3D step (oracle.run3): ragged shapes spanning several 32-cell
segments along each axis and shorter than the 40-cell staged line, both
potential readings, FP64 at 1e-12 and FP32 within its rounding budget,
energy and errors."""
import os

import numpy as np
import pytest

import oracle
from paper_2604_21128_gb300 import build as qbuild
from paper_2604_21128_gb300 import qla

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    qbuild.build()
    oracle.set_threads(os.cpu_count() or 1)


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def medium3(nx, ny, nz, seed):
    rng = np.random.default_rng(seed)
    raw = rng.random((nz, ny, nx))
    # a little smoothing along each axis keeps beta moderate
    for ax in range(3):
        raw = (raw + np.roll(raw, 1, ax) + np.roll(raw, -1, ax)) / 3
    return 1.0 + 2.5 * raw


@pytest.mark.parametrize("kernel", ["march", "passes", "slices", "auto"])
@pytest.mark.parametrize("potential", ["rotation", "none"])
@pytest.mark.parametrize("shape", [(24, 20, 6), (33, 17, 9), (70, 40, 36), (5, 3, 2),
                                   (40, 26, 70), (128, 12, 21)])
def test_fp64_matches_oracle(shape, potential, kernel):
    nx, ny, nz = shape
    n = medium3(nx, ny, nz, seed=nx + ny + nz)
    q0 = np.random.default_rng(nx * ny + nz).standard_normal((6, nz, ny, nx))
    want = oracle.run3(q0, n, 0.7, 3, potential)
    with qla.Grid3(nx, ny, nz, 0.7, "fp64", potential) as g:
        g.set_step_kernel(kernel)
        g.set_medium(n)
        g.set_state(q0)
        g.step(3)
        got = g.get_state()
        e = g.energy()
        assert g.launches >= 3
    assert rel_l2(got, want) <= 1e-12, rel_l2(got, want)
    assert e == pytest.approx(float(np.sum(want ** 2)), rel=1e-12)


def test_fp32_matches_oracle():
    nx, ny, nz = 64, 48, 40
    n = medium3(nx, ny, nz, seed=5)
    q0 = np.random.default_rng(6).standard_normal((6, nz, ny, nx))
    want = oracle.run3(q0, n, 1.0, 8)
    with qla.Grid3(nx, ny, nz, 1.0, "fp32") as g:
        g.set_medium(n)
        g.set_state(q0)
        g.step(8)
        got = g.get_state()
    assert rel_l2(got, want) <= 1e-5, rel_l2(got, want)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("shape", [(64, 48, 40), (37, 19, 53), (130, 24, 33)])
def test_step_kernels_agree_bitwise(shape, precision):
    """The per-axis passes, the fused march and the slices + column pipeline
    apply the same operations in the same order at every site (lattices
    narrower than 64 columns run the passes under "slices")."""
    nx, ny, nz = shape
    n = medium3(nx, ny, nz, seed=11)
    q0 = np.random.default_rng(12).standard_normal((6, nz, ny, nx))
    out = []
    for kernel in ("passes", "march", "slices"):
        with qla.Grid3(nx, ny, nz, 1.0, precision) as g:
            g.set_step_kernel(kernel)
            g.set_medium(n)
            g.set_state(q0)
            g.step(7)
            out.append(g.get_state())
    assert np.array_equal(out[0], out[1])
    assert np.array_equal(out[0], out[2])


def test_energy_conserved_over_many_steps():
    nx, ny, nz = 48, 40, 36
    n = medium3(nx, ny, nz, seed=7)
    q0 = np.random.default_rng(8).standard_normal((6, nz, ny, nx))
    with qla.Grid3(nx, ny, nz, 1.0, "fp64") as g:
        g.set_medium(n)
        g.set_state(q0)
        e0 = g.energy()
        g.step(100)
        assert abs(g.energy() / e0 - 1) < 1e-12


def test_errors():
    lib = qla.load()
    assert lib.qla3_workspace_bytes(8, 8, 8, 0, 1) == 0          # QLA_TE_ONLY: not in 3D
    assert lib.qla3_workspace_bytes(8, 70000, 2, 0, 0) == 0      # ny beyond 65535
    with qla.Grid3(8, 8, 8, 1.0, "fp64") as g:
        with pytest.raises(qla.QLAError) as e:
            g.step(1)
        assert e.value.status == 2                                 # QLA_ESTATE
        with pytest.raises(qla.QLAError) as e:
            g.set_medium(np.zeros((8, 8, 8)))
        assert e.value.status == 1                                 # QLA_EINVAL
