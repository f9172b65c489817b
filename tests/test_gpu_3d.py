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


@pytest.mark.parametrize("precision,rel", [("fp64", 1e-10), ("fp32", 2e-5)])
@pytest.mark.parametrize("shape", [(24, 20, 6), (70, 40, 36)])
def test_divergence_matches_oracle(shape, precision, rel):
    nx, ny, nz = shape
    n = medium3(nx, ny, nz, seed=21)
    q0 = np.random.default_rng(22).standard_normal((6, nz, ny, nx))
    want = oracle.divergence3(oracle.run3(q0, n, 0.8, 3), n, 0.8)
    with qla.Grid3(nx, ny, nz, 0.8, precision) as g:
        g.set_medium(n)
        g.set_state(q0)
        g.step(3)
        got = g.divergence()
    for k in qla.DIV_KEYS:
        assert got[k] == pytest.approx(want[k], rel=rel), (k, got[k], want[k])


def test_divergence_closed_form_through_the_abi():
    """B = D = (s, s, s), s = sin(k.r), on a padded lattice (nx = 40)."""
    import math
    nx, ny, nz, delta = 40, 12, 16, 0.5
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    k = (2 * math.pi * 3 / nx, 2 * math.pi * 2 / ny, 2 * math.pi * 5 / nz)
    s = np.sin(k[0] * x + k[1] * y + k[2] * z)
    n = 1.5 + 0.25 * np.cos(2 * math.pi * x / nx)
    q = np.zeros((6, nz, ny, nx))
    q[3] = q[4] = q[5] = s
    q[0] = q[1] = q[2] = s / n
    with qla.Grid3(nx, ny, nz, delta, "fp64") as g:
        g.set_medium(n)
        g.set_state(q)
        d = g.divergence()
    N = nx * ny * nz
    sines = [math.sin(v) for v in k]
    assert d["div_b_sq"] == pytest.approx(N / 2 * sum(sines) ** 2 / delta ** 2, rel=1e-12)
    assert d["grad_b_sq"] == pytest.approx(N / 2 * sum(v * v for v in sines) / delta ** 2, rel=1e-12)
    assert d["div_d_sq"] == pytest.approx(d["div_b_sq"], rel=1e-12)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-14), ("fp32", 2e-7)])
def test_packet_is_the_2d_packet_in_every_slice(precision, tol):
    nx, ny, nz = 80, 48, 6
    n = medium3(nx, ny, nz, seed=31)
    pk = dict(x0=20.0, y0=30.0, angle=0.4, k0=0.3, width=8.0, transverse_width=12.0)
    want = np.stack([oracle.packet(n[k], 1.0, **pk) for k in range(nz)], axis=1)
    with qla.Grid3(nx, ny, nz, 1.0, precision) as g:
        g.set_medium(n)
        g.set_packet(**pk)
        got = g.get_state()
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))
    assert np.all(got[[0, 1, 5]] == 0)


def test_packet_errors():
    with qla.Grid3(8, 8, 8, 1.0, "fp32") as g:
        with pytest.raises(qla.QLAError) as e:
            g.set_packet(x0=2.0, y0=2.0, angle=0.0, k0=0.3, width=2.0)
        assert e.value.status == 2                                 # no medium yet
        g.set_medium(np.ones((8, 8, 8)))
        for bad in (dict(width=0.0), dict(width=2.0, transverse_width=-1.0),
                    dict(width=float("nan")), dict(width=2.0, amplitude=float("inf"))):
            with pytest.raises(qla.QLAError) as e:
                g.set_packet(x0=2.0, y0=2.0, angle=0.0, k0=0.3, **bad)
            assert e.value.status == 1
        g.set_packet(x0=2.0, y0=2.0, angle=0.0, k0=0.3, width=2.0)
        g.step(2)
        assert g.energy() > 0
