"""Diagonal index tensor media (QLA_ANISOTROPIC, qla_set_medium_tensor) on
the GPU against the oracle's anisotropic step (every pair with its own
angle, Eqs. 2e4, 2e8, 2e13): six-plane and E_z contexts, all three
potential readings, FP64 at 1e-12 and FP32 within its rounding budget;
read-outs (fields, divergence, energy) with the tensor; and the isotropic
special case bit for bit against a scalar-medium context."""
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


def tensor_medium(nx, ny, seed):
    return np.stack([inputs.random_medium(nx, ny, seed=seed + k, lo=1.0, hi=3.5)
                     for k in range(3)])


def run_gpu(nt, delta, q0, steps, precision="fp64", te=False, potential="rotation"):
    _, ny, nx = nt.shape
    with qla.Grid(nx, ny, delta, precision, te_only=te, potential=potential, tensor=True) as g:
        g.set_medium(nt)
        g.set_state(q0)
        g.step(steps)
        return g.get_state(), g.energy(), g.fields(), g.divergence()


@pytest.mark.parametrize("potential", ["rotation", "literal", "none"])
@pytest.mark.parametrize("shape", [(67, 45), (9, 9), (130, 70), (33, 100)])
def test_six_plane_fp64_matches_oracle(shape, potential):
    nx, ny = shape
    nt = tensor_medium(nx, ny, seed=nx * 7 + ny)
    q0 = inputs.random_state(nx, ny, seed=nx + 11 * ny)
    want = oracle.run(q0, nt, 0.7, 6, potential)
    got, e, _, _ = run_gpu(nt, 0.7, q0, 6, potential=potential)
    assert rel_l2(got, want) <= 1e-12, rel_l2(got, want)
    if potential != "literal":
        assert e == pytest.approx(oracle.energy(q0), rel=1e-12)


@pytest.mark.parametrize("te", [True, False])
def test_fp32_matches_oracle(te):
    nx, ny = 160, 96
    nt = tensor_medium(nx, ny, seed=5)
    q0 = inputs.random_state(nx, ny, seed=6, planes=3 if te else 6)
    want = oracle.run(q0, nt, 1.0, 20)
    got, _, _, _ = run_gpu(nt, 1.0, q0, 20, precision="fp32", te=te)
    assert rel_l2(got, want) <= 1e-5, rel_l2(got, want)


def test_te_context_sees_n_z_only():
    """E_z contexts evolve (q2, q3, q4) with n_z alone: the tensor result is
    the oracle's, and bitwise the scalar-medium result with n = n_z."""
    nx, ny = 256, 64
    nt = tensor_medium(nx, ny, seed=9)
    q0 = inputs.random_state(nx, ny, seed=10, planes=3)
    want = oracle.run(q0, nt, 0.9, 9)
    got, _, _, _ = run_gpu(nt, 0.9, q0, 9, te=True)
    assert rel_l2(got, want) <= 1e-12
    with qla.Grid(nx, ny, 0.9, "fp64", te_only=True) as g:
        g.set_medium(nt[2].copy())
        g.set_state(q0)
        g.step(9)
        assert np.array_equal(g.get_state(), got)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_equal_components_are_the_scalar_medium_bitwise(precision):
    nx, ny = 96, 40
    n = inputs.random_medium(nx, ny, seed=12, lo=1.0, hi=3.0)
    q0 = inputs.random_state(nx, ny, seed=13)
    got, _, _, _ = run_gpu(np.stack([n, n, n]), 1.0, q0, 7, precision=precision)
    with qla.Grid(nx, ny, 1.0, precision) as g:
        g.set_step_kernel("tile")
        g.set_medium(n)
        g.set_state(q0)
        g.step(7)
        assert np.array_equal(g.get_state(), got)


def test_fields_and_divergence_use_each_component():
    nx, ny = 70, 44
    nt = tensor_medium(nx, ny, seed=15)
    q0 = inputs.random_state(nx, ny, seed=16)
    q = oracle.run(q0, nt, 0.8, 3)
    _, _, f, d = run_gpu(nt, 0.8, q0, 3)
    want = oracle.fields(q, nt)
    for c, k in enumerate(("Ex", "Ey", "Ez", "Bx", "By", "Bz")):
        assert rel_l2(f[k], want[c]) <= 1e-12, k
    wd = oracle.divergence(q, nt, 0.8)
    for k in qla.DIV_KEYS:
        assert d[k] == pytest.approx(wd[k], rel=1e-10), k


def test_errors():
    n = np.full((16, 64), 1.5)
    with qla.Grid(64, 16, 1.0, "fp64") as g:               # made without the flag
        with pytest.raises(qla.QLAError) as e:
            g.set_medium(np.stack([n, n, n]))
        assert e.value.status == 1
    with qla.Grid(64, 16, 1.0, "fp64", tensor=True) as g:
        bad = np.stack([n, n.copy(), n.copy()])
        bad[1, 3, 5] = 0.0
        with pytest.raises(qla.QLAError) as e:
            g.set_medium(bad)
        assert e.value.status == 1
        with pytest.raises(qla.QLAError) as e:
            g.set_step_kernel("march")
        assert e.value.status == 1
