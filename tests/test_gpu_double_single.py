"""QLA_DOUBLE_SINGLE: FP64 contexts stepped in double-single arithmetic,
against the oracle (the FP64 bar, 1e-12 relative L2) and against the native
FP64 kernels (rounding-level differences only)."""
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


def run(n, delta, steps, q0=None, packet=None, te=False, potential="rotation", ds=True,
        calls=1):
    ny, nx = n.shape
    with qla.Grid(nx, ny, delta, "fp64", te_only=te, potential=potential,
                  double_single=ds) as g:
        g.set_medium(n)
        if q0 is not None:
            g.set_state(q0)
        else:
            g.set_packet(**packet)
        for _ in range(calls):
            g.step(steps // calls)
        return g.get_state(), g.energy()


@pytest.mark.parametrize("te", [True, False])
def test_ellipse_256_400_steps(te):
    w = inputs.ellipse_256()
    n = w.medium()
    pk = w.packet.as_dict()
    want = oracle.run(oracle.packet(n, w.delta, **pk), n, w.delta, w.steps)
    got, e = run(n, w.delta, w.steps, packet=pk, te=te)
    err = rel_l2(got, want)
    print("double-single 400 steps (te=%s): rel L2 %.3e" % (te, err))
    assert err <= 1e-12
    assert abs(e / oracle.energy(want) - 1) <= 1e-12


@pytest.mark.parametrize("te", [True, False])
@pytest.mark.parametrize("potential", ["rotation", "none"])
@pytest.mark.parametrize("shape", [(64, 8), (66, 9), (128, 37), (250, 64), (96, 130)])
def test_random_state_against_oracle_and_native(shape, potential, te):
    nx, ny = shape
    n = inputs.random_medium(nx, ny, seed=nx * 17 + ny, lo=1.0, hi=3.5)
    q0 = inputs.random_state(nx, ny, seed=nx + 5 * ny)
    if te:
        q0[[0, 1, 5]] = 0.0
    want = oracle.run(q0, n, 0.8, 9, potential)
    got, _ = run(n, 0.8, 9, q0=q0, te=te, potential=potential)
    native, _ = run(n, 0.8, 9, q0=q0, te=te, potential=potential, ds=False)
    assert rel_l2(got, want) <= 1e-12, rel_l2(got, want)
    assert rel_l2(got, native) <= 1e-13, rel_l2(got, native)


@pytest.mark.parametrize("potential", ["rotation", "none"])
def test_six_planes_step_each_triple_like_the_e_z_kernel(potential):
    """The operators never couple (q2, q3, q4) with (q0, q1, q5), and a
    six-plane double-single step runs one launch per triple: its (q2, q3, q4)
    planes must be bit-identical to an E_z context's on the same triple, and
    the other triple must not depend on the first."""
    nx, ny = 250, 64
    n = inputs.random_medium(nx, ny, seed=3, lo=1.0, hi=3.5)
    q0 = inputs.random_state(nx, ny, seed=11)
    six, _ = run(n, 0.8, 9, q0=q0, potential=potential)
    te = q0.copy()
    te[[0, 1, 5]] = 0.0
    tri, _ = run(n, 0.8, 9, q0=te, te=True, potential=potential)
    assert np.array_equal(six[[2, 3, 4]], tri[[2, 3, 4]])
    tm = q0.copy()
    tm[[2, 3, 4]] = 0.0
    other, _ = run(n, 0.8, 9, q0=tm, potential=potential)
    assert np.array_equal(six[[0, 1, 5]], other[[0, 1, 5]])
    assert not np.any(other[[2, 3, 4]])


def test_launch_counts_match_the_kernels_each_step_runs():
    """A double-single call converts the state twice and launches the
    marching kernel once per step, twice with six planes (one launch per
    triple); in 3D a step is two slices launches (one per triple) and the
    column launch."""
    nx, ny = 128, 40
    n = inputs.random_medium(nx, ny, seed=1, lo=1.0, hi=3.0)
    q0 = inputs.random_state(nx, ny, seed=2)
    for te, per_step in ((True, 1), (False, 2)):
        q = q0.copy()
        if te:
            q[[0, 1, 5]] = 0.0
        with qla.Grid(nx, ny, 0.8, "fp64", te_only=te, double_single=True) as g:
            g.set_medium(n)
            g.set_state(q)
            before = g.launches
            g.step(5)
            assert g.launches - before == 2 + 5 * per_step, te
    nz = 16
    n3 = np.ones((nz, ny, nx))
    with qla.Grid3(nx, ny, nz, 0.9, "fp64", double_single=True) as g3:
        g3.set_medium(n3)
        g3.set_packet(x0=30.0, y0=20.0, angle=0.0, k0=0.3, width=6.0)
        before = g3.launches
        g3.step(4)
        assert g3.launches - before == 2 + 4 * 3


def test_split_calls_agree_with_one_call():
    # each call converts the state to word pairs and back
    w = inputs.scaled(inputs.ellipse_256(), 128, 128, 60)
    n = w.medium()
    pk = w.packet.as_dict()
    want = oracle.run(oracle.packet(n, w.delta, **pk), n, w.delta, 60)
    one, _ = run(n, w.delta, 60, packet=pk, te=True)
    many, _ = run(n, w.delta, 60, packet=pk, te=True, calls=6)
    assert rel_l2(one, want) <= 1e-12
    assert rel_l2(many, want) <= 1e-12
    assert rel_l2(many, one) <= 1e-13


@pytest.mark.parametrize("kw", [dict(precision="fp32"), dict(potential="literal"),
                                dict(potential="lcu"), dict(tensor=True),
                                dict(nx=32), dict(nx=65), dict(ny=4)])
def test_rejected_configurations(kw):
    args = dict(nx=64, ny=16, precision="fp64", potential="rotation", tensor=False)
    args.update(kw)
    with pytest.raises(qla.QLAError):
        qla.Grid(args["nx"], args["ny"], 1.0, args["precision"], potential=args["potential"],
                 tensor=args["tensor"], double_single=True)


def medium3(nx, ny, nz, seed):
    rng = np.random.default_rng(seed)
    raw = rng.random((nz, ny, nx))
    for ax in range(3):
        raw = (raw + np.roll(raw, 1, ax) + np.roll(raw, -1, ax)) / 3
    return 1.0 + 2.5 * raw


@pytest.mark.parametrize("potential", ["rotation", "none"])
@pytest.mark.parametrize("shape", [(64, 8, 3), (66, 9, 5), (128, 20, 12)])
def test_3d_against_oracle_and_native(shape, potential):
    nx, ny, nz = shape
    n = medium3(nx, ny, nz, seed=nx + ny + nz)
    q0 = np.random.default_rng(nx * ny + nz).standard_normal((6, nz, ny, nx))
    steps = 6
    want = oracle.run3(q0, n, 0.9, steps, potential)
    out = {}
    for ds in (True, False):
        with qla.Grid3(nx, ny, nz, 0.9, "fp64", potential=potential, double_single=ds) as g:
            g.set_medium(n)
            g.set_state(q0)
            g.step(steps)
            out[ds] = g.get_state()
    assert rel_l2(out[True], want) <= 1e-12, rel_l2(out[True], want)
    assert rel_l2(out[True], out[False]) <= 1e-13, rel_l2(out[True], out[False])


@pytest.mark.parametrize("kw", [dict(precision="fp32"), dict(nx=32), dict(nx=65), dict(ny=4)])
def test_3d_rejected_configurations(kw):
    args = dict(nx=64, ny=16, nz=4, precision="fp64")
    args.update(kw)
    with pytest.raises(qla.QLAError):
        qla.Grid3(args["nx"], args["ny"], args["nz"], 1.0, args["precision"], double_single=True)


@pytest.mark.parametrize("rows,potential", [(0, "rotation"), (24, "rotation"), (16, "none")])
def test_plateau_split_bitwise(rows, potential):
    """E_z double-single steps split by plateaus (64-column plateau items
    without the record ring) give the bits of the unsplit kernel; the 256^2
    ellipse-like medium with sharp plateaus and a rough patch has items of
    both kinds."""
    nx, ny = 512, 320
    y, x = np.mgrid[0:ny, 0:nx]
    n = np.full((ny, nx), 2.0)
    n[((x - nx / 2) / (nx / 5)) ** 2 + ((y - ny / 2) / (ny / 4)) ** 2 < 1.0] = 1.0
    n[-40:, -70:] = np.random.default_rng(7).uniform(1.2, 2.8, (40, 70))
    q0 = inputs.random_state(nx, ny, seed=41, planes=3)
    out = {}
    for kernel in ("march", "march_plain"):
        with qla.Grid(nx, ny, 1.0, "fp64", te_only=True, potential=potential,
                      double_single=True) as g:
            g.set_step_kernel(kernel)
            g.set_march_tuning(0, rows)
            g.set_medium(n)
            g.set_state(q0)
            g.step(9)
            out[kernel] = (g.get_state(), g.energy(), g.march_plan)
    items, plateau, recs = out["march"][2]
    assert recs == 2 and 0 < plateau < items, out["march"][2]
    assert out["march_plain"][2] == (0, 0, 0)
    assert np.array_equal(out["march"][0], out["march_plain"][0])
    assert out["march"][1] == out["march_plain"][1]
    want = oracle.run(q0, n, 1.0, 9, potential)
    assert rel_l2(out["march"][0], want) <= 1e-12
