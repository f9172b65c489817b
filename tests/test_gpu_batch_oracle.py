"""Batched lattices against the oracle at the sizes of the 256-instance
workload (square sides 512 to 2048, seeded ellipses, indices and packets):
every instance advanced by the persistent batched kernel, then compared with
the oracle (Eq. 2e14 applied operator by operator) element by element, or on
sampled sites for the 1536 and 2048 sides (periodic oracle windows around
each site, exact inside the dependence cone).  The whole 256-instance batch
is also advanced in its graph-captured form and sampled."""
import os

import numpy as np
import pytest

import oracle
from paper_2604_21128_gb300 import build as qbuild
from paper_2604_21128_gb300 import inputs, qla

pytestmark = pytest.mark.gpu

FULL_SIDES = (512, 768, 1024)     # compared at every site
# FP32 bounds after a few tens of steps: relative L2 of the whole state, and
# absolute per sampled site relative to the packet amplitude (1)
FP32_REL_L2 = 1e-6
FP32_SITE = 2e-6


@pytest.fixture(scope="module", autouse=True)
def _setup():
    qbuild.build()
    oracle.set_threads(os.cpu_count() or 1)


def _pick():
    """Two 512^2 instances and the first instance of every other side."""
    out, seen = [], {}
    for w in inputs.batch_instances():
        c = seen.get(w.nx, 0)
        if c < (2 if w.nx == 512 else 1):
            out.append(w)
            seen[w.nx] = c + 1
    return out


def _sites(w, rng, count=10):
    """Sampled sites: around the packet, on the ellipse's edge band, at
    random, and on the wrap-around edges."""
    pk = w.packet
    i = np.concatenate([int(pk.x0) + rng.integers(-w.nx // 10, w.nx // 10, count // 2),
                        rng.integers(0, w.nx, count - count // 2), [0, w.nx - 1]])
    j = np.concatenate([int(pk.y0) + rng.integers(-w.ny // 10, w.ny // 10, count // 2),
                        rng.integers(0, w.ny, count - count // 2), [w.ny - 1, 0]])
    return i % w.nx, j % w.ny


def _rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("precision,te,tuning", [
    ("fp64", False, (2, 0)),
    ("fp32", True, (1, 0)),
    ("fp32", True, (1, 64)),
    ("fp32", True, (2, 0)),
    ("fp32", True, (4, 0)),
    ("fp32", True, (4, 64)),
    ("fp32", True, "auto"),
])
def test_batch_matches_oracle_at_workload_sizes(precision, te, tuning):
    ws = _pick()
    assert sorted({w.nx for w in ws}) == [512, 768, 1024, 1536, 2048]
    steps1, steps2 = 13, 17
    steps = steps1 + steps2
    media = [w.medium() for w in ws]
    with qla.Batch([(w.nx, w.ny) for w in ws], 1.0, precision, te_only=te) as b:
        if tuning == "auto":
            for k, w in enumerate(ws):
                b.instance(k).set_medium(media[k])
                b.instance(k).set_packet(**w.packet.as_dict())
            b.autotune(trial_steps=1)
        else:
            b.set_tuning(*tuning)
        for k, w in enumerate(ws):
            g = b.instance(k)
            g.set_medium(media[k])
            g.set_packet(**w.packet.as_dict())
        b.step(steps1)
        b.step(steps2)
        energies = b.energy()
        rng = np.random.default_rng(424242)
        for k, w in enumerate(ws):
            g = b.instance(k)
            pk = w.packet.as_dict()
            if w.nx in FULL_SIDES:
                got = g.get_state()
                want = oracle.run(oracle.packet(media[k], w.delta, **pk), media[k], w.delta,
                                  steps)
                err = _rel_l2(got, want)
                print("%s %s side %d: rel L2 %.2e" % (precision, tuning, w.nx, err))
                assert err <= (1e-12 if precision == "fp64" else FP32_REL_L2), (w.nx, err)
                assert abs(energies[k] / oracle.energy(want) - 1) <= \
                    (1e-12 if precision == "fp64" else 1e-6)
                if te:
                    assert np.all(got[[0, 1, 5]] == 0)
            else:
                ii, jj = _sites(w, rng)
                got = g.probe(ii, jj)
                half = oracle.reach_per_step() * steps + 2
                worst = 0.0
                for s in range(len(ii)):
                    want = oracle.run_window(media[k], w.delta, pk, steps,
                                             (int(ii[s]), int(jj[s])), half)
                    d = float(np.max(np.abs(got[s] - want)))
                    worst = max(worst, d)
                    tol = 1e-12 * max(1.0, float(np.max(np.abs(want)))) \
                        if precision == "fp64" else FP32_SITE
                    assert d <= tol, (w.nx, ii[s], jj[s], got[s], want)
                print("%s %s side %d: worst sampled site %.2e" % (precision, tuning, w.nx, worst))


def test_all_256_instances_graph_run_sampled_against_oracle():
    """The full workload: 256 uneven lattices (433 M sites, FP32, E_z planes)
    in one batch, advanced by the graph-captured persistent run with the
    autotuned tiling; two sampled sites of every eighth instance against the
    oracle, and every instance's energy conserved."""
    ws = inputs.batch_instances()
    assert len(ws) == 256
    with qla.Batch([(w.nx, w.ny) for w in ws], 1.0, "fp32", te_only=True) as b:
        media = {}
        for k, w in enumerate(ws):
            n = w.medium()
            if k % 8 == 0:
                media[k] = n
            b.instance(k).set_medium(n)
            b.instance(k).set_packet(**w.packet.as_dict())
        b.autotune(trial_steps=1)
        for k, w in enumerate(ws):
            b.instance(k).set_packet(**w.packet.as_dict())
        e0 = b.energy()
        steps, every = 12, 4
        e = b.run(steps, every)
        assert e.shape == (steps // every, 256)
        drift = np.max(np.abs(e / e0[None, :] - 1))
        print("256 instances: max energy drift %.2e over %d steps" % (drift, steps))
        assert drift <= 1e-6
        rng = np.random.default_rng(256)
        half = oracle.reach_per_step() * steps + 2
        worst = 0.0
        for k in sorted(media):
            w = ws[k]
            pk = w.packet.as_dict()
            ii = np.array([int(pk["x0"]) + int(rng.integers(-20, 20)), int(rng.integers(0, w.nx))])
            jj = np.array([int(pk["y0"]) + int(rng.integers(-20, 20)), int(rng.integers(0, w.ny))])
            ii, jj = ii % w.nx, jj % w.ny
            got = b.instance(k).probe(ii, jj)
            for s in range(2):
                want = oracle.run_window(media[k], w.delta, pk, steps, (int(ii[s]), int(jj[s])),
                                         half)
                d = float(np.max(np.abs(got[s] - want)))
                worst = max(worst, d)
                assert d <= FP32_SITE, (k, ii[s], jj[s], got[s], want)
        print("256 instances: worst sampled site %.2e" % worst)
