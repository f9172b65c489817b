"""The dependency rule of the dataflow steps, on the CPU.

A dataflow launch lets a unit of step s start as soon as the items listed
by qla_flow_item_deps have finished step s - 1 (see include/qla.h).  Two
checks, neither using the GPU:

* The lists against brute force over sets of sites: for every pair of
  items of several ragged plans, whether one's reads meet the other's
  stored sites (either way), with the reads of both kinds of unit a plan
  can hold (a 128-column plateau window from 4 columns left of its stored
  ones; two-column units of 56 stored columns, each reading 64 from 4
  left) and four rows either side of a segment.
* An adversarial schedule: units of a small lattice run one at a time in
  an order that runs ahead wherever the lists allow, each reading the
  current contents of its input buffer, advancing it by one step of
  Eq. 2e14 (the oracle) and keeping only its own stored sites.  The result
  must be the oracle's sequential run bit for bit; with each item waiting
  only for itself it is not."""
import itertools
import os
import random

import numpy as np
import pytest

import oracle
from paper_2604_21128_gb300 import inputs, qla

PWOUT, PW, GWOUT, LAG = 120, 128, 56, 4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    try:
        qla.load()
    except OSError as e:
        pytest.skip(str(e))
    oracle.set_threads(min(4, os.cpu_count() or 1))


def geometry(nx, ny, seg):
    """(x, w, y, h) of every item, item = segment * windows + window."""
    n_wx, n_wy = -(-nx // PWOUT), -(-ny // seg)
    out = []
    for wy in range(n_wy):
        for wx in range(n_wx):
            x, y = wx * PWOUT, wy * seg
            out.append((x, min(PWOUT, nx - x), y, min(seg, ny - y)))
    return out


def read_cols(x, w, nx):
    """Columns (mod nx) a unit of this window reads, either kind of item."""
    cols = {(x - 4 + k) % nx for k in range(PW)}
    for xu in range(x, x + w, GWOUT):
        cols |= {(xu - 4 + k) % nx for k in range(64)}
    return cols


def sets(nx, ny, seg):
    """Per item: stored columns, stored rows, read columns, read rows."""
    out = []
    for x, w, y, h in geometry(nx, ny, seg):
        out.append(({c for c in range(x, x + w)}, {r for r in range(y, y + h)},
                    read_cols(x, w, nx), {(r % ny) for r in range(y - LAG, y + h + LAG)}))
    return out


GEOMS = [(128, 64, 32), (248, 100, 40), (256, 72, 16), (1000, 200, 32), (512, 36, 32),
         (360, 48, 16), (484, 40, 20), (16384, 1024, 192)]


@pytest.mark.parametrize("nx,ny,seg", GEOMS)
def test_dependency_lists_match_brute_force(nx, ny, seg):
    """Every pair whose reads and stored sites meet is listed; the list is
    exactly the product of the per-axis sets (columns that meet either way,
    rows that meet either way), the form the kernel polls."""
    s = sets(nx, ny, seg)
    n_wx = -(-nx // PWOUT)
    items = range(len(s)) if len(s) <= 200 else list(range(0, len(s), 37)) + [len(s) - 1]
    for a in items:
        deps = qla.qla_flow_item_deps(nx, ny, seg, a)
        assert len(deps) == len(set(deps)) <= 16, (a, deps)
        wcol_a, wrow_a, rcol_a, rrow_a = s[a]
        xs, ys = set(), set()
        for b, (wcol_b, wrow_b, rcol_b, rrow_b) in enumerate(s):
            meet_x = bool(rcol_a & wcol_b) or bool(rcol_b & wcol_a)
            meet_y = bool(rrow_a & wrow_b) or bool(rrow_b & wrow_a)
            needed = (bool(rcol_a & wcol_b) and bool(rrow_a & wrow_b)) or \
                     (bool(rcol_b & wcol_a) and bool(rrow_b & wrow_a))
            if needed:
                assert b in deps, (a, b, deps)
            if meet_x:
                xs.add(b % n_wx)
            if meet_y:
                ys.add(b // n_wx)
        assert set(deps) == {y * n_wx + x for x, y in itertools.product(xs, ys)}, (a, deps)


def test_dependency_lists_reject_other_geometries():
    for args in ((126, 64, 32, 0), (130, 64, 32, 0), (256, 64, 15, 0), (256, 64, 18, 0),
                 (256, 7, 16, 0), (256, 64, 16, 12), (256, 64, 16, -1)):
        with pytest.raises(qla.QLAError):
            qla.qla_flow_item_deps(*args)


def emulate(n, q0, steps, seg, deps_of, policy, seed):
    """Run the units of `steps` steps one at a time in the order `policy`
    picks among those whose dependencies (deps_of(item)) have finished the
    previous step; each unit advances its whole input buffer by one step
    with the oracle and keeps only its own stored sites."""
    ny, nx = n.shape
    geo = geometry(nx, ny, seg)
    deps = [deps_of(i) for i in range(len(geo))]
    buf = [q0.copy(), q0.copy()]
    done = [[False] * len(geo) for _ in range(steps)]
    rng = random.Random(seed)
    pending = [(s, i) for s in range(steps) for i in range(len(geo))]
    while pending:
        ready = [(s, i) for s, i in pending
                 if s == 0 or all(done[s - 1][d] for d in deps[i])]
        s, i = policy(ready, rng)
        pending.remove((s, i))
        x, w, y, h = geo[i]
        full = oracle.run(buf[s % 2], n, 1.0, 1)
        buf[(s + 1) % 2][:, y:y + h, x:x + w] = full[:, y:y + h, x:x + w]
        done[s][i] = True
    return buf[steps % 2]


def run_ahead(ready, rng):
    """The unit of the latest step that may run (ties at random)."""
    top = max(s for s, _ in ready)
    return rng.choice([u for u in ready if u[0] == top])


def at_random(ready, rng):
    return rng.choice(ready)


@pytest.mark.parametrize("nx,ny,seg,steps", [(256, 72, 16, 4), (128, 40, 16, 3)])
def test_adversarial_schedules_reproduce_the_sequential_run(nx, ny, seg, steps):
    n = inputs.random_medium(nx, ny, seed=51, lo=1.0, hi=2.5)
    q0 = inputs.random_state(nx, ny, seed=52, planes=3)
    want = oracle.run(q0, n, 1.0, steps)
    listed = lambda i: qla.qla_flow_item_deps(nx, ny, seg, i)
    for policy, seed in ((run_ahead, 1), (run_ahead, 2), (at_random, 3)):
        got = emulate(n, q0, steps, seg, listed, policy, seed)
        assert np.array_equal(got, want), policy.__name__
    # the same schedule with every item waiting only for itself: a unit of
    # step s then reads neighbours' sites that are not yet at step s - 1 or
    # already at step s + 1
    alone = emulate(n, q0, steps, seg, lambda i: [i], run_ahead, 1)
    assert not np.array_equal(alone, want)
