"""Pins of the oracle's three-dimensional step.  The paper prints the x and
y sequences only; the z construction is read off Eq. 3b4 (see the oracle
header).  What fixes it independently of that construction: the generator
(step - I)/delta^2 converging at second order to the right-hand side of
Eq. 3b4 in all six components, rigid translation of a vacuum wave along z,
the exact reduction to the 2D step for fields and media uniform in z, and
energy conservation (unitarity of the rotation reading)."""
import math

import numpy as np
import pytest

import oracle
from paper_2604_21128_gb300 import inputs

oracle.set_threads(min(8, max(1, __import__("os").cpu_count() or 1)))


def _generator_error_3d(N, L=32.0):
    k = 2 * math.pi / L
    d = L / N
    ax = np.arange(N) * d
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    n = 1.5 + 0.3 * np.sin(k * x) + 0.2 * np.cos(k * y) + 0.25 * np.sin(k * z + 0.4)
    nx_, ny_, nz_ = 0.3 * k * np.cos(k * x), -0.2 * k * np.sin(k * y), 0.25 * k * np.cos(k * z + 0.4)
    spec = [(1, 2, 1, 0.1), (2, -1, 1, 0.7), (1, 1, -2, 1.3), (-1, 2, 1, 2.1), (2, 1, 1, 0.4),
            (1, -2, 2, 1.9)]
    q, gx, gy, gz = [], [], [], []
    for m, p, r, ph in spec:
        arg = k * (m * x + p * y + r * z) + ph
        q.append(np.sin(arg))
        gx.append(k * m * np.cos(arg))
        gy.append(k * p * np.cos(arg))
        gz.append(k * r * np.cos(arg))
    q = np.array(q)
    # Eq. 3b4 with i dQ/dt = (W^-1/2 M W^-1/2) Q, isotropic n; d(f/n) expanded
    r = np.zeros_like(q)
    r[0] = gy[5] / n - gz[4] / n
    r[1] = gz[3] / n - gx[5] / n
    r[2] = -gy[3] / n + gx[4] / n
    r[3] = gz[1] / n - q[1] * nz_ / n ** 2 - gy[2] / n + q[2] * ny_ / n ** 2
    r[4] = -gz[0] / n + q[0] * nz_ / n ** 2 + gx[2] / n - q[2] * nx_ / n ** 2
    r[5] = gy[0] / n - q[0] * ny_ / n ** 2 - gx[1] / n + q[1] * nx_ / n ** 2
    G = (oracle.run3(q, n, d, 1) - q) / d ** 2
    return max(np.linalg.norm(G[c] - r[c]) / np.linalg.norm(r[c]) for c in range(6))


def test_generator_recovers_eq_3b4_at_second_order():
    e64, e128 = _generator_error_3d(64), _generator_error_3d(128)
    print("3D generator error: %.3e %.3e (ratio %.2f)" % (e64, e128, e64 / e128))
    assert e128 < 0.05 and 3.6 < e64 / e128 < 4.4, (e64, e128)


def test_generator_without_potential_does_not_converge():
    """Without V the gradient terms of Eq. 3b4 are missing (plateau)."""
    def err(N, L=32.0):
        k = 2 * math.pi / L
        d = L / N
        ax = np.arange(N) * d
        z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
        n = 1.5 + 0.3 * np.sin(k * z)
        q = np.zeros((6, N, N, N))
        q[1] = np.sin(k * (z + 2 * x))
        G = (oracle.run3(q, n, d, 1, "none") - q) / d ** 2
        want = -q[1] * 0.3 * k * np.cos(k * z) / n ** 2 + np.cos(k * (z + 2 * x)) * k / n
        return np.linalg.norm(G[3] - want) / np.linalg.norm(want)
    e32, e64 = err(32), err(64)
    assert e64 > 0.05 and e32 / e64 < 2.0


@pytest.mark.parametrize("pol", ["Ex", "Ey"])
def test_vacuum_wave_translates_along_z(pol):
    """A plane wave in vacuum moving along +z: E_x with B_y = E_x (q0, q4) or
    E_y with B_x = -E_y (q1, q3) (Eq. 3b4 with n = 1); it must arrive at
    z0 + T with second-order convergence in delta."""
    errs = []
    for delta in (0.5, 0.25):
        N = int(64 / delta)
        zz = np.arange(N) * delta
        f = np.exp(-(zz - 20.0) ** 2 / 36.0) * np.cos(0.5 * zz)
        q = np.zeros((6, N, 2, 2))
        if pol == "Ex":
            q[0], q[4] = f[:, None, None], f[:, None, None]
            c = 0
        else:
            q[1], q[3] = f[:, None, None], -f[:, None, None]
            c = 1
        T = 16.0
        qT = oracle.run3(q, np.ones((N, 2, 2)), delta, int(round(T / delta ** 2)))
        exact = np.exp(-(zz - 20.0 - T) ** 2 / 36.0) * np.cos(0.5 * (zz - T))
        errs.append(np.linalg.norm(qT[c, :, 0, 0] - exact) / np.linalg.norm(exact))
    # O(delta^2) truncation as in the 2D vacuum test; a wave going the wrong
    # way or at the wrong speed gives O(1)
    assert errs[1] < 0.07 and 3.5 < errs[0] / errs[1] < 4.5, errs


def test_z_uniform_fields_reduce_to_the_2d_step():
    nx, ny, nz = 24, 20, 5
    n2 = inputs.random_medium(nx, ny, seed=1, lo=1.0, hi=3.0)
    q2 = inputs.random_state(nx, ny, seed=2)
    q3 = np.repeat(q2[:, None], nz, axis=1)
    got = oracle.run3(q3, np.repeat(n2[None], nz, axis=0), 0.7, 6)
    want = oracle.run(q2, n2, 0.7, 6)
    assert np.max(np.abs(got - want[:, None])) < 1e-13


def test_energy_conserved_in_3d():
    rng = np.random.default_rng(3)
    n = 1.0 + 2.0 * rng.random((6, 10, 12))
    q = rng.standard_normal((6, 6, 10, 12))
    qT = oracle.run3(q, n, 1.0, 20)
    assert abs(np.sum(qT ** 2) / np.sum(q ** 2) - 1) < 1e-13


def _plane3(nx, ny, nz, m):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    kx, ky, kz = (2 * math.pi * m[0] / nx, 2 * math.pi * m[1] / ny, 2 * math.pi * m[2] / nz)
    return kx, ky, kz, np.sin(kx * x + ky * y + kz * z)


@pytest.mark.parametrize("delta", [1.0, 0.5])
def test_divergence3_closed_form(delta):
    """B = D = (s, s, s), s = sin(k.r): div = cos(k.r)(sin kx + sin ky + sin kz)/delta,
    so the sums are N/2 (sum of sines)^2 / delta^2 and N/2 (sum of squared
    sines) / delta^2; D enters as n q (q_E = s / n)."""
    nx, ny, nz = 20, 12, 16
    kx, ky, kz, s = _plane3(nx, ny, nz, (3, 2, 5))
    rng = np.random.default_rng(2)
    n = 1.0 + rng.random((nz, ny, nx))
    q = np.zeros((6, nz, ny, nx))
    q[3] = q[4] = q[5] = s
    q[0] = q[1] = q[2] = s / n
    d = oracle.divergence3(q, n, delta)
    N = nx * ny * nz
    sines = (math.sin(kx), math.sin(ky), math.sin(kz))
    for key in ("b", "d"):
        assert d["div_%s_sq" % key] == pytest.approx(N / 2 * sum(sines) ** 2 / delta ** 2, rel=1e-12)
        assert d["grad_%s_sq" % key] == pytest.approx(N / 2 * sum(v * v for v in sines)
                                                       / delta ** 2, rel=1e-12)


def test_divergence3_of_a_discrete_curl_is_zero():
    """B = curl A and D = curl A (q_E = (curl A)/n) with centred differences:
    the differences commute, so both divergences vanish to rounding."""
    nx, ny, nz, delta = 13, 11, 9, 0.7
    rng = np.random.default_rng(5)
    A = rng.standard_normal((3, nz, ny, nx))
    n = 1.0 + rng.random((nz, ny, nx))
    d = lambda f, ax: (np.roll(f, -1, ax) - np.roll(f, 1, ax)) / (2 * delta)   # ax: 2 x, 1 y, 0 z
    curl = np.array([d(A[2], 1) - d(A[1], 0), d(A[0], 0) - d(A[2], 2), d(A[1], 2) - d(A[0], 1)])
    q = np.zeros((6, nz, ny, nx))
    q[3:6] = curl
    q[0:3] = curl / n
    r = oracle.divergence3(q, n, delta)
    assert r["div_b_sq"] <= 1e-28 * r["grad_b_sq"]
    assert r["div_d_sq"] <= 1e-28 * r["grad_d_sq"]
    assert r["grad_b_sq"] > 1.0


def test_divergence3_of_z_uniform_fields_is_the_2d_one():
    nx, ny, nz = 24, 20, 5
    n2 = inputs.random_medium(nx, ny, seed=9, lo=1.0, hi=3.0)
    q2 = inputs.random_state(nx, ny, seed=10)
    d3 = oracle.divergence3(np.repeat(q2[:, None], nz, axis=1), np.repeat(n2[None], nz, axis=0), 0.8)
    d2 = oracle.divergence(q2, n2, 0.8)
    for k in ("div_b_sq", "grad_b_sq", "div_d_sq", "grad_d_sq"):
        assert d3[k] == pytest.approx(nz * d2[k], rel=1e-12)
    assert d3["div_b_max"] == pytest.approx(d2["div_b_max"], rel=1e-12)
