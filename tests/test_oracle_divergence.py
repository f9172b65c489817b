"""Pins of the oracle's Gauss-law monitors (Eqs. 3.1, 3.2; centred periodic
differences, the reading taken where the paper does not state the discrete
derivative).  Closed forms on plane-wave fields, the discrete identity
div(curl) = 0, and the exactly divergence-free planar packet."""
import math

import numpy as np
import pytest

import oracle



def _plane(nx, ny, mx, my):
    i = np.arange(nx)[None, :]
    j = np.arange(ny)[:, None]
    kx, ky = 2 * math.pi * mx / nx, 2 * math.pi * my / ny
    return kx, ky, np.sin(kx * i + ky * j)


@pytest.mark.parametrize("delta", [1.0, 0.25])
def test_closed_form_on_plane_waves(delta):
    """B = D = (s, s) with s = sin(kx i + ky j): the centred difference of s
    along x is cos(.) sin(kx) / delta, so over the lattice (sum of cos^2 =
    N / 2) div_sq = N/2 (sin kx + sin ky)^2 / delta^2 and the scale is
    N/2 (sin^2 kx + sin^2 ky) / delta^2.  D enters as n q: q0 = q1 = s / n."""
    nx, ny = 48, 30
    kx, ky, s = _plane(nx, ny, 5, 2)
    rng = np.random.default_rng(1)
    n = 1.0 + rng.random((ny, nx))
    q = np.zeros((6, ny, nx))
    q[3] = q[4] = s
    q[0] = q[1] = s / n
    d = oracle.divergence(q, n, delta)
    N = nx * ny
    want_div = N / 2 * (math.sin(kx) + math.sin(ky)) ** 2 / delta ** 2
    want_grad = N / 2 * (math.sin(kx) ** 2 + math.sin(ky) ** 2) / delta ** 2
    for key in ("b", "d"):
        assert d["div_%s_sq" % key] == pytest.approx(want_div, rel=1e-12)
        assert d["grad_%s_sq" % key] == pytest.approx(want_grad, rel=1e-12)
    # the maximum of |cos(.)| (sin kx + sin ky) / delta over the lattice sites
    i = np.arange(nx)[None, :]
    j = np.arange(ny)[:, None]
    cmax = np.max(np.abs(np.cos(kx * i + ky * j)))
    assert d["div_b_max"] == pytest.approx(cmax * (math.sin(kx) + math.sin(ky)) / delta, rel=1e-12)


def test_opposite_components_cancel_only_with_the_right_signs():
    """B = (s, -s) with kx = ky: div = cos(.) (sin kx - sin ky) = 0."""
    nx = ny = 40
    kx, ky, s = _plane(nx, ny, 3, 3)
    q = np.zeros((6, ny, nx))
    q[3], q[4] = s, -s
    d = oracle.divergence(q, np.ones((ny, nx)), 1.0)
    assert d["div_b_sq"] <= 1e-26 * d["grad_b_sq"]
    assert d["grad_b_sq"] == pytest.approx(nx * ny * math.sin(kx) ** 2, rel=1e-12)


def test_discrete_curl_is_divergence_free():
    """With centred differences D_x D_y = D_y D_x, so B = (D_y A, -D_x A) and
    D = (D_y A, -D_x A) have zero divergence to rounding for any A and n."""
    nx, ny, delta = 37, 29, 0.5
    rng = np.random.default_rng(7)
    A = rng.standard_normal((ny, nx))
    n = 1.0 + 2.0 * rng.random((ny, nx))
    dxA = (np.roll(A, -1, axis=1) - np.roll(A, 1, axis=1)) / (2 * delta)
    dyA = (np.roll(A, -1, axis=0) - np.roll(A, 1, axis=0)) / (2 * delta)
    q = np.zeros((6, ny, nx))
    q[3], q[4] = dyA, -dxA
    q[0], q[1] = dyA / n, -dxA / n
    d = oracle.divergence(q, n, delta)
    assert d["div_b_sq"] <= 1e-28 * d["grad_b_sq"]
    assert d["div_d_sq"] <= 1e-28 * d["grad_d_sq"]
    assert d["grad_b_sq"] > 1.0


def test_planar_packet_along_x_is_exactly_divergence_free():
    """A planar E_z packet moving along +x has B = (0, -q2(x)): no term of
    div B survives, exactly (and D has no in-plane part).  (A packet with a
    transverse envelope is not divergence-free even in the continuum: its
    plane-wave B has div B = -dF/d(eta).)"""
    nx, ny = 64, 16
    n = np.full((ny, nx), 1.5)
    q = oracle.packet(n, 1.0, 20.0, 8.0, 0.0, 0.3, 6.0)
    d = oracle.divergence(q, n, 1.0)
    assert np.abs(q[4]).max() > 0.1
    assert d["div_b_sq"] == 0.0 and d["grad_b_sq"] == 0.0 and d["div_d_sq"] == 0.0


def test_qla_keeps_div_b_zero_to_second_order():
    """Maxwell's equations keep div B at its initial value; a scheme
    consistent with them to O(delta^2) (Eq. 2e14) keeps the discrete div B
    of a divergence-free start at O(delta^2).  Same physical problem (a
    planar E_z packet in vacuum heading into a tilted dielectric ellipse,
    t = 20) at delta = 1/2 and 1/4: the relative divergence must fall by
    more than 3 (second order: 4; first order would give 2)."""
    from paper_2604_21128_gb300 import inputs
    L, T = 64.0, 20.0
    rel = []
    for delta in (0.5, 0.25):
        N = int(L / delta)
        n = inputs.ellipse_medium(N, N, delta, a=9.0, b=6.0, n_in=2.0, n_out=1.0, edge=2.0,
                                  angle=0.5, centre=(42.0, L / 2))
        q = oracle.packet(n, delta, 14.0, L / 2, 0.0, 0.5, 3.0)
        d0 = oracle.divergence(q, n, delta)
        q = oracle.run(q, n, delta, int(round(T / delta ** 2)))
        d = oracle.divergence(q, n, delta)
        # divergence-free start (the packet's tails barely touch the medium)
        assert math.sqrt(d0["div_b_sq"] / d["grad_b_sq"]) < 1e-6
        rel.append(math.sqrt(d["div_b_sq"] / d["grad_b_sq"]))
    print("relative div B at delta 1/2, 1/4: %.3e %.3e (ratio %.2f)" % (rel[0], rel[1], rel[0] / rel[1]))
    assert rel[0] / rel[1] > 3.0
    assert rel[1] < 0.03


def test_tensor_medium_uses_n_x_and_n_y_for_d():
    """D = (n_x q0, n_y q1): with q0 = s / n_x and q1 = s / n_y the closed form
    of the plane wave holds; dividing by the wrong components breaks it."""
    nx, ny = 48, 30
    kx, ky, s = _plane(nx, ny, 5, 2)
    rng = np.random.default_rng(5)
    nt = 1.0 + rng.random((3, ny, nx))
    q = np.zeros((6, ny, nx))
    q[0], q[1] = s / nt[0], s / nt[1]
    d = oracle.divergence(q, nt, 1.0)
    N = nx * ny
    assert d["div_d_sq"] == pytest.approx(N / 2 * (math.sin(kx) + math.sin(ky)) ** 2, rel=1e-12)
    q[0], q[1] = s / nt[1], s / nt[0]
    assert oracle.divergence(q, nt, 1.0)["div_d_sq"] != pytest.approx(d["div_d_sq"], rel=1e-3)
