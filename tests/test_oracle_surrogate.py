"""Pins of the surrogate's FP64 reference (oracle/surrogate.py)."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import surrogate as ref


def test_parameter_count_matches_the_shapes():
    n = sum(co * ci * 9 + co for ci, co in ref.conv_shapes())
    assert ref.param_count() == n
    assert ref.conv_shapes()[0] == (6, 32) and ref.conv_shapes()[-1] == (32, 3)


def test_tap_orientation_and_circular_padding():
    """A kernel with a single 1 at (ky, kx) = (0, 1) reads in[y - 1, x]:
    out[y, x] = sum W[ky, kx] in[y + ky - 1, x + kx - 1], periodic."""
    x = torch.arange(5 * 7, dtype=torch.float64).reshape(1, 1, 5, 7)
    w = torch.zeros(1, 1, 3, 3, dtype=torch.float64)
    w[0, 0, 0, 1] = 1.0
    y = ref.conv(x, w)
    assert torch.equal(y, torch.roll(x, shifts=1, dims=2))
    w = torch.zeros(1, 1, 3, 3, dtype=torch.float64)
    w[0, 0, 1, 2] = 1.0   # reads in[y, x + 1]
    assert torch.equal(ref.conv(x, w), torch.roll(x, shifts=-1, dims=3))


def test_pool_and_upsample_are_adjoint_up_to_four():
    rng = np.random.default_rng(0)
    a = torch.as_tensor(rng.standard_normal((2, 3, 8, 6)))
    b = torch.as_tensor(rng.standard_normal((2, 3, 4, 3)))
    lhs = (F.avg_pool2d(a, 2) * b).sum()
    rhs = (a * F.interpolate(b, scale_factor=2, mode="nearest")).sum() / 4
    assert float(lhs) == pytest.approx(float(rhs), rel=1e-13)


def test_periodic_shift_equivariance():
    """Circular convolutions and 2x2 pooling at four levels commute with
    periodic shifts by multiples of 16."""
    rng = np.random.default_rng(1)
    theta = rng.standard_normal(ref.param_count()) * 0.05
    f = rng.standard_normal((1, 32, 32, 6))
    y = ref.forward(theta, f)
    ys = ref.forward(theta, np.roll(f, (16, 16), axis=(1, 2)))
    assert np.allclose(np.roll(y, (16, 16), axis=(1, 2)), ys, atol=1e-12)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    theta = rng.standard_normal(ref.param_count()) * 0.05
    f = rng.standard_normal((1, 16, 16, 6))
    t = rng.standard_normal((1, 16, 16, 3)) * 0.1
    loss, g = ref.loss_grad(theta, f, t)
    idx = rng.choice(theta.size, 24, replace=False)
    # include first-layer, a decoder bias and last-layer entries
    idx = np.concatenate([idx, [0, ref.param_count() - 1, ref.param_count() - 4]])
    h = 1e-6
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        lp, _ = ref.loss_grad(tp, f, t)
        lm, _ = ref.loss_grad(tm, f, t)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])), (k, fd, g[k])
