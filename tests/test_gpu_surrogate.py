"""Learned surrogate on the GPU: its contraction kernels against exact FP64
sums on BF16 data, its forward pass and parameter gradients against the
FP64 reference network (oracle/surrogate.py), training, and the fallback
path of surr_advance."""
import ctypes

import numpy as np
import pytest

from oracle import surrogate as ref
from paper_2604_21128_gb300 import build as qbuild
from paper_2604_21128_gb300 import inputs, qla
from paper_2604_21128_gb300 import surrogate as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    qbuild.build()


def _bf16(rng, shape, scale=1.0):
    import torch
    a = torch.tensor(rng.standard_normal(shape) * scale, dtype=torch.float32)
    return a.to(torch.bfloat16).cuda()


def _ref_conv(x_nhwc, w):
    """fp64 periodic conv: w [co][9][ci], x [B][H][W][ci] -> [B][H][W][co]."""
    import torch
    co, _, ci = w.shape
    W = w.double().cpu().reshape(co, 3, 3, ci).permute(0, 3, 1, 2).contiguous()
    x = x_nhwc.double().cpu().permute(0, 3, 1, 2)
    return ref.conv(x, W).permute(0, 2, 3, 1)


@pytest.mark.parametrize("B,H,W,cin,cout", [(2, 16, 16, 32, 32), (1, 8, 24, 64, 64),
                                            (1, 16, 16, 256, 128), (1, 7, 9, 32, 64),
                                            (3, 4, 4, 128, 256),
                                            # widths that are multiples of 128: row patches
                                            (1, 3, 128, 32, 32), (2, 2, 256, 64, 32),
                                            (1, 4, 128, 32, 64), (1, 2, 128, 128, 32),
                                            (1, 2, 256, 32, 128), (1, 2, 128, 64, 128),
                                            (1, 2, 128, 256, 32)])
def test_conv_kernel_is_exact_on_bf16_data(B, H, W, cin, cout):
    import torch
    rng = np.random.default_rng(B * 1000 + cin + cout)
    x = _bf16(rng, (B, H, W, cin))
    w = _bf16(rng, (cout, 9, cin), 0.1)
    out = torch.empty((B, H, W, cout), dtype=torch.float32, device="cuda")
    st = qla.load().surr_conv3x3_raw(ctypes.c_void_p(x.data_ptr()), B, H, W, cin,
                                     ctypes.c_void_p(w.data_ptr()), cout,
                                     ctypes.c_void_p(out.data_ptr()), None)
    assert st == 0
    torch.cuda.synchronize()
    want = _ref_conv(x, w).numpy()
    got = out.cpu().numpy()
    # products of BF16 values are exact in FP32; only the FP32 accumulation
    # of 9 * cin terms rounds (~sqrt(9 cin) * 6e-8 relative)
    assert np.linalg.norm(got - want) <= 1e-5 * np.linalg.norm(want)


@pytest.mark.parametrize("B,H,W,cout,cin,splits", [(2, 16, 16, 32, 32, 1), (1, 16, 32, 64, 32, 3),
                                                   (1, 8, 8, 256, 128, 2), (1, 5, 7, 32, 64, 2)])
def test_weight_grad_kernel_is_exact_on_bf16_data(B, H, W, cout, cin, splits):
    import torch
    rng = np.random.default_rng(7 + cout + cin)
    dz = _bf16(rng, (B, H, W, cout))
    x = _bf16(rng, (B, H, W, cin))
    part = torch.empty(splits * cout * 9 * cin, dtype=torch.float32, device="cuda")
    dw = torch.empty((cout, 9, cin), dtype=torch.float32, device="cuda")
    st = qla.load().surr_weight_grad_raw(ctypes.c_void_p(dz.data_ptr()),
                                         ctypes.c_void_p(x.data_ptr()), B, H, W, cout, cin, splits,
                                         ctypes.c_void_p(part.data_ptr()),
                                         ctypes.c_void_p(dw.data_ptr()), None)
    assert st == 0
    torch.cuda.synchronize()
    dzd, xd = dz.double().cpu(), x.double().cpu()
    want = np.empty((cout, 9, cin))
    for tap in range(9):
        dy, dx = tap // 3 - 1, tap % 3 - 1
        xs = torch.roll(xd, shifts=(-dy, -dx), dims=(1, 2))   # xs[y, x] = x[y + dy, x + dx]
        want[:, tap, :] = (dzd.reshape(-1, cout).T @ xs.reshape(-1, cin)).numpy()
    got = dw.cpu().numpy()
    assert np.linalg.norm(got - want) <= 1e-5 * np.linalg.norm(want)


def _net_and_data(B=2, H=32, W=32, seed=3, scale=0.05):
    import torch
    net = S.Surrogate(H, W, max_batch=B, seed=seed)
    rng = np.random.default_rng(seed)
    theta = (rng.standard_normal(net.nparams) * scale).astype(np.float32)
    net.set_params(theta)
    feat = torch.tensor(rng.standard_normal((B, H, W, 6)), dtype=torch.float32, device="cuda")
    target = torch.tensor(rng.standard_normal((B, H, W, 3)) * 0.1, dtype=torch.float32,
                          device="cuda")
    return net, theta, feat, target


def test_params_round_trip():
    net, theta, _, _ = _net_and_data()
    assert net.nparams == ref.param_count()
    assert np.array_equal(net.params(), theta)


@pytest.mark.parametrize("B,H,W", [(2, 32, 32), (1, 32, 128)])
def test_forward_matches_fp64_reference(B, H, W):
    net, theta, feat, _ = _net_and_data(B, H, W)
    got = net.forward(feat).cpu().numpy()
    want = ref.forward(theta.astype(np.float64), feat.cpu().numpy())
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    print("forward rel L2 vs fp64: %.3e" % err)
    assert err <= 3e-2


@pytest.mark.parametrize("B,H,W", [(2, 32, 32), (1, 32, 128)])
def test_gradients_match_fp64_reference(B, H, W):
    net, theta, feat, target = _net_and_data(B, H, W)
    loss, g = net.loss_grad(feat, target)
    rloss, rg = ref.loss_grad(theta.astype(np.float64), feat.cpu().numpy(), target.cpu().numpy())
    assert abs(loss / rloss - 1) <= 3e-2
    off = 0
    worst = 0.0
    for ci, co in ref.conv_shapes():
        n = co * ci * 9 + co
        a, b = g[off:off + n], rg[off:off + n]
        e = np.linalg.norm(a - b) / np.linalg.norm(b)
        worst = max(worst, e)
        off += n
    total = np.linalg.norm(g - rg) / np.linalg.norm(rg)
    print("gradient rel L2 vs fp64: total %.3e, worst layer %.3e" % (total, worst))
    assert total <= 5e-2 and worst <= 1e-1


def test_training_on_library_windows_reduces_loss():
    X, T = S.make_windows(48, size=128, K=8, seed=11, instances=16, restart_every=3)
    net = S.Surrogate(128, 128, max_batch=8, seed=2)
    losses = S.train(net, X, T, steps=120, batch=8, lr=2e-3)
    first, last = np.mean(losses[:5]), np.mean(losses[-5:])
    print("training loss %.3e -> %.3e" % (first, last))
    assert np.isfinite(last) and last < 0.5 * first


def test_advance_rejecting_every_window_is_plain_qla():
    """With a tolerance nothing meets, every window falls back to qla_step:
    the result is the plain QLA result bit for bit."""
    size, K, windows = 64, 8, 4
    rng = np.random.default_rng(4)
    med, pk = inputs.surrogate_instance(rng, size)
    n = inputs.ellipse_medium(size, size, 1.0, **med)
    net = S.Surrogate(size, size, max_batch=1, seed=1)
    with qla.Grid(size, size, 1.0, "fp32", te_only=True) as g:
        g.set_medium(n)
        g.set_packet(**pk)
        acc, e = net.advance(g, windows, K, energy_tol=-1.0, div_tol=-1.0)
        got = g.get_state()
    with qla.Grid(size, size, 1.0, "fp32", te_only=True) as g:
        g.set_medium(n)
        g.set_packet(**pk)
        g.step(windows * K)
        want = g.get_state()
        e_ref = g.energy()
    assert acc == 0
    assert np.array_equal(got, want)
    assert e[-1] == e_ref


def test_trained_network_beats_the_zero_change_predictor_and_checks_hold():
    """What training buys: over one K-step window on held-out lattices the
    trained network's error is a small fraction of the error of leaving the
    state unchanged (the best a method without the network can do without
    running QLA).  With the energy / div B checks on, chained windows end
    within the check-controlled error of plain QLA."""
    import torch
    size, K = 128, 16
    X, T = S.make_windows(1024, size=size, K=K, seed=21, instances=64, restart_every=8)
    net = S.Surrogate(size, size, max_batch=8, seed=4)
    losses = S.train(net, X, T, steps=1500, batch=8, lr=1e-3)
    var = float(T.pow(2).mean())
    del X, T
    print("loss / target variance: %.3e" % (np.mean(losses[-50:]) / var))
    rng = np.random.default_rng(77)
    for _ in range(2):
        med, pk = inputs.surrogate_instance(rng, size)
        n = inputs.ellipse_medium(size, size, 1.0, **med)
        with qla.Grid(size, size, 1.0, "fp32", te_only=True) as g:
            g.set_medium(n)
            g.set_packet(**pk)
            f0 = S.features(g).unsqueeze(0).contiguous()
            y = net.forward(f0)[0]
            g.step(K)
            d = S.features(g)[..., :3] - f0[0, ..., :3]
            state = (f0[0, ..., :3] + d).norm()
            e_net, e_zero = float((y - d).norm() / state), float(d.norm() / state)
            g.set_packet(**pk)
            g.step(8 * K)
            ref = g.get_state()
        with qla.Grid(size, size, 1.0, "fp32", te_only=True) as g:
            g.set_medium(n)
            g.set_packet(**pk)
            acc, _ = net.advance(g, 8, K, 2e-3, 3e-2)
            got = g.get_state()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        print("one window: network %.3e, zero change %.3e; 8 checked windows: %d accepted, "
              "rel L2 %.3e" % (e_net, e_zero, acc, err))
        assert e_net < 0.25 * e_zero
        assert err <= 0.25
        torch.cuda.synchronize()


def test_conv_wait_that_runs_out_reports_timeout_and_recovers():
    """A CTA whose mbarrier wait never completes gives up (2 s bound), skips its
    output and the call returns QLA_ETIMEOUT; the next call is exact again."""
    import time

    import torch
    lib = qla.load()
    rng = np.random.default_rng(99)
    B, H, W, cin, cout = 1, 8, 16, 32, 32
    x = _bf16(rng, (B, H, W, cin))
    w = _bf16(rng, (cout, 9, cin), 0.1)
    out = torch.zeros((B, H, W, cout), dtype=torch.float32, device="cuda")

    def call():
        return lib.surr_conv3x3_raw(ctypes.c_void_p(x.data_ptr()), B, H, W, cin,
                                    ctypes.c_void_p(w.data_ptr()), cout,
                                    ctypes.c_void_p(out.data_ptr()), None)

    assert lib.surr_test_stall_conv(1) == 0
    try:
        t0 = time.perf_counter()
        st = call()
        dt = time.perf_counter() - t0
    finally:
        assert lib.surr_test_stall_conv(0) == 0
    assert st == 5, st                      # QLA_ETIMEOUT
    assert 1.0 < dt < 30.0, dt
    assert call() == 0
    torch.cuda.synchronize()
    want = _ref_conv(x, w).numpy()
    assert np.linalg.norm(out.cpu().numpy() - want) <= 1e-5 * np.linalg.norm(want)
