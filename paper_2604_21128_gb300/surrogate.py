"""Learned surrogate on top of the QLA library (surr_* in the C ABI).

A five-level convolutional operator advances an FP32 E_z lattice K steps at
once; it is trained on windows that the library's own batched QLA runs
produce, with the library's BF16 tensor-core kernels; plain QLA stays the
fallback and the arbiter (``Surrogate.advance``).  This module only marshals
arguments and orders the calls; every computation runs in libqla.
"""
from __future__ import annotations

import ctypes
import math
import time

import numpy as np

from . import inputs, qla

FEAT, NOUT = 6, 3


def _check(n, status):
    if status != 0:
        msg = qla.load().surr_last_error(n).decode() if n else ""
        raise qla.QLAError(status, msg)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class Surrogate:
    def __init__(self, height, width, max_batch=8, seed=1, device=None, stream=None):
        import torch
        lib = qla.load()
        self.h, self.w, self.max_batch = int(height), int(width), int(max_batch)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        nbytes = int(lib.surr_workspace_bytes(self.h, self.w, self.max_batch))
        if nbytes == 0:
            raise qla.QLAError(1, "height and width must be multiples of 16")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            n = ctypes.c_void_p()
            _check(None, lib.surr_create(ctypes.byref(n), self.h, self.w, self.max_batch, int(seed),
                                         ctypes.c_void_p(self.stream.cuda_stream),
                                         _ptr(self.workspace), nbytes))
            self._n = n
        self.nparams = int(lib.surr_param_count(self._n))

    def params(self):
        out = np.empty(self.nparams, dtype=np.float32)
        _check(self._n, qla.load().surr_get_params(self._n, ctypes.c_void_p(out.ctypes.data)))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.nparams
        _check(self._n, qla.load().surr_set_params(self._n, ctypes.c_void_p(p.ctypes.data)))

    def forward(self, feat):
        """feat: CUDA float32 tensor (B, h, w, 6) -> (B, h, w, 3)."""
        import torch
        feat = feat.contiguous()
        out = torch.empty(feat.shape[:3] + (NOUT,), dtype=torch.float32, device=feat.device)
        _check(self._n, qla.load().surr_forward(self._n, _ptr(feat), int(feat.shape[0]), _ptr(out)))
        return out

    def loss_grad(self, feat, target):
        loss = ctypes.c_double()
        g = np.empty(self.nparams, dtype=np.float32)
        _check(self._n, qla.load().surr_loss_grad(self._n, _ptr(feat.contiguous()),
                                                  _ptr(target.contiguous()), int(feat.shape[0]),
                                                  ctypes.byref(loss), ctypes.c_void_p(g.ctypes.data)))
        return loss.value, g

    def train_step(self, feat, target, lr):
        loss = ctypes.c_double()
        _check(self._n, qla.load().surr_train_step(self._n, _ptr(feat), _ptr(target),
                                                   int(feat.shape[0]), float(lr), ctypes.byref(loss)))
        return loss.value

    def advance(self, grid, windows, K=32, energy_tol=1e-3, div_tol=1e-2):
        """Chained windows with fallback; returns (accepted, energies)."""
        import torch
        scratch = torch.empty(12 * grid.nx * grid.ny, dtype=torch.float32, device=self.device)
        acc = ctypes.c_int()
        e = np.empty(int(windows))
        with torch.cuda.device(self.device):
            _check(self._n, qla.load().surr_advance(grid._ctx, self._n, int(windows), int(K),
                                                    float(energy_tol), float(div_tol), _ptr(scratch),
                                                    ctypes.byref(acc),
                                                    ctypes.c_void_p(e.ctypes.data)))
        return acc.value, e

    def close(self):
        if getattr(self, "_n", None):
            qla.load().surr_destroy(self._n)
            self._n = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def features(grid, out=None):
    """Features of a Grid's current state (CUDA tensor (ny, nx, 6))."""
    import torch
    if out is None:
        out = torch.empty((grid.ny, grid.nx, FEAT), dtype=torch.float32, device=grid.device)
    qla._check(grid._ctx, qla.load().surr_features(grid._ctx, _ptr(out)))
    return out


def make_windows(count, size=256, K=32, seed=5, instances=32, restart_every=16, stream=None):
    """Training windows from the library's own batched QLA runs: features of
    a state and, as target, the change of (q2, q3, q4) over the next K steps.
    Lattices of the scaled vacuum-bubble geometry with seeded random media
    and packets; every ``restart_every`` windows the packets restart."""
    import torch
    rng = np.random.default_rng(seed)
    X = torch.empty((count, size, size, FEAT), dtype=torch.float32, device="cuda")
    T = torch.empty((count, size, size, NOUT), dtype=torch.float32, device="cuda")
    m = min(instances, count)
    with qla.Batch([(size, size)] * m, 1.0, "fp32", te_only=True, stream=stream) as b:
        grids = [b.instance(k) for k in range(m)]
        cur = torch.empty((m, size, size, FEAT), dtype=torch.float32, device="cuda")
        filled, since = 0, restart_every
        while filled < count:
            if since >= restart_every:
                for g in grids:
                    med, pk = inputs.surrogate_instance(rng, size)
                    g.set_medium(inputs.ellipse_medium(size, size, 1.0, **med))
                    g.set_packet(**pk)
                since = 0
            for k, g in enumerate(grids):
                features(g, cur[k])
            b.step(K)
            take = min(m, count - filled)
            nxt = torch.empty_like(cur)
            for k in range(take):
                features(grids[k], nxt[k])
            X[filled:filled + take] = cur[:take]
            T[filled:filled + take] = nxt[:take, ..., :NOUT] - cur[:take, ..., :NOUT]
            filled += take
            since += 1
    torch.cuda.synchronize()
    return X, T


def train(net, X, T, steps, batch=8, lr=1e-3, lr_min=1e-5, warmup=300, seed=0, log_every=0):
    """Adam over ``steps`` minibatches drawn (seeded) from the windows X, T:
    the rate rises linearly over the first ``warmup`` steps (without it this
    normalisation-free U-Net diverges at rates above ~1e-3), then follows a
    cosine schedule from ``lr`` to ``lr_min``.  Returns the losses."""
    rng = np.random.default_rng(seed)
    n = X.shape[0]
    losses = []
    for s in range(int(steps)):
        i = int(rng.integers(0, n - batch + 1))
        rate = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * s / max(1, steps)))
        rate *= min(1.0, (s + 1) / max(1, warmup))
        losses.append(net.train_step(X[i:i + batch], T[i:i + batch], rate))
        if log_every and s % log_every == 0:
            print("step %d loss %.4e lr %.2e" % (s, losses[-1], rate), flush=True)
    return losses
