"""FP64 CPU reference of the learned surrogate network.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): used by the tests to check
the CUDA surrogate's forward pass and parameter gradients.  Plain PyTorch CPU
ops in float64; gradients by autograd.  The surrogate is not part of the
paper's method; its definition is the library's (include/qla.h, surr_*):

  five levels, widths 32, 64, 128, 256, 256; every convolution 3x3 with
  periodic (circular) padding, out[y, x] = sum W[co, ci, ky, kx]
  in[y + ky - 1, x + kx - 1] + b[co]; leaky ReLU slope 0.1;
  E0 = a(conv(X)), E_l = a(conv(avgpool2(E_{l-1}))), l = 1..4;
  D3 = a(conv(up2(E4)) + E3), D_l = a(conv(up2(D_{l+1})) + E_l), l = 2..0;
  Y = conv(D0) (3 outputs).  Loss = mean of (Y - target)^2.

Parameter vector layout (surr_get_params): per convolution, in the order
E0..E4, D3..D0, output, the weights (cout, cin, 3, 3) then the bias (cout).

Parity status: pinned by tests/test_oracle_surrogate.py (finite-difference
gradients, the orientation of the 3x3 taps and the circular padding on a
shift kernel, pooling/upsampling adjointness, periodic shift equivariance).
"""
import numpy as np
import torch
import torch.nn.functional as F

WIDTH = (32, 64, 128, 256, 256)
FEAT, NOUT, LEAK = 6, 3, 0.1


def conv_shapes():
    """(cin, cout) of the ten convolutions in parameter order."""
    s = [(FEAT, WIDTH[0])]
    s += [(WIDTH[l - 1], WIDTH[l]) for l in range(1, 5)]
    s += [(WIDTH[l + 1], WIDTH[l]) for l in (3, 2, 1, 0)]
    s += [(WIDTH[0], NOUT)]
    return s


def param_count():
    return sum(co * ci * 9 + co for ci, co in conv_shapes())


def unpack(flat):
    """Flat parameter vector -> list of (W, b) float64 tensors."""
    if not isinstance(flat, torch.Tensor):
        flat = torch.as_tensor(np.asarray(flat), dtype=torch.float64)
    out, off = [], 0
    for ci, co in conv_shapes():
        w = flat[off:off + co * ci * 9].reshape(co, ci, 3, 3)
        off += co * ci * 9
        b = flat[off:off + co]
        off += co
        out.append((w, b))
    assert off == flat.numel()
    return out


def conv(x, w, b=None):
    """3x3 convolution with periodic padding (cross-correlation)."""
    return F.conv2d(F.pad(x, (1, 1, 1, 1), mode="circular"), w, b)


def act(x):
    return F.leaky_relu(x, LEAK)


def forward_t(p, feat):
    """p: list of (W, b) tensors; feat: tensor (B, H, W, 6). Returns (B, H, W, 3)."""
    x = feat.permute(0, 3, 1, 2)
    E = []
    h = x
    for l in range(5):
        if l:
            h = F.avg_pool2d(E[-1], 2)
        h = act(conv(h, *p[l]))
        E.append(h)
    d = E[4]
    for i, l in enumerate((3, 2, 1, 0)):
        d = act(conv(F.interpolate(d, scale_factor=2, mode="nearest"), *p[5 + i]) + E[l])
    y = conv(d, *p[9])
    return y.permute(0, 2, 3, 1)


def forward(flat, feat):
    """numpy in, numpy out (float64)."""
    with torch.no_grad():
        f = torch.as_tensor(np.asarray(feat), dtype=torch.float64)
        return forward_t(unpack(flat), f).numpy()


def loss_grad(flat, feat, target):
    """Mean-square loss and its gradient with respect to the flat parameters."""
    theta = torch.tensor(np.asarray(flat), dtype=torch.float64, requires_grad=True)
    f = torch.as_tensor(np.asarray(feat), dtype=torch.float64)
    t = torch.as_tensor(np.asarray(target), dtype=torch.float64)
    y = forward_t(unpack(theta), f)
    loss = ((y - t) ** 2).mean()
    loss.backward()
    return float(loss.detach()), theta.grad.numpy().copy()
