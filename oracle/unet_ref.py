"""FP64 CPU reference of the warm-start surrogate network (test
infrastructure: only tests/, the smoke check and the bench's CPU baseline use
it; the product path never does).

The surrogate is not part of the paper: it is a convolutional U-Net that
proposes the initial control which the paper's gradient algorithm (Sec.
3.2.1) then refines.  This module writes the network out from its
definition, in plain PyTorch CPU operations in float64, so that the library's
BF16 tensor-core kernels can be checked against it:

  conv(x; w, b)    y[b,o,p] = b[o] + sum_{c,t} w[o,c,t] x[b,c,p+t]
                   (3x3 with zero padding 1, or 1x1; cross-correlation)
  pool2            2x2 average, stride 2
  up2              nearest-neighbour 2x upsampling
  encoder level l  [pool2 if l > 0] -> conv+ReLU -> conv+ReLU  (skip s_l)
  decoder level l  up2 -> conv+ReLU -> (+ s_l) -> conv+ReLU
  head             1x1 conv, no activation
  loss             mean of (out - target)^2
  Adam             m <- b1 m + (1-b1) g; v <- b2 v + (1-b2) g^2;
                   p <- p - lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)

Gradients come from torch.autograd on these float64 operations; the tests
pin them against central finite differences and the forward operations
against explicit loops.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

DT = torch.float64


def conv(x, w, b=None, relu=False):
    ks = w.shape[-1]
    y = F.conv2d(x, w, b, padding=ks // 2)
    return torch.relu(y) if relu else y


def conv_loops(x, w, b=None):
    """The convolution written out element by element (small inputs only)."""
    x, w = np.asarray(x, dtype=np.float64), np.asarray(w, dtype=np.float64)
    B, C, H, W = x.shape
    O, _, k, _ = w.shape
    pad = k // 2
    y = np.zeros((B, O, H, W))
    for bb in range(B):
        for o in range(O):
            for yy in range(H):
                for xx in range(W):
                    s = 0.0 if b is None else float(b[o])
                    for c in range(C):
                        for dy in range(k):
                            for dx in range(k):
                                sy, sx = yy + dy - pad, xx + dx - pad
                                if 0 <= sy < H and 0 <= sx < W:
                                    s += w[o, c, dy, dx] * x[bb, c, sy, sx]
                    y[bb, o, yy, xx] = s
    return y


def pool2(x):
    return F.avg_pool2d(x, 2)


def up2(x):
    return x.repeat_interleave(2, dim=-2).repeat_interleave(2, dim=-1)


def layer_shapes(cin, cout, chans):
    """(cout, cin, ks) of every convolution, in the order encoder (two per
    level), decoder (levels 0..L-2, two each), head."""
    out = []
    c_prev = cin
    for c in chans:
        out += [(c, c_prev, 3), (c, c, 3)]
        c_prev = c
    for l in range(len(chans) - 1):
        out += [(chans[l], chans[l + 1], 3), (chans[l], chans[l], 3)]
    out.append((cout, chans[0], 1))
    return out


def forward(params, x, chans):
    """params: list of (w, b) in layer_shapes order (float64 tensors)."""
    L = len(chans)
    enc = params[: 2 * L]
    dec = {l: params[2 * L + 2 * l: 2 * L + 2 * l + 2] for l in range(L - 1)}
    head = params[-1]
    skips = []
    h = x
    for l in range(L):
        if l > 0:
            h = pool2(h)
        h = conv(h, *enc[2 * l], relu=True)
        h = conv(h, *enc[2 * l + 1], relu=True)
        skips.append(h)
    for l in range(L - 2, -1, -1):
        (w1, b1), (w2, b2) = dec[l]
        h = conv(up2(h), w1, b1, relu=True) + skips[l]
        h = conv(h, w2, b2, relu=True)
    return conv(h, *head)


def mse(out, target):
    return torch.mean((out - target) ** 2)


def loss_and_grads(params, x, target, chans):
    """(loss, [(dw, db)]) in float64."""
    ps = [(w.detach().clone().to(DT).requires_grad_(True), b.detach().clone().to(DT).requires_grad_(True))
          for w, b in params]
    out = forward(ps, x.to(DT), chans)
    loss = mse(out, target.to(DT))
    loss.backward()
    return float(loss), [(w.grad, b.grad) for w, b in ps], out.detach()


def adam(p, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    p = p - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    return p, m, v
