"""Warm-start surrogate: a 4-level convolutional U-Net (32-256 channels, BF16
weights and activations, FP32 accumulation) whose prediction becomes the
proposed initial control of a problem (warmstart.py).  The paper's gradient
algorithm (Sec. 3.2.1) then refines the proposal; started from g = 0 it is
the fallback and the reference the surrogate's error is measured against.

Every layer runs in the library's hand-written kernels (cx_nn_* in
include/cxlbm.h): direct convolutions on the tensor cores (tcgen05 for 32-128
output channels, mma.sync otherwise) for the forward, data-gradient and
weight-gradient passes, and elementwise kernels for
ReLU, pooling, upsampling, skips, the loss and Adam.  PyTorch only holds the
memory and the stream.

Architecture (additive skips):
    encoder level l: [pool2 if l > 0] -> conv3x3+ReLU -> conv3x3+ReLU (skip s_l)
    decoder level l: up2 -> conv3x3+ReLU -> + s_l -> conv3x3+ReLU
    head: conv1x1 (no activation)
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Conv:
    def __init__(self, cin, cout, ks, rng, device):
        fan_in = cin * ks * ks
        w = rng.standard_normal((cout, cin, ks, ks)) * np.sqrt(2.0 / fan_in)
        self.cin, self.cout, self.ks = cin, cout, ks
        self.w = torch.as_tensor(w, dtype=torch.float32, device=device).contiguous()
        self.b = torch.zeros(cout, dtype=torch.float32, device=device)
        self.wb = torch.empty(self.w.shape, dtype=torch.bfloat16, device=device)
        self.bb = torch.empty(cout, dtype=torch.bfloat16, device=device)  # BF16 copy Adam writes (bias stays FP32)
        self.gw = torch.zeros_like(self.w)
        self.gb = torch.zeros_like(self.b)
        self.mw, self.vw = torch.zeros_like(self.w), torch.zeros_like(self.w)
        self.mb, self.vb = torch.zeros_like(self.b), torch.zeros_like(self.b)


class UNet:
    def __init__(self, cin=5, cout=4, chans=(32, 64, 128, 256), seed=0, device="cuda"):
        self.lib = _lib.load()
        self.device = torch.device(device)
        self.stream = torch.cuda.current_stream(self.device)
        rng = np.random.default_rng(seed)
        self.chans = tuple(chans)
        self.L = len(chans)
        self.enc = []
        c_prev = cin
        for c in chans:
            self.enc.append((Conv(c_prev, c, 3, rng, device), Conv(c, c, 3, rng, device)))
            c_prev = c
        self.dec = {}
        for l in range(self.L - 2, -1, -1):
            self.dec[l] = (Conv(chans[l + 1], chans[l], 3, rng, device), Conv(chans[l], chans[l], 3, rng, device))
        self.head = Conv(chans[0], cout, 1, rng, device)
        self.layers = [c for pair in self.enc for c in pair] + [c for l in sorted(self.dec) for c in self.dec[l]] + [
            self.head]
        for c in self.layers:  # packed BF16 copies the convolution kernels read
            c.wf = torch.empty(self.lib.cx_nn_packed_weights(c.cout, c.cin, c.ks, 0), dtype=torch.bfloat16,
                               device=self.device)
            c.wbk = torch.empty(self.lib.cx_nn_packed_weights(c.cout, c.cin, c.ks, 1), dtype=torch.bfloat16,
                                device=self.device)
        self.cin, self.cout = cin, cout
        self.t = 0
        self.sync_bf16()

    # -------------------------------------------------------------- plumbing
    def _s(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def sync_bf16(self):
        for c in self.layers:
            _lib.check(self.lib.cx_nn_cast_bf16(_p(c.w), _p(c.wb), c.w.numel(), self._s()), "cx_nn_cast_bf16")
            self._pack(c)

    def _pack(self, c):
        _lib.check(self.lib.cx_nn_pack_weights(_p(c.wb), c.cout, c.cin, c.ks, _p(c.wf), _p(c.wbk), self._s()),
                   "cx_nn_pack_weights")

    def _new(self, B, C, H, W):
        return torch.empty((B, C, H, W), dtype=torch.bfloat16, device=self.device)

    def _conv(self, c: Conv, x, relu, out_f32=False):
        B, _, H, W = x.shape
        if out_f32:
            y = torch.empty((B, c.cout, H, W), dtype=torch.float32, device=self.device)
            _lib.check(self.lib.cx_nn_conv_forward_f32(_p(x), _p(c.wf), _p(c.b), _p(y), B, c.cin, c.cout, H, W, c.ks,
                                                       self._s()), "cx_nn_conv_forward_f32")
            return y
        y = self._new(B, c.cout, H, W)
        _lib.check(self.lib.cx_nn_conv_forward(_p(x), _p(c.wf), _p(c.b), _p(y), B, c.cin, c.cout, H, W, c.ks,
                                               1 if relu else 0, self._s()), "cx_nn_conv_forward")
        return y

    @staticmethod
    def wgrad_on_tcgen05(cin, H, W, ks):
        """Whether the 3x3 weight gradient runs on the tcgen05 kernel: measured
        faster from 64x64 pixels up (up to 2x), and at 32x32 with 128 or more
        input channels; the mma.sync kernel wins on the small deep levels
        (fewer pixel tiles than the tensor-core pipeline needs to fill)."""
        return ks == 3 and H % 8 == 0 and W % 8 == 0 and (H * W >= 4096 or (H * W >= 1024 and cin >= 128))

    def _conv_back(self, c: Conv, x, dy, need_dx=True):
        B, _, H, W = x.shape
        # split the pixel tiles so that about 2 blocks per SM run (fewer partials to reduce)
        ntiles = B * ((H + 7) // 8) * ((W + 7) // 8)
        tc = self.wgrad_on_tcgen05(c.cin, H, W, c.ks)
        base = ((c.cin + 15) // 16) * ((c.cout + 127) // 128 if tc else (c.cout + 63) // 64)
        splits = int(max(1, min(ntiles, -(-304 // base))))
        nbytes = self.lib.cx_nn_conv_backward_weight_scratch(B, c.cin, c.cout, H, W, c.ks, splits)
        scratch = torch.empty(max(1, nbytes // 4), dtype=torch.float32, device=self.device)
        if tc:
            _lib.check(self.lib.cx_nn_conv_backward_weight_tc(_p(x), _p(dy), _p(c.gw), _p(c.gb), _p(scratch), splits,
                                                              B, c.cin, c.cout, H, W, c.ks, None, self._s()),
                       "cx_nn_conv_backward_weight_tc")
        else:
            _lib.check(self.lib.cx_nn_conv_backward_weight(_p(x), _p(dy), _p(c.gw), _p(c.gb), _p(scratch), splits, B,
                                                           c.cin, c.cout, H, W, c.ks, self._s()),
                       "cx_nn_conv_backward_weight")
        if not need_dx:
            return None
        dx = self._new(B, c.cin, H, W)
        _lib.check(self.lib.cx_nn_conv_backward_data(_p(dy), _p(c.wbk), _p(dx), B, c.cin, c.cout, H, W, c.ks,
                                                     self._s()), "cx_nn_conv_backward_data")
        return dx

    def _relu_back(self, y, dy):
        dz = torch.empty_like(dy)
        _lib.check(self.lib.cx_nn_relu_backward(_p(y), _p(dy), _p(dz), y.numel(), self._s()), "cx_nn_relu_backward")
        return dz

    def _add(self, a, b):
        o = torch.empty_like(a)
        _lib.check(self.lib.cx_nn_add(_p(a), _p(b), _p(o), a.numel(), self._s()), "cx_nn_add")
        return o

    def _pool(self, x, backward=False):
        B, C, H, W = x.shape
        if not backward:
            y = self._new(B, C, H // 2, W // 2)
            _lib.check(self.lib.cx_nn_pool2(_p(x), _p(y), B * C, H, W, 0, self._s()), "cx_nn_pool2")
        else:  # x = dY at half resolution
            y = self._new(B, C, 2 * H, 2 * W)
            _lib.check(self.lib.cx_nn_pool2(_p(x), _p(y), B * C, 2 * H, 2 * W, 1, self._s()), "cx_nn_pool2")
        return y

    def _up(self, x, backward=False):
        B, C, H, W = x.shape
        if not backward:
            y = self._new(B, C, 2 * H, 2 * W)
            _lib.check(self.lib.cx_nn_up2(_p(x), _p(y), B * C, H, W, 0, self._s()), "cx_nn_up2")
        else:  # x = dY at double resolution
            y = self._new(B, C, H // 2, W // 2)
            _lib.check(self.lib.cx_nn_up2(_p(x), _p(y), B * C, H // 2, W // 2, 1, self._s()), "cx_nn_up2")
        return y

    # -------------------------------------------------------------- network
    def forward(self, x, out_f32=False):
        """x: BF16 [B, cin, H, W] (H, W divisible by 2^(levels-1)); returns
        [B, cout, H, W] in BF16 (training) or FP32 (out_f32: inference)."""
        x = x.to(torch.bfloat16).contiguous()
        cache = {"enc": [], "dec": {}}
        h = x
        for l, (c1, c2) in enumerate(self.enc):
            if l > 0:
                h = self._pool(h)
            a1 = self._conv(c1, h, True)
            a2 = self._conv(c2, a1, True)
            cache["enc"].append((h, a1, a2))
            h = a2
        for l in range(self.L - 2, -1, -1):
            c1, c2 = self.dec[l]
            u = self._up(h)
            d1 = self._conv(c1, u, True)
            s = self._add(d1, cache["enc"][l][2])
            d2 = self._conv(c2, s, True)
            cache["dec"][l] = (u, d1, s, d2)
            h = d2
        out = self._conv(self.head, h, False, out_f32=out_f32)
        cache["head_in"] = h
        self.cache = cache
        return out

    def backward(self, dout):
        """Gradients of sum(dout * out) into every layer's gw, gb (FP32)."""
        cache = self.cache
        dh = self._conv_back(self.head, cache["head_in"], dout.contiguous())
        dskip = {}
        for l in range(0, self.L - 1):
            c1, c2 = self.dec[l]
            u, d1, s, d2 = cache["dec"][l]
            dz = self._relu_back(d2, dh)
            ds = self._conv_back(c2, s, dz)
            dskip[l] = ds
            dz1 = self._relu_back(d1, ds)
            du = self._conv_back(c1, u, dz1)
            dh = self._up(du, backward=True)
        for l in range(self.L - 1, -1, -1):
            c1, c2 = self.enc[l]
            h_in, a1, a2 = cache["enc"][l]
            g2 = dh if l == self.L - 1 else self._add(dh, dskip[l])
            dz = self._relu_back(a2, g2)
            da1 = self._conv_back(c2, a1, dz)
            dz1 = self._relu_back(a1, da1)
            dh_in = self._conv_back(c1, h_in, dz1, need_dx=l > 0)
            if l > 0:
                dh = self._pool(dh_in, backward=True)

    def loss(self, out, target, want_grad=True):
        """Mean squared error (FP32 target) and its BF16 gradient."""
        loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        dout = torch.empty_like(out) if want_grad else None
        target = target.to(torch.float32).contiguous()  # held for the call
        _lib.check(self.lib.cx_nn_mse(_p(out), _p(target), _p(dout), _p(loss), out.numel(), self._s()), "cx_nn_mse")
        return loss, dout

    def adam_step(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.t += 1
        for c in self.layers:
            _lib.check(self.lib.cx_nn_adam(_p(c.w), _p(c.mw), _p(c.vw), _p(c.gw), _p(c.wb), c.w.numel(), lr, b1, b2,
                                           eps, self.t, self._s()), "cx_nn_adam")
            _lib.check(self.lib.cx_nn_adam(_p(c.b), _p(c.mb), _p(c.vb), _p(c.gb), _p(c.bb), c.b.numel(), lr, b1, b2,
                                           eps, self.t, self._s()), "cx_nn_adam")
            self._pack(c)

    def train_step(self, x, target, lr=1e-3):
        out = self.forward(x)
        loss, dout = self.loss(out, target)
        self.backward(dout)
        self.adam_step(lr)
        return loss

    def smooth(self, y, sigma):
        """Periodic Gaussian low-pass (standard deviation sigma cells) of every
        [H][W] plane of the FP32 tensor y."""
        if sigma <= 0:
            return y
        r = int(np.ceil(3 * sigma))
        d = np.arange(-r, r + 1)
        taps = np.exp(-0.5 * (d / sigma) ** 2)
        taps = torch.as_tensor(taps / taps.sum(), dtype=torch.float32, device=self.device)
        B, C, H, W = y.shape
        tmp = torch.empty_like(y)
        out = torch.empty_like(y)
        _lib.check(self.lib.cx_nn_smooth(_p(y), _p(tmp), _p(out), B * C, H, W, _p(taps), r, self._s()),
                   "cx_nn_smooth")
        return out

    def flops(self, B, H, W, training=True):
        """Convolution FLOPs (2 per multiply-add) of one forward, or of one
        training step (forward, data gradients except the input layer's, and
        weight gradients), for a batch of B H x W inputs."""
        total = 0
        h, w = H, W
        sizes = []
        for l in range(self.L):
            if l > 0:
                h, w = h // 2, w // 2
            sizes.append((h, w))
        for l, (c1, c2) in enumerate(self.enc):
            hh, ww = sizes[l]
            for c, first in ((c1, l == 0), (c2, False)):
                f = 2 * B * hh * ww * c.cout * c.cin * c.ks * c.ks
                total += f * (1 + (0 if first else 1) + 1) if training else f
        for l, (c1, c2) in self.dec.items():
            hh, ww = sizes[l]
            for c in (c1, c2):
                f = 2 * B * hh * ww * c.cout * c.cin * c.ks * c.ks
                total += 3 * f if training else f
        f = 2 * B * H * W * self.head.cout * self.head.cin
        total += 3 * f if training else f
        return total

    def state(self):
        return {"w": [c.w.cpu() for c in self.layers], "b": [c.b.cpu() for c in self.layers]}
