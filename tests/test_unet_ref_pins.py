"""Pins of the FP64 reference network (oracle/unet_ref.py) against
definitions that do not go through it: explicit loops for the convolution,
hand-computed pooling/upsampling, the adjoint pairing of pooling and
upsampling, central finite differences for the autograd gradients, and the
constant-gradient closed form of Adam."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import unet_ref as R  # noqa: E402


def test_conv_against_loops():
    g = torch.Generator().manual_seed(0)
    x = torch.randn((2, 3, 5, 7), generator=g, dtype=torch.float64)
    for ks in (3, 1):
        w = torch.randn((4, 3, ks, ks), generator=g, dtype=torch.float64)
        b = torch.tensor([0.1, -0.2, 0.3, 0.0], dtype=torch.float64)
        ref = R.conv_loops(x.numpy(), w.numpy(), b.numpy())
        assert np.abs(R.conv(x, w, b).numpy() - ref).max() <= 1e-13
    # a one-hot kernel shifts the image (cross-correlation orientation, zero padding)
    w = torch.zeros((1, 1, 3, 3), dtype=torch.float64)
    w[0, 0, 0, 2] = 1.0  # reads x[y - 1, x + 1]
    img = torch.arange(20, dtype=torch.float64).reshape(1, 1, 4, 5)
    y = R.conv(img, w)
    assert y[0, 0, 1, 0] == img[0, 0, 0, 1] and y[0, 0, 0, 0] == 0 and y[0, 0, 1, 4] == 0


def test_pool_up_definitions_and_adjoint():
    x = torch.arange(16, dtype=torch.float64).reshape(1, 1, 4, 4)
    assert torch.equal(R.pool2(x)[0, 0], torch.tensor([[2.5, 4.5], [10.5, 12.5]], dtype=torch.float64))
    u = R.up2(torch.tensor([[[[1.0, 2.0], [3.0, 4.0]]]], dtype=torch.float64))
    assert torch.equal(u[0, 0], torch.tensor([[1, 1, 2, 2], [1, 1, 2, 2], [3, 3, 4, 4], [3, 3, 4, 4]],
                                             dtype=torch.float64))
    g = torch.Generator().manual_seed(1)
    a = torch.randn((2, 3, 5, 6), generator=g, dtype=torch.float64)
    bb = torch.randn((2, 3, 10, 12), generator=g, dtype=torch.float64)
    # <up2 a, b> = <a, 4 pool2 b>: nearest upsampling is 4x the adjoint of 2x2 averaging
    assert abs(float((R.up2(a) * bb).sum() - (a * 4 * R.pool2(bb)).sum())) <= 1e-12 * float(bb.abs().sum())


def test_network_gradient_fd():
    chans = (3, 4)
    g = torch.Generator().manual_seed(2)
    params = [(0.5 * torch.randn(s[:2] + (s[2], s[2]), generator=g, dtype=torch.float64),
               0.1 * torch.randn(s[0], generator=g, dtype=torch.float64)) for s in R.layer_shapes(2, 2, chans)]
    x = torch.randn((2, 2, 8, 8), generator=g, dtype=torch.float64)
    t = torch.randn((2, 2, 8, 8), generator=g, dtype=torch.float64)
    L0, grads, _ = R.loss_and_grads(params, x, t, chans)

    def loss(ps):
        return float(R.mse(R.forward(ps, x, chans), t))

    rng = np.random.default_rng(3)
    h = 1e-6
    for li in range(len(params)):
        w, b = params[li]
        for _ in range(3):
            idx = tuple(int(rng.integers(0, s)) for s in w.shape)
            wp, wm = w.clone(), w.clone()
            wp[idx] += h
            wm[idx] -= h
            pp = list(params)
            pp[li] = (wp, b)
            pm = list(params)
            pm[li] = (wm, b)
            fd = (loss(pp) - loss(pm)) / (2 * h)
            assert abs(fd - float(grads[li][0][idx])) <= 1e-6 * max(1e-3, abs(fd)) + 1e-9, (li, idx)
    assert L0 > 0


def test_adam_constant_gradient_closed_form():
    """With a constant gradient g the bias-corrected moments are g and g^2, so
    every step moves p by lr |g| / (|g| + eps) against the sign of g."""
    p, m, v = np.array([1.0, -2.0]), np.zeros(2), np.zeros(2)
    g = np.array([0.3, -4.0])
    for t in range(1, 8):
        p, m, v = R.adam(p, m, v, g, t, lr=0.01)
    step = 0.01 * np.abs(g) / (np.abs(g) + 1e-8)
    assert np.allclose(p, np.array([1.0, -2.0]) - 7 * np.sign(g) * step, rtol=0, atol=1e-12)
