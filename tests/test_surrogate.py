"""Warm-start surrogate kernels (BF16 tensor-core convolutions with FP32
accumulation, pooling, upsampling, ReLU, loss, Adam) against the FP64 CPU
reference network, and the whole U-Net's forward and parameter gradients.

Tolerances: a kernel that reads BF16 inputs and accumulates in FP32 differs
from the FP64 result on the same BF16 inputs by the FP32 accumulation error
(~1e-6 relative) plus the final rounding of a BF16 output (2^-8 relative at
most), so BF16 outputs are checked to 2^-8 relative per element (plus a tiny
absolute floor for cancellation) and FP32 outputs to 1e-4 relative L2.  The
whole network rounds every activation to BF16, so its output and gradients
are checked in relative L2 (3e-2 / 6e-2) and by direction (cosine > 0.998).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import unet_ref as R  # noqa: E402

BF = torch.bfloat16


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_03876_gb300.build import build

    build()


def _lib():
    from paper_1908_03876_gb300 import _lib

    return _lib.load(), _lib.check


def packed(lib, check, wd, Cout, Cin, ks):
    """Forward and data-gradient packs of device BF16 weights wd."""
    wf = torch.empty(lib.cx_nn_packed_weights(Cout, Cin, ks, 0), dtype=BF, device="cuda")
    wb = torch.empty(lib.cx_nn_packed_weights(Cout, Cin, ks, 1), dtype=BF, device="cuda")
    check(lib.cx_nn_pack_weights(_p(wd), Cout, Cin, ks, _p(wf), _p(wb), _s()), "pack")
    return wf, wb


def _p(t):
    import ctypes

    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _s():
    import ctypes

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def bf16_data(shape, seed, scale=1.0):
    g = torch.Generator().manual_seed(seed)
    return (scale * torch.randn(shape, generator=g, dtype=torch.float64)).to(BF)


def check_bf16(out, ref, label):
    o = out.double().cpu()
    r = torch.as_tensor(ref, dtype=torch.float64)
    err = (o - r).abs()
    bound = 2.0 ** -8 * r.abs() + 1e-3 * r.abs().max()
    bad = int((err > bound).sum())
    print(f"[{label}] max rel {float((err / r.abs().clamp_min(1e-30)).max()):.2e} violations {bad}")
    assert bad == 0


def rel_l2(a, b):
    a = torch.as_tensor(a, dtype=torch.float64).cpu()
    b = torch.as_tensor(b, dtype=torch.float64).cpu()
    return float((a - b).norm() / b.norm())


@pytest.mark.parametrize("B,Cin,Cout,H,W,ks,relu", [
    (3, 5, 32, 20, 22, 3, True),      # ragged pixel tiles, K = 45 (not a multiple of 32)
    (2, 64, 96, 16, 16, 3, False),    # several K tiles and M tiles, ragged M
    (2, 32, 8, 18, 14, 1, False),     # 1x1 head shape
    (1, 256, 128, 8, 8, 3, True),     # deep level
    (4, 64, 32, 4, 4, 3, True),       # image smaller than the 8x8 pixel tile
    (2, 6, 1, 12, 20, 1, False),      # one output channel (the head), Cin below one chunk
    (1, 40, 70, 13, 11, 3, True),     # ragged everything
])
def test_conv_forward(B, Cin, Cout, H, W, ks, relu):
    lib, check = _lib()
    x = bf16_data((B, Cin, H, W), 1)
    w = bf16_data((Cout, Cin, ks, ks), 2, scale=1.0 / np.sqrt(Cin * ks * ks))
    b = torch.linspace(-0.5, 0.5, Cout, dtype=torch.float32)
    y = torch.empty((B, Cout, H, W), dtype=BF, device="cuda")
    xd, wd, bd = x.cuda(), w.cuda(), b.cuda()  # held: the call only sees raw pointers
    wf, _ = packed(lib, check, wd, Cout, Cin, ks)
    check(lib.cx_nn_conv_forward(_p(xd), _p(wf), _p(bd), _p(y), B, Cin, Cout, H, W, ks, int(relu), _s()), "conv")
    ref = R.conv(x.double(), w.double(), b.double(), relu=relu)
    check_bf16(y, ref, f"conv fwd {Cin}->{Cout} k{ks}")


@pytest.mark.parametrize("ks", [3, 1])
def test_conv_backward(ks):
    lib, check = _lib()
    B, Cin, Cout, H, W = 3, 40, 72, 18, 20
    x = bf16_data((B, Cin, H, W), 5)
    w = bf16_data((Cout, Cin, ks, ks), 6, scale=0.1)
    dy = bf16_data((B, Cout, H, W), 7)
    xd, wd, dyd = x.cuda(), w.cuda(), dy.cuda()
    dx = torch.empty_like(xd)
    _, wbk = packed(lib, check, wd, Cout, Cin, ks)
    check(lib.cx_nn_conv_backward_data(_p(dyd), _p(wbk), _p(dx), B, Cin, Cout, H, W, ks, _s()), "bwd data")
    for splits in (1, 7, 200):
        nbytes = lib.cx_nn_conv_backward_weight_scratch(B, Cin, Cout, H, W, ks, splits)
        scratch = torch.empty(nbytes // 4, dtype=torch.float32, device="cuda")
        dw = torch.empty((Cout, Cin, ks, ks), dtype=torch.float32, device="cuda")
        db = torch.empty(Cout, dtype=torch.float32, device="cuda")
        check(lib.cx_nn_conv_backward_weight(_p(xd), _p(dyd), _p(dw), _p(db), _p(scratch), splits, B, Cin, Cout, H, W,
                                             ks, _s()), "bwd weight")
        xr = x.double().requires_grad_(True)
        wr = w.double().requires_grad_(True)
        br = torch.zeros(Cout, dtype=torch.float64, requires_grad=True)
        (R.conv(xr, wr, br) * dy.double()).sum().backward()
        e_w, e_b = rel_l2(dw, wr.grad), rel_l2(db, br.grad)
        print(f"[conv bwd k{ks} splits {splits}] dW {e_w:.2e} db {e_b:.2e}")
        assert e_w < 1e-4 and e_b < 1e-4
    check_bf16(dx, xr.grad, f"conv bwd data k{ks}")


def test_pool_up_relu_add():
    lib, check = _lib()
    x = bf16_data((2, 3, 8, 10), 8)
    xd = x.cuda()
    y = torch.empty((2, 3, 4, 5), dtype=BF, device="cuda")
    check(lib.cx_nn_pool2(_p(xd), _p(y), 6, 8, 10, 0, _s()), "pool")
    check_bf16(y, R.pool2(x.double()), "pool2")
    dy = bf16_data((2, 3, 4, 5), 9)
    dx = torch.empty_like(xd)
    dyd = dy.cuda()
    check(lib.cx_nn_pool2(_p(dyd), _p(dx), 6, 8, 10, 1, _s()), "pool bwd")
    xr = x.double().requires_grad_(True)
    (R.pool2(xr) * dy.double()).sum().backward()
    check_bf16(dx, xr.grad, "pool2 bwd")
    up = torch.empty((2, 3, 16, 20), dtype=BF, device="cuda")
    check(lib.cx_nn_up2(_p(xd), _p(up), 6, 8, 10, 0, _s()), "up")
    assert torch.equal(up.cpu(), R.up2(x.double()).to(BF))
    dup = bf16_data((2, 3, 16, 20), 10)
    dxu = torch.empty_like(xd)
    dupd = dup.cuda()
    check(lib.cx_nn_up2(_p(dupd), _p(dxu), 6, 8, 10, 1, _s()), "up bwd")
    xr = x.double().requires_grad_(True)
    (R.up2(xr) * dup.double()).sum().backward()
    check_bf16(dxu, xr.grad, "up2 bwd")
    yr = torch.relu(x.double()).to(BF).cuda()
    dz = torch.empty_like(xd)
    g = bf16_data((2, 3, 8, 10), 11).cuda()
    check(lib.cx_nn_relu_backward(_p(yr), _p(g), _p(dz), x.numel(), _s()), "relu bwd")
    assert torch.equal(dz.cpu(), torch.where(x.double() > 0, g.cpu().double(), 0.0).to(BF))
    o = torch.empty_like(xd)
    check(lib.cx_nn_add(_p(xd), _p(g), _p(o), x.numel(), _s()), "add")
    check_bf16(o, x.double() + g.cpu().double(), "add")


def test_mse_and_adam():
    lib, check = _lib()
    out = bf16_data((4, 8, 6, 6), 12)
    tgt = torch.randn((4, 8, 6, 6), generator=torch.Generator().manual_seed(13)).float()
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    dout = torch.empty((4, 8, 6, 6), dtype=BF, device="cuda")
    outd, tgtd = out.cuda(), tgt.cuda()
    check(lib.cx_nn_mse(_p(outd), _p(tgtd), _p(dout), _p(loss), out.numel(), _s()), "mse")
    o = out.double().requires_grad_(True)
    L = R.mse(o, tgt.double())
    L.backward()
    assert abs(float(loss) - float(L)) <= 1e-6 * float(L)
    check_bf16(dout, o.grad, "mse grad")
    n = 1000
    rng = np.random.default_rng(14)
    p0 = rng.standard_normal(n).astype(np.float32)
    p, m, v = p0.astype(np.float64), np.zeros(n), np.zeros(n)
    pd = torch.as_tensor(p0, device="cuda")
    md, vd = torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    pb = torch.empty(n, dtype=BF, device="cuda")
    for t in range(1, 6):
        g = rng.standard_normal(n).astype(np.float32)
        gd = torch.as_tensor(g, device="cuda")
        check(lib.cx_nn_adam(_p(pd), _p(md), _p(vd), _p(gd), _p(pb), n, 1e-2, 0.9, 0.999, 1e-8, t, _s()), "adam")
        p, m, v = R.adam(p, m, v, g.astype(np.float64), t, 1e-2)
    assert np.abs(pd.cpu().numpy() - p).max() <= 1e-5
    assert torch.equal(pb.cpu(), pd.cpu().to(BF))


def _ref_params(net):
    return [(c.wb.double().cpu(), c.b.double().cpu()) for c in net.layers]


def test_unet_forward_backward_against_reference():
    """Whole U-Net (4 levels, 32-256 channels) on a batch of 2 32x32 inputs:
    output and every parameter gradient against the FP64 reference evaluated
    with the same BF16 weights and input."""
    from paper_1908_03876_gb300.surrogate import UNet

    chans = (32, 64, 128, 256)
    net = UNet(cin=5, cout=8, chans=chans, seed=3)
    x = bf16_data((2, 5, 32, 32), 15)
    tgt = (0.3 * torch.randn((2, 8, 32, 32), generator=torch.Generator().manual_seed(16))).float()
    out = net.forward(x.cuda())
    loss, dout = net.loss(out, tgt.cuda())
    net.backward(dout)
    torch.cuda.synchronize()
    Lr, grads, out_r = R.loss_and_grads(_ref_params(net), x.double(), tgt.double(), chans)
    e_out = rel_l2(out.float(), out_r)
    print(f"[unet] out rel {e_out:.2e} loss {float(loss):.6e} vs {Lr:.6e}")
    assert e_out < 3e-2
    assert abs(float(loss) - Lr) <= 3e-2 * Lr
    worst = 0.0
    for c, (gw, gb) in zip(net.layers, grads):
        e = rel_l2(c.gw, gw)
        cos = float(torch.nn.functional.cosine_similarity(c.gw.double().cpu().flatten(), gw.flatten(), dim=0))
        worst = max(worst, e)
        assert e < 6e-2 and cos > 0.998, (c.cout, c.cin, e, cos)
        if gb.norm() > 0:
            assert rel_l2(c.gb, gb) < 6e-2
    print(f"[unet] worst weight-gradient rel L2 {worst:.2e}")


def test_unet_training_lowers_loss():
    """A few hundred Adam steps fit a fixed smooth map of the inputs."""
    from paper_1908_03876_gb300.surrogate import UNet

    net = UNet(cin=5, cout=2, chans=(16, 32, 64, 128), seed=1)
    g = torch.Generator().manual_seed(17)
    x = torch.randn((8, 5, 32, 32), generator=g)
    tgt = torch.stack([x[:, 0] * 0.5 + x[:, 1] * x[:, 2] * 0.2, torch.tanh(x[:, 3])], dim=1).float()
    xd, td = x.to(BF).cuda(), tgt.cuda()
    first = float(net.train_step(xd, td, lr=2e-3))
    for _ in range(300):
        last = float(net.train_step(xd, td, lr=2e-3))
    print(f"[unet train] loss {first:.3e} -> {last:.3e}")
    assert last < 0.1 * first


def test_conv_forward_f32_and_smooth():
    """FP32-output head convolution, and the periodic Gaussian low-pass
    against an explicit periodic sum."""
    lib, check = _lib()
    B, Cin, Cout, H, W = 2, 32, 8, 12, 16
    x = bf16_data((B, Cin, H, W), 20)
    w = bf16_data((Cout, Cin, 1, 1), 21, scale=0.2)
    b = torch.linspace(-0.1, 0.1, Cout, dtype=torch.float32)
    xd, wd, bd = x.cuda(), w.cuda(), b.cuda()
    wf, _ = packed(lib, check, wd, Cout, Cin, 1)
    y = torch.empty((B, Cout, H, W), dtype=torch.float32, device="cuda")
    check(lib.cx_nn_conv_forward_f32(_p(xd), _p(wf), _p(bd), _p(y), B, Cin, Cout, H, W, 1, _s()), "conv f32")
    ref = R.conv(x.double(), w.double(), b.double())
    assert rel_l2(y, ref) < 1e-6
    sigma, r = 1.5, 5
    d = np.arange(-r, r + 1)
    taps = np.exp(-0.5 * (d / sigma) ** 2)
    taps /= taps.sum()
    f = torch.randn((3, H, W), generator=torch.Generator().manual_seed(22), dtype=torch.float64)
    fd = f.float().cuda()
    tmp, out = torch.empty_like(fd), torch.empty_like(fd)
    td = torch.as_tensor(taps, dtype=torch.float32, device="cuda")
    check(lib.cx_nn_smooth(_p(fd), _p(tmp), _p(out), 3, H, W, _p(td), r, _s()), "smooth")
    g = f.numpy()
    ex = sum(taps[i] * np.roll(g, -int(d[i]), axis=2) for i in range(len(d)))
    ex = sum(taps[i] * np.roll(ex, -int(d[i]), axis=1) for i in range(len(d)))
    assert np.abs(out.cpu().numpy() - ex).max() < 1e-5


@pytest.mark.parametrize("B,Cin,Cout,H,W,ks,relu", [
    (2, 40, 64, 20, 13, 3, True),     # ragged input chunk and pixel tiles
    (3, 32, 32, 16, 16, 1, False),    # 1x1
    (1, 5, 32, 33, 9, 3, True),       # fewer inputs than one chunk
    (2, 64, 128, 16, 24, 3, True),    # 128-channel tile
    (1, 128, 256, 8, 8, 3, False),    # 256-channel tile, image smaller than the pixel tile
    (2, 48, 96, 12, 12, 3, True),     # 96 channels: three 32-channel tiles
    (2, 256, 128, 16, 16, 1, False),  # 1x1 with 16 input chunks
])
def test_conv_forward_tcgen05(B, Cin, Cout, H, W, ks, relu):
    """Convolution on the tcgen05 tensor cores (accumulator in tensor memory)
    against the FP64 reference and the mma.sync kernel."""
    lib, check = _lib()
    x = bf16_data((B, Cin, H, W), 31)
    w = bf16_data((Cout, Cin, ks, ks), 32, scale=1.0 / np.sqrt(Cin * ks * ks))
    b = torch.linspace(-0.3, 0.3, Cout, dtype=torch.float32)
    xd, wd, bd = x.cuda(), w.cuda(), b.cuda()
    wf, _ = packed(lib, check, wd, Cout, Cin, ks)
    y = torch.empty((B, Cout, H, W), dtype=BF, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    check(lib.cx_nn_conv_forward_tc(_p(xd), _p(wf), _p(bd), _p(y), B, Cin, Cout, H, W, ks, int(relu), _p(st), _s()),
          "conv tc")
    # the mma.sync kernel (through the FP32-output entry, no tensor-core dispatch)
    y2 = torch.empty((B, Cout, H, W), dtype=torch.float32, device="cuda")
    check(lib.cx_nn_conv_forward_f32(_p(xd), _p(wf), _p(bd), _p(y2), B, Cin, Cout, H, W, ks, _s()), "conv f32")
    if relu:
        y2 = torch.relu(y2)
    y2 = y2.to(BF)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    check_bf16(y, R.conv(x.double(), w.double(), b.double(), relu=relu), f"conv tcgen05 {Cin}->{Cout} k{ks}")
    d = (y.double() - y2.double()).abs().max().item()
    print(f"tcgen05 vs mma.sync max |diff| {d:.3e}")
    assert d <= 2.0 ** -7 * y2.double().abs().max().item()


@pytest.mark.parametrize("B,Cin,Cout,H,W", [
    (2, 40, 72, 16, 24),    # ragged input chunk, fewer than 128 output channels
    (1, 6, 32, 32, 32),     # the first layer (6 inputs, one chunk mostly padding)
    (2, 64, 256, 16, 16),   # two 128-channel output tiles
    (1, 256, 128, 8, 8),    # deep level: one pixel tile, 16 input chunks
    (3, 32, 32, 24, 40),    # tiles at every image border
])
def test_conv_backward_weight_tcgen05(B, Cin, Cout, H, W):
    """3x3 weight and bias gradients on the tcgen05 tensor cores against the
    FP64 reference and the mma.sync kernel, with 1, a few and more splits
    than pixel tiles (empty splits write zeros)."""
    lib, check = _lib()
    x = bf16_data((B, Cin, H, W), 41)
    dy = bf16_data((B, Cout, H, W), 42)
    xd, dyd = x.cuda(), dy.cuda()
    w = torch.zeros((Cout, Cin, 3, 3), dtype=torch.float64)
    xr = x.double().requires_grad_(True)
    wr = w.requires_grad_(True)
    br = torch.zeros(Cout, dtype=torch.float64, requires_grad=True)
    (R.conv(xr, wr, br) * dy.double()).sum().backward()
    ntiles = B * (H // 8) * (W // 8)
    for splits in (1, 5, ntiles + 3):
        nbytes = lib.cx_nn_conv_backward_weight_scratch(B, Cin, Cout, H, W, 3, splits)
        scratch = torch.full((nbytes // 4,), float("nan"), dtype=torch.float32, device="cuda")
        dw = torch.empty((Cout, Cin, 3, 3), dtype=torch.float32, device="cuda")
        db = torch.empty(Cout, dtype=torch.float32, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        check(lib.cx_nn_conv_backward_weight_tc(_p(xd), _p(dyd), _p(dw), _p(db), _p(scratch), splits, B, Cin, Cout, H,
                                                W, 3, _p(st), _s()), "bwd weight tc")
        dw2 = torch.empty_like(dw)
        db2 = torch.empty_like(db)
        scratch2 = torch.empty_like(scratch)
        check(lib.cx_nn_conv_backward_weight(_p(xd), _p(dyd), _p(dw2), _p(db2), _p(scratch2), splits, B, Cin, Cout, H,
                                             W, 3, _s()), "bwd weight")
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        e_w, e_b = rel_l2(dw, wr.grad), rel_l2(db, br.grad)
        d_w = rel_l2(dw, dw2)
        print(f"[wgrad tcgen05 {Cin}->{Cout} {H}x{W} splits {splits}] dW {e_w:.2e} db {e_b:.2e} vs mma.sync {d_w:.2e}")
        assert e_w < 1e-5 and e_b < 1e-5 and d_w < 1e-5
