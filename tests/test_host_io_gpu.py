"""cx_gradient_host: one gradient evaluation whose control comes from and
whose gradient goes to host memory, the copies overlapped with the kernels
chunk by chunk.  It must return exactly what cx_gradient returns on device
buffers (the same kernels run on the same inputs), with pinned and with
pageable host buffers, with time windows and across repeated calls."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1908_03876_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_03876_gb300.build import build

    build()


def _case(name):
    if name == "aniso32_windows":  # 40 windows of 2 steps: 20 chunks of 2 windows each way
        w = W.aniso(96, 64, 80, seed=21, precision=32, ckpt_every=7)
        w.windows = 40
    elif name == "geometry64":  # masked control window, solid nodes, FP64
        w = W.geometry(160, 48, 24, seed=5, precision=64, ckpt_every=5, win=40, rmin=3, rmax=7)
    else:  # one step per window, fewer windows than chunks: one window per chunk
        w = W.aniso(64, 64, 9, seed=22, precision=32, ckpt_every=4)
    return w


@pytest.mark.parametrize("name", ["aniso32_windows", "geometry64", "aniso32_short"])
@pytest.mark.parametrize("pinned", [True, False])
def test_gradient_host_equals_device_gradient(name, pinned):
    from paper_1908_03876_gb300.problem import Problem

    w = _case(name)
    p = Problem(w)
    outs = []
    for seed in (3, 4):  # two calls in a row reuse the copy streams and events
        g = torch.as_tensor(w.random_control(seed, 0.02), dtype=p.dtype, device="cuda").contiguous()
        J_dev, E_dev = p.gradient(g)
        J_dev = float(J_dev.item())
        E_ref = E_dev.cpu().numpy().copy()
        g_host = torch.empty(g.shape, dtype=g.dtype, pin_memory=pinned)
        g_host.copy_(g.cpu())
        E_host = torch.full(g.shape, float("nan"), dtype=g.dtype, pin_memory=pinned)
        J = p.gradient_host(g_host, E_host)
        nd = int(np.count_nonzero(E_host.numpy() != E_ref))
        print(f"[{name} pinned={pinned} seed={seed}] J {J:.17g} vs {J_dev:.17g}; gradient entries differing: {nd}")
        assert J == J_dev
        assert nd == 0
        outs.append(E_ref)
    assert not np.array_equal(outs[0], outs[1])  # the second call really used its own control
    p.close()


def test_gradient_host_rejects_null_buffers():
    from paper_1908_03876_gb300.problem import Problem

    w = _case("aniso32_short")
    p = Problem(w)
    rc = p.lib.cx_gradient_host(p.h, None, None, None, None, None)
    assert rc == 1  # CX_ERR_INVALID_ARG
    p.close()
