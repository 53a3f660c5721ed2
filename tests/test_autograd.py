"""MRTSolve: the forward solve as a torch.autograd.Function whose backward is
the checkpointed AMRT sweep, against finite differences and the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1908_03876_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_03876_gb300.build import build

    build()
    oracle.build()


def _crop_problem(N=12, k=4):
    # a 32x32 crop of the complex-geometry workload (discs, frame, masked window), FP64
    w = W.geometry(32, 32, N, seed=2, precision=64, ckpt_every=k, win=16, rmin=2, rmax=5)
    w.alpha = 1e-2
    return w


def test_autograd_matches_finite_differences():
    from paper_1908_03876_gb300.autograd import solve
    from paper_1908_03876_gb300.problem import Problem

    w = _crop_problem()
    p = Problem(w)
    rng = np.random.default_rng(0)
    wu = torch.as_tensor(rng.standard_normal((w.ny, w.nx)), device=p.device)
    wv = torch.as_tensor(rng.standard_normal((w.ny, w.nx)), device=p.device)
    mask = torch.as_tensor(1 - w.solid, device=p.device, dtype=torch.float64)

    def loss_of(g):
        u, v = solve(g, p)
        return (wu * mask * u).sum() + (wv * mask * v).sum() + 0.3 * (g * g).sum()

    g = torch.as_tensor(w.random_control(3, 0.05), device=p.device).requires_grad_(True)
    L = loss_of(g)
    L.backward()
    grad = g.grad.clone()
    h = 1e-6
    for seed in range(4):
        d = torch.as_tensor(np.random.default_rng(10 + seed).standard_normal(g.shape), device=p.device)
        with torch.no_grad():
            fd = (loss_of(g + h * d) - loss_of(g - h * d)) / (2 * h)
        ad = (grad * d).sum()
        print(f"direction {seed}: autograd {ad.item():.12e} fd {fd.item():.12e}")
        assert abs(ad.item() - fd.item()) <= 1e-7 * abs(fd.item()) + 1e-9


def test_autograd_matches_oracle_vjp():
    """The backward equals the oracle's seeded adjoint with alpha = 0."""
    from paper_1908_03876_gb300.autograd import solve
    from paper_1908_03876_gb300.problem import Problem

    w = _crop_problem(N=10, k=3)
    p = Problem(w)
    rng = np.random.default_rng(2)
    su, sv = rng.standard_normal((w.ny, w.nx)) * (1 - w.solid), rng.standard_normal((w.ny, w.nx)) * (1 - w.solid)
    g0 = w.random_control(4, 0.05)
    g = torch.as_tensor(g0, device=p.device).requires_grad_(True)
    u, v = solve(g, p)
    (u * torch.as_tensor(su, device=p.device)).sum().backward(retain_graph=True)
    gu = g.grad.clone()
    g.grad = None
    (v * torch.as_tensor(sv, device=p.device)).sum().backward()
    gv = g.grad.clone()
    po = oracle.from_workload(w)
    po.alpha = 0.0
    _, Eu, _ = oracle.adjoint(po, g0, su, np.zeros_like(sv))
    _, Ev, _ = oracle.adjoint(po, g0, np.zeros_like(su), sv)
    for a, b, name in ((gu, Eu, "u"), (gv, Ev, "v")):
        err = np.linalg.norm(a.cpu().numpy() - b) / np.linalg.norm(b)
        print(f"VJP through {name}^N vs oracle: rel L2 {err:.2e}")
        assert err < 1e-12


def test_autograd_windowed_control_with_penalty():
    """Time-windowed control (W = 4 windows of 3 steps) with alpha > 0: the
    backward is the library's penalty-free vector-Jacobian product, equal to
    the oracle's seeded adjoint with alpha = 0 (summed over each window's
    steps), and to central differences of a loss that adds its own penalty."""
    from paper_1908_03876_gb300.autograd import solve
    from paper_1908_03876_gb300.problem import Problem

    w = W.aniso(40, 32, 12, seed=9, precision=64, ckpt_every=5)
    w.windows = 4
    w.alpha = 0.05
    p = Problem(w)
    rng = np.random.default_rng(7)
    su, sv = rng.standard_normal((w.ny, w.nx)), rng.standard_normal((w.ny, w.nx))
    tsu, tsv = torch.as_tensor(su, device=p.device), torch.as_tensor(sv, device=p.device)
    g0 = w.random_control(8, 0.05)
    assert g0.shape == (4, 32, 40)

    def loss_of(g):
        u, v = solve(g, p)
        return (tsu * u).sum() + (tsv * v).sum() + 0.7 * (g * g).sum()

    g = torch.as_tensor(g0, device=p.device).requires_grad_(True)
    loss_of(g).backward()
    po = oracle.from_workload(w)
    po.alpha = 0.0
    _, Eo, _ = oracle.adjoint(po, g0, su, sv)
    vjp = g.grad.cpu().numpy() - 1.4 * g0
    err = np.linalg.norm(vjp - Eo) / np.linalg.norm(Eo)
    print(f"windowed VJP (alpha = {w.alpha}) vs oracle with alpha = 0: rel L2 {err:.2e}")
    assert err < 1e-12
    h = 1e-6
    for seed in range(3):
        d = torch.as_tensor(np.random.default_rng(20 + seed).standard_normal(g.shape), device=p.device)
        with torch.no_grad():
            fd = (loss_of(g + h * d) - loss_of(g - h * d)) / (2 * h)
        ad = (g.grad * d).sum()
        print(f"direction {seed}: autograd {ad.item():.12e} fd {fd.item():.12e}")
        assert abs(ad.item() - fd.item()) <= 1e-7 * abs(fd.item()) + 1e-9


def test_backward_after_other_forward_recomputes():
    """Two solves on one problem, then both backwards: the earlier one restores
    its checkpoints first, so both gradients are right."""
    from paper_1908_03876_gb300.autograd import solve
    from paper_1908_03876_gb300.problem import Problem

    w = _crop_problem(N=8, k=3)
    p = Problem(w)
    g1 = torch.as_tensor(w.random_control(5, 0.05), device=p.device).requires_grad_(True)
    g2 = torch.as_tensor(w.random_control(6, 0.05), device=p.device).requires_grad_(True)
    u1, _ = solve(g1, p)
    u2, _ = solve(g2, p)
    (u1.sum() + 2.0 * u2.sum()).backward()
    ref1 = torch.as_tensor(w.random_control(5, 0.05), device=p.device).requires_grad_(True)
    solve(ref1, p)[0].sum().backward()
    assert torch.allclose(g1.grad, ref1.grad, rtol=1e-13, atol=1e-15)


def test_gradcheck_tiny():
    from paper_1908_03876_gb300.autograd import MRTSolve
    from paper_1908_03876_gb300.problem import Problem

    w = W.aniso(8, 8, 4, seed=1, precision=64, ckpt_every=2)
    w.alpha = 0.0
    p = Problem(w)
    g = torch.as_tensor(w.random_control(7, 0.05), device=p.device).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda x: MRTSolve.apply(x, p), (g,), eps=1e-6, atol=1e-8, rtol=1e-6,
                                    fast_mode=True)
