"""The Python use shown in the README runs as written (small sizes)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_03876_gb300.build import build

    build()


def test_readme_python_use(tmp_path):
    from paper_1908_03876_gb300 import autograd, autotune
    from paper_1908_03876_gb300 import workloads as W
    from paper_1908_03876_gb300.batch import Batch
    from paper_1908_03876_gb300.problem import Problem

    w = W.aniso(64, 64, 40, precision=32, ckpt_every=10)
    p = Problem(w)
    g = p.zeros_control()
    J0 = float(p.forward(g).item())
    J, E = p.gradient(g)
    info = p.step(g)
    assert info["J"] < J0
    info = p.cg_step(g, "PR")
    assert info["J"] <= info["J0"]
    u, v = autograd.solve(g.requires_grad_(), p)
    (u.sum() + v.sum()).backward()
    assert g.grad is not None and bool(torch.isfinite(g.grad).all())

    b = Batch([W.aniso(128, 64, 20, ckpt_every=10), W.aniso(64, 128, 20, ckpt_every=10)])
    b.bind(b.zeros_controls())
    cfg = autotune.autotune(b, probe_steps=6, cache_path=tmp_path / "tiles.txt")
    J, gsq, gmax = b.gradient()
    assert cfg["threads"] in (128, 256) and bool(torch.isfinite(J).all()) and bool((gsq > 0).all())
