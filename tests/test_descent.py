"""The optimisation loop (paper_1908_03876_gb300/descent.py): stopping rules,
the JSON-lines log and checkpoint/resume, on a stand-in problem whose
iterations are exact steps on a quadratic (the loop's host logic only; the
library's own iterations are checked against the oracle in the GPU tests)."""
import json

import pytest

torch = pytest.importorskip("torch")

from paper_1908_03876_gb300 import descent  # noqa: E402


class Quadratic:
    """J(g) = 1/2 |g - t|^2; every iteration takes the exact half step
    g <- g - (g - t) / 2, so J falls by 4x per iteration."""

    device = torch.device("cpu")
    dtype = torch.float64

    def __init__(self, t):
        self.t = t
        self.calls = 0

    def _J(self, g):
        return 0.5 * float(((g - self.t) ** 2).sum())

    def _iterate(self, g):
        self.calls += 1
        J0, E = self._J(g), g - self.t
        g -= 0.5 * E
        return dict(J0=J0, J=self._J(g), lam=0.5, grad_sq=float((E * E).sum()), grad_inf=float(E.abs().max()),
                    trials=1)

    def step(self, g, E=None):
        return self._iterate(g)

    def lma_step(self, g, E=None):
        return self._iterate(g)

    def cg_step(self, g, variant="PR"):
        info = self._iterate(g)
        info.pop("grad_inf")
        return info


def _problem():
    t = torch.linspace(-1.0, 2.0, 24, dtype=torch.float64).reshape(4, 6)
    return Quadratic(t), torch.zeros(4, 6, dtype=torch.float64)


def test_stops_at_the_target_cost_and_logs_every_iteration(tmp_path):
    p, g = _problem()
    J_start = p._J(g)
    log = tmp_path / "run.jsonl"
    recs = descent.descend(p, g, 50, target=J_start * 4.0 ** -5 * 1.0000001, log=str(log))
    assert len(recs) == 5 and recs[-1]["stop"] == "target"
    lines = [json.loads(ln) for ln in log.read_text().splitlines()]
    assert [r["iter"] for r in lines] == list(range(5))
    assert all(r["J"] == pytest.approx(r["J0"] / 4.0) for r in lines)
    assert all({"lam", "trials", "grad_norm", "grad_inf", "seconds", "method"} <= set(r) for r in lines)


def test_stops_on_the_gradient_ratio_and_the_iteration_count():
    p, g = _problem()
    recs = descent.descend(p, g, 50, grad_ratio=0.1)  # |E| halves per iteration: 0.5^4 < 0.1 at the 5th
    assert len(recs) == 5 and recs[-1]["stop"] == "grad_ratio"
    p, g = _problem()
    recs = descent.descend(p, g, 3, method="cg-PR")
    assert len(recs) == 3 and recs[-1]["stop"] == "iters" and "grad_inf" not in recs[-1]


def test_checkpoint_and_resume_continue_the_same_descent(tmp_path):
    p, g = _problem()
    straight = descent.descend(p, g.clone(), 8)
    ck = tmp_path / "ck.pt"
    p, g = _problem()
    first = descent.descend(p, g, 3, method="lma", checkpoint=str(ck))
    assert first[-1]["stop"] == "iters"
    q, _ = _problem()
    g2, start, method, last = descent.resume(str(ck), q)
    assert start == 3 and method == "lma" and last["iter"] == 2
    rest = descent.descend(q, g2, 8, method=method, start=start)
    assert [r["iter"] for r in rest] == list(range(3, 8))
    assert [r["J"] for r in first + rest] == pytest.approx([r["J"] for r in straight], rel=1e-15)


def test_rejects_an_unknown_method():
    p, g = _problem()
    with pytest.raises(ValueError):
        descent.descend(p, g, 2, method="newton")
