"""Learned warm start, end to end at a small size: the plain batched descent
generates optimal solutions, the U-Net is trained on their terminal residuals
with the library's BF16 kernels, and on held-out problems the warm start
(proposal from the predicted residual by one forward and one seeded AMRT
sweep) reaches the plain optimum (J <= J* (1 + 1e-6)) in fewer descent
iterations than the plain method from g = 0, with a proposal closer to g*
than the zero control."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_03876_gb300.build import build

    build()


def test_warm_start_gains_over_plain_descent():
    from paper_1908_03876_gb300 import warmstart as WS

    train = WS.problems(512, 5000, size=64, N=64, windows=8, ckpt_every=16)
    test = WS.problems(16, 700000, size=64, N=64, windows=8, ckpt_every=16)
    ref = WS.descend(train, max_iter=200, want_residual=True)
    model = WS.Surrogate(seed=1)
    D = np.stack([r - r0 for r, r0 in zip(ref["residual"], ref["residual_init"])])
    losses = model.fit(WS.features(train), np.stack(ref["residual_init"]), D, epochs=30, batch_size=16, lr=2e-3)
    assert losses[-1] < 0.5 * losses[1]
    ref_te = WS.descend(test, max_iter=200, want_residual=True)
    ev = WS.evaluate(model, test, ref_te)
    print(ev)
    assert ev["warm_reached"] >= len(test) - 3, ev   # the rest fall back to the plain method
    assert ev["g0_rel_err_median"] < 0.4, ev         # the zero control has relative error 1
    assert ev["J_excess_at_g0_median"] < 0.3 * ev["J_excess_at_zero_median"], ev
    # descent iterations including the fallback runs
    assert ev["warm_iters_total"] < 0.95 * ev["cold_iters_total"], ev
