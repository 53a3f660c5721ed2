"""Three-species (attraction-repulsion chemotaxis, logistic source) CUDA path
against the FP64 oracle: forward fields and cost, the exact discrete adjoint
gradient, seeded vector-Jacobian products, an Armijo step, FP32 accuracy, and
a directional-derivative check at a larger size.  All calls go through the C
ABI of include/cxarc.h."""
import numpy as np
import pytest

import oracle
from paper_1908_03876_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _arc(nx, ny, N, k, precision=64, ctrl=2, aniso="rotated", adv="row", order=2, seed=5):
    w = W.arc(nx, ny, N, seed=seed, precision=precision, ckpt_every=k, ctrl_species=ctrl)
    # kinetics strong enough that every term matters over a few steps
    w.a1, w.a2, w.b1, w.b2, w.b3, w.c1, w.c2 = 0.05, 0.03, 0.04, 0.02, 0.01, 0.03, 0.05
    w.source_order = order
    if aniso == "const":
        w.aniso = "const"
        w.D_u_const, w.D_v_const, w.D_w_const = (0.06, 0.01, 0.03), (0.2, -0.02, 0.1), (0.12, 0.03, 0.08)
    elif aniso == "field":
        Du, Dv, Dw = w.D_fields()
        w.aniso, w.D_u_field, w.D_v_field, w.D_w_field = "field", Du, Dv, Dw
    if adv == "none":
        w.adv = "none"
    elif adv == "field":
        a = w.a_fields()
        a[..., 1] = 0.02 * np.cos(2 * np.pi * np.arange(nx) / nx)[None, :]
        w.adv, w.a_field = "field", a
    return w


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _problem(w, staging=1):
    from paper_1908_03876_gb300.arc import ArcProblem
    p = ArcProblem(w)
    p.set_staging(staging)
    return p


CASES = [
    dict(nx=40, ny=36, N=9, k=4),                                     # three segments, ragged last
    dict(nx=33, ny=20, N=7, k=7, ctrl=1, aniso="const", adv="none"),  # odd width, one segment
    dict(nx=48, ny=24, N=8, k=3, aniso="field", adv="field", order=1),
    dict(nx=300, ny=17, N=5, k=2),                                    # rows longer than a block
]


@pytest.mark.parametrize("staging", [0, 2], ids=["per-thread", "row-window"])
@pytest.mark.parametrize("case", CASES, ids=[str(i) for i in range(len(CASES))])
def test_arc_fp64_forward_and_gradient_match_oracle(case, staging):
    """Both kernel forms (the row-window kernels take every step they can:
    rows of whole 16-byte units, pulled inputs) against the oracle."""
    w = _arc(**case)
    p = _problem(w, staging)
    g = w.random_control(11, 0.05)
    J = float(p.forward(g).item())
    u, v, ww = (t.cpu().numpy() for t in p.fields())
    po = oracle.from_workload3(w)
    Jo, uvw = oracle.forward3(po, g)
    print("J", J, Jo)
    assert abs(J - Jo) <= 1e-12 * abs(Jo)
    for a, b in zip((u, v, ww), uvw):
        assert _rel(a, b) <= 1e-12
    _, E = p.gradient(g)
    _, Eo, _ = oracle.adjoint3(po, g)
    err = _rel(E.cpu().numpy(), Eo)
    print("dJ/dg rel L2", err)
    assert err <= 1e-12
    _, e2, einf = p.norms()
    assert abs(e2 - float(np.sum(Eo * Eo))) <= 1e-11 * float(np.sum(Eo * Eo))
    assert abs(einf - float(np.abs(Eo).max())) <= 1e-12 * float(np.abs(Eo).max())


def test_arc_fp64_seeded_vjp_matches_oracle():
    """Seeds on all three species, with and without the penalty term."""
    w = _arc(40, 36, 9, 4)
    p = _problem(w)
    g = w.random_control(12, 0.05)
    rng = np.random.default_rng(3)
    seeds = rng.standard_normal((3, w.ny, w.nx))
    p.forward(g)
    E = p.adjoint(g, seeds=list(seeds), penalty=True).cpu().numpy()
    po = oracle.from_workload3(w)
    _, Eo, _ = oracle.adjoint3(po, g, seeds)
    assert _rel(E, Eo) <= 1e-12
    V = p.adjoint(g, seeds=[seeds[0], None, seeds[2]], penalty=False).cpu().numpy()
    po.alpha = 0.0
    s2 = seeds.copy()
    s2[1] = 0.0
    _, Vo, _ = oracle.adjoint3(po, g, s2)
    assert _rel(V, Vo) <= 1e-12


def test_arc_fp64_armijo_step():
    """The accepted cost equals the oracle's cost at the updated control, and
    descends; the next step reuses the accepted trial's forward."""
    w = _arc(40, 36, 9, 4)
    p = _problem(w, 2)
    g = p.zeros_control()
    po = oracle.from_workload3(w)
    J_prev = None
    for it in range(3):
        info = p.step(g)
        Jo, _ = oracle.forward3(po, g.cpu().numpy())
        print(it, info, Jo)
        assert info["J"] < info["J0"]
        assert abs(info["J"] - Jo) <= 1e-12 * abs(Jo)
        if J_prev is not None:
            assert abs(info["J0"] - J_prev) <= 1e-12 * abs(J_prev)
        J_prev = info["J"]


@pytest.mark.parametrize("ctrl,staging", [(1, 0), (2, 0), (1, 2), (2, 2)])
def test_arc_fp32_against_fp64_oracle(ctrl, staging):
    """FP32 lattices against the FP64 oracle over 200 steps: fields within
    1e-4 and the gradient within 1e-3 (relative L2)."""
    w = _arc(64, 48, 200, 50, precision=32, ctrl=ctrl)
    w.a1, w.a2, w.b1, w.b2, w.b3, w.c1, w.c2 = 2e-3, 1e-3, 2e-3, 3e-3, 1e-3, 2e-3, 4e-3
    p = _problem(w, staging)
    g = w.random_control(13, 0.01)
    J, E = p.gradient(g)
    u, v, ww = (t.cpu().numpy() for t in p.fields())
    po = oracle.from_workload3(w)
    Jo, uvw = oracle.forward3(po, g)
    _, Eo, _ = oracle.adjoint3(po, g)
    errs = [_rel(a, b) for a, b in zip((u, v, ww), uvw)]
    eg = _rel(E.cpu().numpy(), Eo)
    print("FP32 field errors", errs, "gradient", eg, "J", float(J.item()), Jo)
    assert max(errs) <= 1e-4
    assert eg <= 1e-3
    assert abs(float(J.item()) - Jo) <= 1e-4 * abs(Jo)


def test_arc_fp64_directional_derivative_256():
    """At 256^2 (beyond what the oracle runs here), <dJ/dg, d> equals the
    central difference of J along a random direction d (FP64 GPU solves)."""
    w = _arc(256, 256, 40, 10)
    p = _problem(w)
    rng = np.random.default_rng(7)
    g = torch.as_tensor(w.random_control(14, 0.02), device="cuda")
    d = torch.as_tensor(rng.standard_normal(w.ctrl_shape), device="cuda")
    _, E = p.gradient(g)
    dd = float(torch.sum(E * d).item())
    h = 1e-4
    Jp = float(p.forward(g + h * d).item())
    Jm = float(p.forward(g - h * d).item())
    fd = (Jp - Jm) / (2 * h)
    print("directional", dd, fd)
    assert abs(dd - fd) <= 1e-5 * abs(dd)


def test_arc_errors():
    from paper_1908_03876_gb300 import _lib
    w = _arc(40, 36, 9, 4)
    p = _problem(w)
    with pytest.raises(_lib.CxError):
        p.adjoint(None)  # no forward yet
    w2 = _arc(40, 36, 9, 4)
    w2.lam_u = (-0.5, 0.02)  # a negative diffusivity gives a K eigenvalue outside (0, 2)
    with pytest.raises(_lib.CxError):
        _problem(w2)


def test_arc_fp32_staging_forms_agree_at_1024():
    """At the benchmark's grid (1024^2, the row-window kernels' default
    launch), 20 steps: the row-window and per-thread forms give the same
    fields and gradient to FP32 rounding, and the FP32 gradient is finite."""
    w = _arc(1024, 1024, 20, 10, precision=32)
    g = torch.as_tensor(w.random_control(15, 0.01), dtype=torch.float32, device="cuda")
    out = []
    for staging in (1, 0):
        p = _problem(w, staging)
        J, E = p.gradient(g)
        out.append((float(J.item()), E.clone(), [t.clone() for t in p.fields()]))
        p.close()
    (J1, E1, F1), (J0, E0, F0) = out
    assert abs(J1 - J0) <= 1e-6 * abs(J0)
    assert bool(torch.isfinite(E1).all())
    assert float(torch.linalg.norm(E1 - E0) / torch.linalg.norm(E0)) <= 1e-5
    for a, b in zip(F1, F0):
        assert float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) <= 1e-6


def test_arc_fp64_full_grid_against_oracle():
    """The bench's full 1024^2 grid (its physics, FP64), three steps: fields,
    J and the gradient at every node against the oracle on the same grid."""
    w = W.arc(1024, 1024, 3, seed=5, precision=64, ckpt_every=3)
    p = _problem(w)
    g = w.random_control(22, 0.01)
    _, E = p.gradient(g)
    J = float(p.norms()[0])
    fields = [t.cpu().numpy() for t in p.fields()]
    po = oracle.from_workload3(w)
    Jo, uvw = oracle.forward3(po, g)
    assert abs(J - Jo) <= 1e-12 * abs(Jo)
    for a, b in zip(fields, uvw):
        assert _rel(a, b) <= 1e-12
    _, Eo, _ = oracle.adjoint3(po, g)
    assert _rel(E.cpu().numpy(), Eo) <= 1e-12
