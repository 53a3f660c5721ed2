"""D3Q19 CUDA path (include/cx3d.h) against the D3Q19 oracle: forward
fields and cost, the exact discrete adjoint gradient, seeded vector-Jacobian
products, an Armijo step, FP32 accuracy and a directional derivative at a
larger size."""
import numpy as np
import pytest

import oracle
from paper_1908_03876_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _w(nx, ny, nz, N, k, precision=64, aniso="const", adv="row", order=2, seed=6):
    w = W.aniso3d(N=N, seed=seed, precision=precision, ckpt_every=k, nx=nx, ny=ny, nz=nz)
    w.chi, w.r_vu, w.r_vv = -0.3, 0.05, -0.04
    w.s = (1.0, 1.1, 0.9, 1.2, 1.05, 0.95, 1.15)
    w.source_order = order
    rng = np.random.default_rng(seed)
    w.v0 = 0.5 + 0.1 * rng.standard_normal((nz, ny, nx))
    if aniso == "field":
        Du, Dv = w.D_fields()
        z = np.arange(nz)[:, None, None, None] / nz
        w.aniso, w.D_u_field, w.D_v_field = "field", Du * (1 + 0.3 * np.sin(2 * np.pi * z)), Dv
    if adv == "none":
        w.adv = "none"
    elif adv == "field":
        a = w.a_fields()
        a[..., 2] = 0.02 * np.cos(2 * np.pi * np.arange(nx) / nx)[None, None, :]
        w.adv, w.a_field = "field", a
    return w


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _problem(w):
    from paper_1908_03876_gb300.d3 import D3Problem
    return D3Problem(w)


CASES = [
    dict(nx=12, ny=10, nz=8, N=9, k=4),                                  # three segments, ragged last
    dict(nx=9, ny=7, nz=5, N=6, k=6, aniso="field", adv="none"),         # odd sizes, one segment
    dict(nx=10, ny=6, nz=12, N=7, k=3, adv="field", order=1),
    dict(nx=70, ny=5, nz=4, N=4, k=2),                                   # rows longer than a warp
]


@pytest.mark.parametrize("case", CASES, ids=[str(i) for i in range(len(CASES))])
def test_d3q19_fp64_forward_and_gradient_match_oracle(case):
    w = _w(**case)
    p = _problem(w)
    g = w.random_control(11, 0.05)
    J = float(p.forward(g).item())
    u, v = (t.cpu().numpy() for t in p.fields())
    po = oracle.from_workload3d(w)
    Jo, uo, vo = oracle.forward3d(po, g)
    print("J", J, Jo)
    assert abs(J - Jo) <= 1e-12 * abs(Jo)
    assert _rel(u, uo) <= 1e-12 and _rel(v, vo) <= 1e-12
    _, E = p.gradient(g)
    _, Eo, _ = oracle.adjoint3d(po, g)
    err = _rel(E.cpu().numpy(), Eo)
    print("dJ/dg rel L2", err)
    assert err <= 1e-12
    _, e2, einf = p.norms()
    assert abs(e2 - float(np.sum(Eo * Eo))) <= 1e-11 * float(np.sum(Eo * Eo))
    assert abs(einf - float(np.abs(Eo).max())) <= 1e-12 * float(np.abs(Eo).max())


def test_d3q19_fp64_seeded_vjp_matches_oracle():
    w = _w(12, 10, 8, 9, 4)
    p = _problem(w)
    g = w.random_control(12, 0.05)
    rng = np.random.default_rng(3)
    su, sv = rng.standard_normal((2, w.nz, w.ny, w.nx))
    p.forward(g)
    E = p.adjoint(g, seed_u=su, seed_v=sv, penalty=True).cpu().numpy()
    po = oracle.from_workload3d(w)
    _, Eo, _ = oracle.adjoint3d(po, g, su, sv)
    assert _rel(E, Eo) <= 1e-12
    V = p.adjoint(g, seed_u=None, seed_v=sv, penalty=False).cpu().numpy()
    po.alpha = 0.0
    _, Vo, _ = oracle.adjoint3d(po, g, np.zeros_like(su), sv)
    assert _rel(V, Vo) <= 1e-12


def test_d3q19_fp64_armijo_step():
    w = _w(12, 10, 8, 9, 4)
    p = _problem(w)
    g = p.zeros_control()
    po = oracle.from_workload3d(w)
    J_prev = None
    for it in range(3):
        info = p.step(g)
        Jo, _, _ = oracle.forward3d(po, g.cpu().numpy())
        print(it, info, Jo)
        assert info["J"] < info["J0"]
        assert abs(info["J"] - Jo) <= 1e-12 * abs(Jo)
        if J_prev is not None:
            assert abs(info["J0"] - J_prev) <= 1e-12 * abs(J_prev)
        J_prev = info["J"]


def test_d3q19_fp32_against_fp64_oracle():
    """FP32 lattices against the FP64 oracle over 100 steps on 24^3: fields
    within 1e-4 and the gradient within 1e-3 (relative L2)."""
    w = _w(24, 24, 24, 100, 25, precision=32)
    w.chi, w.r_vu, w.r_vv = -0.1, 0.01, -0.005
    p = _problem(w)
    g = w.random_control(13, 0.01)
    J, E = p.gradient(g)
    u, v = (t.cpu().numpy() for t in p.fields())
    po = oracle.from_workload3d(w)
    Jo, uo, vo = oracle.forward3d(po, g)
    _, Eo, _ = oracle.adjoint3d(po, g)
    eu, ev, eg = _rel(u, uo), _rel(v, vo), _rel(E.cpu().numpy(), Eo)
    print("FP32 errors u", eu, "v", ev, "dJ/dg", eg, "J", float(J.item()), Jo)
    assert max(eu, ev) <= 1e-4 and eg <= 1e-3
    assert abs(float(J.item()) - Jo) <= 1e-4 * abs(Jo)


def test_d3q19_fp64_directional_derivative_64():
    """At 64^3, <dJ/dg, d> equals the central difference of J along a random
    direction (FP64 GPU solves)."""
    w = _w(64, 64, 64, 12, 4)
    p = _problem(w)
    rng = np.random.default_rng(7)
    g = torch.as_tensor(w.random_control(14, 0.02), device="cuda")
    d = torch.as_tensor(rng.standard_normal(w.ctrl_shape), device="cuda")
    _, E = p.gradient(g)
    dd = float(torch.sum(E * d).item())
    h = 1e-4
    fd = (float(p.forward(g + h * d).item()) - float(p.forward(g - h * d).item())) / (2 * h)
    print("directional", dd, fd)
    assert abs(dd - fd) <= 1e-5 * abs(dd)


def test_d3q19_fp64_full_grid_against_oracle():
    """The bench's full 128^3 grid (its physics, FP64), three steps: fields and
    J against the oracle run on the same grid, and the gradient of the first
    step at every node."""
    w = W.aniso3d(128, 3, seed=6, precision=64, ckpt_every=3)
    p = _problem(w)
    g = w.random_control(21, 0.01)
    _, E = p.gradient(g)
    J = float(p.norms()[0])
    u, v = (t.cpu().numpy() for t in p.fields())
    po = oracle.from_workload3d(w)
    Jo, uo, vo = oracle.forward3d(po, g)
    assert abs(J - Jo) <= 1e-12 * abs(Jo)
    assert _rel(u, uo) <= 1e-12 and _rel(v, vo) <= 1e-12
    _, Eo, _ = oracle.adjoint3d(po, g)
    assert _rel(E.cpu().numpy(), Eo) <= 1e-12
