"""GPU path (CUDA library through the C ABI) against the FP64 CPU oracle.

Tolerances (relative L2 against the oracle, from the project's accuracy bar):
  FP64 GPU: 1e-12 on u^N, v^N, psi^0 and dJ/dg, and on J;
  FP32 GPU: 1e-4 on fields, 1e-3 on dJ/dg.
Every comparison prints its measured error.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1908_03876_gb300 import workloads as W  # noqa: E402

TOL64 = 1e-12
TOL32_FIELD = 1e-4
TOL32_GRAD = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_03876_gb300.build import build

    build()
    oracle.build()


def rel(a, b):
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    b = np.asarray(b)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def run_both(w, g, seeds=None, launch=None):
    from paper_1908_03876_gb300.problem import Problem

    p = Problem(w)
    if launch:
        p.set_launch(*launch)
    J = p.forward(g)
    su, sv = (None, None) if seeds is None else seeds
    E = p.adjoint(g, su, sv)
    u, v = p.fields()
    psi0 = p.psi0()
    torch.cuda.synchronize()
    po = oracle.from_workload(w)
    Jo, uo, vo = oracle.forward(po, g)
    _, Eo, psio = oracle.adjoint(po, g, su, sv, want_psi0=True)
    # oracle psi0 is [ny][nx][2][Q]; the GPU's is [2][Q][ny][nx]
    psio = np.transpose(psio, (2, 3, 0, 1))
    if w.solid is not None:  # solid nodes hold no populations
        solid = torch.as_tensor(w.solid, device=psi0.device).bool()[None, None]
        psi0 = torch.where(solid, torch.zeros_like(psi0), psi0)
    return dict(J=(float(J.item()), Jo), u=(u, uo), v=(v, vo), E=(E, Eo), psi0=(psi0, psio), p=p)


def check(res, tol_field, tol_grad, label):
    eJ = abs(res["J"][0] - res["J"][1]) / abs(res["J"][1])
    eu, ev = rel(*res["u"]), rel(*res["v"])
    eE, ep = rel(*res["E"]), rel(*res["psi0"])
    print(f"[{label}] rel err: J {eJ:.2e} u {eu:.2e} v {ev:.2e} dJ/dg {eE:.2e} psi0 {ep:.2e}")
    assert eJ < tol_field and eu < tol_field and ev < tol_field
    assert eE < tol_grad and ep < tol_grad


# ---------------------------------------------------------------- FP64 parity

def test_plain64_d2q5_fp64_full():
    """The 64x64 D2Q5 FP64 problem in full (200 steps)."""
    w = W.plain64()
    g = w.random_control(1, 0.02)
    check(run_both(w, g), TOL64, TOL64, "plain64 D2Q5 fp64")


@pytest.mark.parametrize("Q", [5, 9])
def test_plain_ragged_fp64(Q):
    """Several tiles with a ragged tail in x and y; checkpoint interval not dividing N."""
    w = W.plain64(150, 37, 23, sigma=3.0, Q=Q)
    w.ckpt_every = 6
    g = w.random_control(2, 0.02)
    check(run_both(w, g), TOL64, TOL64, f"plain ragged Q{Q}")


def test_aniso_fp64_checkpointed():
    """Rotated anisotropic tensors, shear convection, chemotaxis; k = 7."""
    w = W.aniso(72, 56, 31, seed=1, precision=64, ckpt_every=7)
    g = w.random_control(3, 0.02)
    check(run_both(w, g), TOL64, TOL64, "aniso fp64")


def test_geometry_fp64():
    """Solid discs with bounce-back, solid frame, masked control window."""
    w = W.geometry(96, 80, 25, seed=2, precision=64, ckpt_every=8, win=40, rmin=3, rmax=9)
    g = w.random_control(4, 0.02)
    check(run_both(w, g), TOL64, TOL64, "geometry fp64")


def test_field_tensors_and_velocity_fp64():
    """Per-node tensor fields and per-node convection (FIELD modes)."""
    w = W.aniso(48, 40, 16, seed=5, precision=64, ckpt_every=5)
    Du, Dv = w.D_fields()
    rng = np.random.default_rng(0)
    w.aniso, w.D_u_field, w.D_v_field = "field", Du, Dv * 1.3
    w.adv = "field"
    w.a_field = rng.uniform(-0.03, 0.03, (w.ny, w.nx, 2))
    g = w.random_control(5, 0.02)
    check(run_both(w, g), TOL64, TOL64, "field modes fp64")


@pytest.mark.parametrize("source_order", [1, 2])
def test_explicit_seeds_fp64(source_order):
    """Adjoint seeded with arbitrary (seed_u, seed_v): the VJP used by autograd."""
    w = W.aniso(40, 32, 12, seed=6, precision=64, ckpt_every=4)
    w.source_order = source_order
    rng = np.random.default_rng(1)
    seeds = (rng.standard_normal((w.ny, w.nx)), rng.standard_normal((w.ny, w.nx)))
    g = w.random_control(6, 0.02)
    check(run_both(w, g, seeds=seeds), TOL64, TOL64, f"seeded order {source_order}")


def test_launch_shape_independent_bitwise():
    """FP64 fields and gradients are bitwise identical across launch shapes of
    the persistent kernels (no race between chunks or pipeline stages)."""
    w = W.geometry(80, 64, 12, seed=3, precision=64, ckpt_every=5, win=30, rmin=3, rmax=8)
    g = w.random_control(7, 0.02)
    from paper_1908_03876_gb300.problem import Problem

    outs = []
    for shape in [(256, 0), (128, 0), (64, 0), (256, 7), (64, 13)]:  # (threads, persistent blocks)
        p = Problem(w)
        p.set_launch(*shape)
        p.forward(g)
        E = p.adjoint(g)
        u, v = p.fields()
        outs.append((u.cpu().numpy(), v.cpu().numpy(), E.cpu().numpy()))
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a, b)


def _staging_case(case):
    if case == "aniso32_ragged":   # 200 columns: a partial last row segment for 128 and 256 threads
        w = W.aniso(200, 48, 14, seed=11, precision=32, ckpt_every=5)
    elif case == "aniso64_window":  # control on a sub-window: g arrives by per-thread copies
        w = W.aniso(96, 40, 12, seed=12, precision=64, ckpt_every=4)
        w.window = (10, 6, 50, 20)
    elif case == "plain64_q5_windows":
        w = W.plain64(64, 64, 24, sigma=4.0, Q=5)
        w.ckpt_every, w.windows = 6, 4
    elif case == "geometry64":  # solid discs and frame: bounce-back flags staged with each row segment
        w = W.geometry(160, 48, 12, seed=5, precision=64, ckpt_every=4, win=40, rmin=3, rmax=7)
    elif case == "geometry32":  # 208 columns: a partial last segment for 128 and 256 threads
        w = W.geometry(208, 56, 14, seed=6, precision=32, ckpt_every=5, win=48, rmin=3, rmax=8)
    elif case == "geometry64_periodic":  # no solid frame: fluid runs and walls across the periodic ends
        from dataclasses import replace

        w = W.geometry(160, 48, 12, seed=5, precision=64, ckpt_every=4, win=40, rmin=3, rmax=7)
        solid = w.solid.copy()
        solid[:, 0] = solid[:, -1] = 0
        solid[0, :] = solid[-1, :] = 0
        solid[10:14, 156:160] = 1  # a wall on the right end whose neighbours wrap to column 0
        solid[20:22, 0:3] = 1
        x0, y0, cnx, cny = w.window
        w = replace(w, solid=solid, cmask=(1 - solid[y0:y0 + cny, x0:x0 + cnx]).astype(np.uint8))
    else:  # one 16-byte unit per row (nx = 4): every segment touches both periodic ends
        w = W.aniso(4, 24, 10, seed=13, precision=32, ckpt_every=5)
    return w


@pytest.mark.parametrize("case", ["aniso32_ragged", "aniso64_window", "plain64_q5_windows", "aniso32_nx4",
                                  "geometry64", "geometry32", "geometry64_periodic"])
@pytest.mark.parametrize("threads", [128, 256])
def test_row_window_staging_bitwise(case, threads):
    """Bulk row-window staging (cp.async.bulk + mbarrier per row segment) and
    per-thread staging give bitwise identical J, fields and dJ/dg; the
    row-window result also matches the oracle."""
    from paper_1908_03876_gb300.problem import Problem

    w = _staging_case(case)
    g = w.random_control(21, 0.02)
    outs = []
    for rows in (True, False):
        p = Problem(w)
        p.set_launch(threads, 4)  # several row segments per block: the row-window kernels take the steps
        p.set_staging(rows)
        J = float(p.forward(g).item())
        E = p.adjoint(g)
        u, v = p.fields()
        torch.cuda.synchronize()
        outs.append((J, u.cpu().numpy(), v.cpu().numpy(), E.cpu().numpy()))
    assert outs[0][0] == outs[1][0]
    for a, b in zip(outs[0][1:], outs[1][1:]):
        assert np.array_equal(a, b)
    po = oracle.from_workload(w)
    Jo, uo, _ = oracle.forward(po, g)
    _, Eo, _ = oracle.adjoint(po, g)
    tol_f, tol_g = (TOL64, TOL64) if w.precision == 64 else (TOL32_FIELD, TOL32_GRAD)
    eJ, eu, eE = abs(outs[0][0] - Jo) / abs(Jo), rel(outs[0][1], uo), rel(outs[0][3], Eo)
    print(f"[row windows {case} t{threads}] rel err: J {eJ:.2e} u {eu:.2e} dJ/dg {eE:.2e}")
    assert eJ < tol_f and eu < tol_f and eE < tol_g


def test_row_window_wait_timeout_is_reported():
    """A stage wait that never completes ends its launch within the wait's
    time bound instead of hanging: in the staging test mode every stage
    expects 16 bytes more than it copies, the next synchronising call reports
    CX_ERR_TIMEOUT (and keeps reporting it), and the context stays usable: a
    new problem then matches the oracle."""
    import time

    from paper_1908_03876_gb300 import _lib
    from paper_1908_03876_gb300.problem import Problem

    w = W.aniso(64, 32, 6, seed=3, precision=32, ckpt_every=3)
    g = w.random_control(5, 0.02)
    p = Problem(w)
    _lib.check(p.lib.cx_set_staging(p.h, 2), "cx_set_staging")
    t0 = time.perf_counter()
    p.forward(g)
    with pytest.raises(_lib.CxError) as ei:
        p.norms()
    dt = time.perf_counter() - t0
    print(f"timeout reported after {dt:.2f} s")
    assert ei.value.code == 7 and dt < 30
    p.forward(g)
    with pytest.raises(_lib.CxError) as ei:
        p.norms()
    assert ei.value.code == 7
    q = Problem(w)
    J = float(q.forward(g).item())
    Jo, _, _ = oracle.forward(oracle.from_workload(w), g)
    assert abs(J - Jo) / abs(Jo) < TOL32_FIELD


def test_repeated_adjoint_and_state():
    """A second adjoint after one forward repeats the first (tape bookkeeping);
    adjoint before any forward is refused."""
    from paper_1908_03876_gb300 import _lib
    from paper_1908_03876_gb300.problem import Problem

    w = W.aniso(40, 40, 20, seed=8, precision=64, ckpt_every=6)
    g = w.random_control(8, 0.02)
    p = Problem(w)
    with pytest.raises(_lib.CxError) as ei:
        p.adjoint(g)
    assert ei.value.code == 4
    p.forward(g)
    E1 = p.adjoint(g).clone()
    E2 = p.adjoint(g)
    assert torch.equal(E1, E2)


def test_step_matches_oracle_fp64():
    """One Armijo steepest-descent iteration (cx_step) against the oracle's."""
    from paper_1908_03876_gb300.problem import Problem

    w = W.plain64(32, 32, 30, sigma=2.0, Q=9)
    p = Problem(w)
    g = p.zeros_control()
    info = p.step(g)
    go, io = oracle.gd_step(oracle.from_workload(w), np.zeros(w.ctrl_shape))
    print("step", info, io)
    assert abs(info["J0"] - io["J0"]) <= 1e-12 * abs(io["J0"])
    assert abs(info["J"] - io["J"]) <= 1e-12 * abs(io["J"])
    assert abs(info["lam"] - io["lam"]) <= 1e-12 * io["lam"] and info["trials"] == io["trials"]
    assert rel(g, go) < 1e-12
    info2 = p.step(g)
    go2, io2 = oracle.gd_step(oracle.from_workload(w), go, lam_prev=io["lam"])
    assert abs(info2["J"] - io2["J"]) <= 1e-12 * abs(io2["J"])
    assert rel(g, go2) < 1e-12


@pytest.mark.parametrize("k", [5, 30])
def test_windowed_control_fp64(k):
    """Control piecewise constant over W = 5 time windows (30 steps): J, fields
    and the window gradients (sums of the per-step gradients) against the
    oracle; checkpoint intervals that cut windows (k = 5 with 6-step windows)
    and a single segment."""
    w = W.aniso(40, 36, 30, seed=4, precision=64, ckpt_every=k)
    w.windows = 5
    g = w.random_control(7, 0.05)
    assert g.shape == (5, 36, 40)
    check(run_both(w, g), TOL64, TOL64, f"windowed fp64 k{k}")


def test_windowed_step_matches_oracle_fp64():
    """cx_step on a windowed control against the oracle's Armijo iteration."""
    from paper_1908_03876_gb300.problem import Problem

    w = W.plain64(24, 24, 20, sigma=2.0, Q=9)
    w.windows = 4
    p = Problem(w)
    g = p.zeros_control()
    assert tuple(g.shape) == (4, 24, 24)
    info = p.step(g)
    go, io = oracle.gd_step(oracle.from_workload(w), np.zeros(w.ctrl_shape))
    assert abs(info["J"] - io["J"]) <= 1e-12 * abs(io["J"]) and info["trials"] == io["trials"]
    assert rel(g, go) < 1e-12


@pytest.mark.parametrize("variant", ["FR", "PR", "HS", "DY"])
def test_cg_matches_oracle_fp64(variant):
    """Nonlinear CG (Wolfe-Powell line search) on the GPU against the
    oracle's iterations: J, step, trials, r and restarts per iteration, and
    the control after four iterations."""
    from paper_1908_03876_gb300.problem import Problem

    w = W.aniso(40, 36, 20, seed=4, precision=64, ckpt_every=7)
    w.windows = 4
    w.chi = -0.3
    p = Problem(w)
    g = p.zeros_control()
    po = oracle.from_workload(w)
    go, st = np.zeros(w.ctrl_shape), None
    for it in range(4):
        info = p.cg_step(g, variant)
        go, st, io = oracle.cg_iteration(po, go, st, variant=variant)
        print(variant, it, info, {k: io[k] for k in ("J", "lam", "trials", "r", "restarted")})
        assert abs(info["J"] - io["J"]) <= 1e-12 * abs(io["J"])
        assert abs(info["lam"] - io["lam"]) <= 1e-10 * io["lam"] and info["trials"] == io["trials"]
        assert abs(info["r"] - io["r"]) <= 1e-8 * max(1e-3, abs(io["r"])) and info["restarted"] == io["restarted"]
    assert rel(g, go) < 1e-11


def test_cg_fp32_runs_to_the_rounding_floor():
    """FP32 lattices: nonlinear CG keeps decreasing J until the Wolfe search
    can no longer make progress, where it falls back to Armijo steps (soft
    reset) instead of failing; J never increases and ends well below J(0)."""
    from paper_1908_03876_gb300._lib import CxError
    from paper_1908_03876_gb300.problem import Problem

    w = W.aniso(64, 64, 40, seed=3, precision=32, ckpt_every=10)
    w.windows = 4
    w.chi = -0.3
    p = Problem(w)
    g = p.zeros_control()
    Js, fallbacks = [], 0
    for it in range(80):
        try:
            info = p.cg_step(g, "PR")
        except CxError as e:
            assert e.code == 6  # not even a steepest-descent step decreased J: converged
            break
        fallbacks += info["trials"] > 30
        if Js:
            assert info["J0"] <= Js[-1] * (1 + 1e-12)
        assert info["J"] <= info["J0"]
        Js.append(info["J"])
    print(f"CG FP32: {len(Js)} iterations, J {Js[0]:.6e} -> {Js[-1]:.6e}, {fallbacks} fallback steps")
    assert len(Js) >= 10 and Js[-1] < Js[0]


@pytest.mark.parametrize("k", [6, 20])
def test_tlm_matches_oracle_fp64(k):
    """Sensitivity problem (tangent-linear MRT pass) along a random direction:
    du^N, dv^N against the oracle's tangent-linear model, with checkpoint
    segments (k = 6) and without (k = N)."""
    from paper_1908_03876_gb300.problem import Problem

    w = W.aniso(40, 36, 20, seed=6, precision=64, ckpt_every=k)
    w.windows = 4
    w.chi = -0.3
    g = w.random_control(11, 0.05)
    dg = w.random_control(12, 1.0)
    p = Problem(w)
    p.forward(g)
    du, dv, sq = p.tlm(g, dg)
    _, duo, dvo = oracle.tlm(oracle.from_workload(w), g, dg)
    print(f"tlm k={k}: du {rel(du, duo):.2e} dv {rel(dv, dvo):.2e}")
    assert rel(du, duo) < 1e-12 and rel(dv, dvo) < 1e-12
    assert abs(sq - np.sum(duo * duo)) <= 1e-12 * np.sum(duo * duo)
    # the forward state survives: an adjoint after the sensitivity pass is the plain one
    E = p.adjoint(g)
    _, Eo, _ = oracle.adjoint(oracle.from_workload(w), g)
    assert rel(E, Eo) < 1e-12


@pytest.mark.parametrize("window", [None, (10, 6, 60, 20)])
@pytest.mark.parametrize("threads", [128, 256])
def test_tlm_row_windows_bitwise(window, threads):
    """The sensitivity pass with row-window staging (k_tlm_rows) and with
    per-thread staging gives bitwise identical du^N, dv^N (FP32, a partial
    last row segment; with the control on a sub-window dg is staged per
    thread)."""
    from paper_1908_03876_gb300.problem import Problem

    w = W.aniso(200, 40, 12, seed=7, precision=32, ckpt_every=5)
    w.windows = 4
    w.window = window
    g = w.random_control(13, 0.05)
    dg = w.random_control(14, 1.0)
    outs = []
    for rows in (True, False):
        p = Problem(w)
        p.set_launch(threads, 4)  # several row segments per block: the row-window kernels take the steps
        p.set_staging(rows)
        p.forward(g)
        du, dv, sq = p.tlm(g, dg)
        torch.cuda.synchronize()
        outs.append((du.cpu().numpy(), dv.cpu().numpy(), sq))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert outs[0][2] == outs[1][2]


@pytest.mark.parametrize("window", [None, (10, 6, 60, 20)])
def test_cadjoint_row_windows_bitwise(window):
    """The continuous adjoint with row-window staging (k_cadj_rows) and with
    per-thread staging give bitwise identical gradients (FP32, a partial last
    row segment; with the control on a sub-window g is staged per thread).
    Both inline the same node body; it is compiled without multiply-add
    contraction so that both round every operation alike."""
    from paper_1908_03876_gb300.problem import Problem

    w = W.aniso(200, 40, 12, seed=8, precision=32, ckpt_every=5)
    w.windows = 4
    w.window = window
    g = w.random_control(15, 0.05)
    outs = []
    for rows in (True, False):
        p = Problem(w)
        p.set_launch(256, 4)  # several row segments per block: the row-window kernels take the steps
        p.set_staging(rows)
        p.forward(g)
        E = p.cadjoint(g)
        torch.cuda.synchronize()
        outs.append(E.cpu().numpy().astype(np.float64))
    nd = int(np.count_nonzero(outs[0] != outs[1]))
    print(f"cadjoint row windows vs per-thread ({window}): {nd} entries differ")
    assert nd == 0


@pytest.mark.parametrize("window", [None, (10, 6, 60, 20)])
def test_cadjoint_row_windows_fp64_against_oracle(window):
    """The continuous adjoint with row-window staging (k_cadj_rows takes every
    step but the first: 200 columns, a partial last row segment, four blocks
    of 256 threads so each walks many segments) against the oracle's at 1e-12
    in FP64, and bitwise against per-thread staging."""
    from paper_1908_03876_gb300.problem import Problem

    w = W.aniso(200, 40, 12, seed=8, precision=64, ckpt_every=5)
    w.windows = 4
    w.window = window
    w.chi = -0.3
    g = w.random_control(15, 0.05)
    outs = []
    for rows in (True, False):
        p = Problem(w)
        p.set_launch(256, 4)
        p.set_staging(rows)
        p.forward(g)
        outs.append(p.cadjoint(g).cpu().numpy())
    _, Eo = oracle.cadjoint(oracle.from_workload(w), g)
    e = rel(outs[0], Eo)
    nd = int(np.count_nonzero(outs[0] != outs[1]))
    print(f"cadjoint row windows fp64 ({window}): rel {e:.2e} vs oracle, {nd} entries differ from per-thread")
    assert e < 1e-12
    assert nd == 0


@pytest.mark.parametrize("case", ["aniso", "geometry"])
def test_continuous_adjoint_matches_oracle_fp64(case):
    """Continuous-adjoint gradient (time-reversed MRT solve of the adjoint
    PDE) against the oracle's: rotated tensors with shear convection and time
    windows, or solid discs with a masked control window; checkpointed."""
    from paper_1908_03876_gb300.problem import Problem

    if case == "aniso":
        w = W.aniso(40, 36, 20, seed=7, precision=64, ckpt_every=6)
        w.windows = 4
        w.chi = -0.3
    else:
        w = W.geometry(48, 40, 16, seed=2, precision=64, ckpt_every=5, win=24, rmin=3, rmax=6)
    g = w.random_control(13, 0.05)
    p = Problem(w)
    p.forward(g)
    Ec = p.cadjoint(g)
    _, Eo = oracle.cadjoint(oracle.from_workload(w), g)
    print(f"continuous adjoint {case}: rel {rel(Ec, Eo):.2e}")
    assert rel(Ec, Eo) < 1e-12


def test_lma_step_matches_oracle_fp64():
    """Steepest descent with the linearised line search: three iterations
    against the oracle's."""
    from paper_1908_03876_gb300.problem import Problem

    w = W.aniso(40, 36, 20, seed=4, precision=64, ckpt_every=7)
    w.windows = 4
    w.chi = -0.3
    p = Problem(w)
    g = p.zeros_control()
    po = oracle.from_workload(w)
    go = np.zeros(w.ctrl_shape)
    for it in range(3):
        info = p.lma_step(g)
        go, io = oracle.lma_step(po, go)
        assert abs(info["J"] - io["J"]) <= 1e-12 * abs(io["J"])
        assert abs(info["lam"] - io["lam"]) <= 1e-10 * io["lam"] and info["trials"] == io["trials"]
    assert rel(g, go) < 1e-11


# ---------------------------------------------------------------- FP32 parity

def test_aniso_fp32_against_fp64_oracle():
    w = W.aniso(96, 80, 60, seed=1, precision=32, ckpt_every=16)
    g = w.random_control(9, 0.02)
    check(run_both(w, g), TOL32_FIELD, TOL32_GRAD, "aniso fp32")


def test_geometry_fp32_against_fp64_oracle():
    w = W.geometry(96, 96, 40, seed=2, precision=32, ckpt_every=10, win=48, rmin=3, rmax=10)
    g = w.random_control(10, 0.02)
    check(run_both(w, g), TOL32_FIELD, TOL32_GRAD, "geometry fp32")


@pytest.mark.parametrize("case", ["aniso128_2000", "geometry80_5000"])
def test_fp32_at_full_horizon_against_fp64_oracle(case):
    """FP32 lattices over the benchmark workloads' full horizons, element-wise
    against the FP64 oracle: the anisotropic problem (shear convection,
    chemotaxis) at 128x128 for 2000 steps with a checkpoint every 100, and
    the complex-geometry problem (discs, bounce-back, masked control window)
    at 80x80 for 5000 steps with a checkpoint every 100.  u^N and v^N within
    1e-4 relative L2, dJ/dg within 1e-3; the measured errors are printed."""
    if case == "aniso128_2000":
        w = W.aniso(128, 128, 2000, seed=1, precision=32, ckpt_every=100)
    else:
        w = W.geometry(80, 80, 5000, seed=2, precision=32, ckpt_every=100, win=40, rmin=3, rmax=8)
    g = w.random_control(9, 0.01)
    oracle.set_threads(0)
    check(run_both(w, g), TOL32_FIELD, TOL32_GRAD, f"{case} fp32 vs fp64 oracle")


# ------------------------------------------------- full-size workload (sampled)

def test_aniso1024_fp32_full_size_sampled():
    """1024x1024 D2Q9 FP32 in the benchmark's launch configuration: the first
    steps against the oracle (every node), and u-mass conservation over the
    full 2000 steps (sum_i S_i = 0, no source in the u equation)."""
    from paper_1908_03876_gb300.problem import Problem

    wf = W.aniso()  # 1024^2, N = 2000, k = 100
    short = W.aniso(N=3, ckpt_every=2)
    g = short.random_control(11, 0.02)
    check(run_both(short, g), TOL32_FIELD, TOL32_GRAD, "aniso1024 fp32, 3 steps")
    p = Problem(wf)
    J = p.forward(None)
    u, v = p.fields()
    mass0 = float(np.sum(wf.u0))
    massN = float(u.double().sum().item())
    print(f"aniso1024 2000 steps: J={J.item():.6e}, u-mass drift {abs(massN / mass0 - 1):.2e}")
    assert np.isfinite(J.item())
    assert abs(massN / mass0 - 1) < 1e-5


def _crop(w, x0, y0, nx, ny, N, k):
    """The sub-problem on [x0, x0 + nx) x [y0, y0 + ny) of workload w (inside
    its control window), periodic at its own edges: its nodes farther than
    2N from the crop's edges see exactly the full problem's data for N steps
    (one lattice link per step in the forward and again in the adjoint)."""
    from dataclasses import replace

    wx0, wy0, wcx, wcy = w.win
    assert wx0 <= x0 and x0 + nx <= wx0 + wcx and wy0 <= y0 and y0 + ny <= wy0 + wcy
    sl = (slice(y0, y0 + ny), slice(x0, x0 + nx))
    cm = None if w.cmask is None else w.cmask[y0 - wy0:y0 - wy0 + ny, x0 - wx0:x0 - wx0 + nx].copy()
    return replace(w, nx=nx, ny=ny, N=N, ckpt_every=k, theta=w.theta[sl].copy(),
                   solid=None if w.solid is None else w.solid[sl].copy(), u0=w.u0[sl].copy(),
                   v0=w.v0[sl].copy(), u_tgt=w.u_tgt[sl].copy(), window=(0, 0, nx, ny), cmask=cm)


def test_geometry4096_fp32_full_size_sampled():
    """4096x4096 D2Q9 FP32 complex geometry (random discs, 20% solid, control
    on the 256x256 window) in the benchmark's launch configuration.
    (1) Three steps on the full grid: u^N, v^N and dJ/dg on a 128x128 patch
    inside the control window against the oracle run on that patch (nodes at
    least 10 links from the patch edges, which the patch's own periodic edges
    cannot reach in 2 x 3 steps).  (2) The full 5000 steps (checkpoint every
    100): J and the gradient finite, the gradient zero on solid window nodes,
    and u-mass conserved (bounce-back walls, and the chemotactic source has
    zero mass)."""
    from paper_1908_03876_gb300.problem import Problem

    N, m = 3, 10
    wf = W.geometry(N=N, ckpt_every=2)
    wx0, wy0 = wf.win[0], wf.win[1]
    g = wf.random_control(12, 0.02)
    p = Problem(wf)
    J = p.forward(g)
    E = p.adjoint(g)
    u, v = p.fields()
    torch.cuda.synchronize()
    x0, y0, n = 65, wy0 + 128, 128  # a patch whose interior is 30% solid
    wc = _crop(wf, x0, y0, n, n, N, 2)
    gc = g[:, y0 - wy0:y0 - wy0 + n, x0 - wx0:x0 - wx0 + n].copy()
    assert wc.solid[m:-m, m:-m].mean() > 0.2, "the patch should contain solid nodes"
    po = oracle.from_workload(wc)
    _, uo, vo = oracle.forward(po, gc)
    _, Eo, _ = oracle.adjoint(po, gc)
    ins = (slice(m, n - m), slice(m, n - m))
    ug = u[y0:y0 + n, x0:x0 + n].cpu().numpy()[ins]
    vg = v[y0:y0 + n, x0:x0 + n].cpu().numpy()[ins]
    Eg = E[:, y0 - wy0:y0 - wy0 + n, x0 - wx0:x0 - wx0 + n].cpu().numpy()[(slice(None),) + ins]
    eu, ev, eE = rel(ug, uo[ins]), rel(vg, vo[ins]), rel(Eg, Eo[(slice(None),) + ins])
    print(f"geometry4096 fp32, 3 steps, patch interior: u {eu:.2e} v {ev:.2e} dJ/dg {eE:.2e}; J={J.item():.6e}")
    assert eu < TOL32_FIELD and ev < TOL32_FIELD and eE < TOL32_GRAD
    del p, u, v, E
    torch.cuda.empty_cache()

    from dataclasses import replace

    wl = replace(wf, N=5000, ckpt_every=100)  # the full workload: 5000 steps, checkpoint every 100
    p = Problem(wl)
    gl = torch.as_tensor(wl.random_control(13, 0.01), dtype=torch.float32, device="cuda")
    _, E = p.gradient(gl)
    J, _, ginf = p.norms()
    u, _ = p.fields()
    solid_win = torch.as_tensor(1 - wl.cmask, device="cuda").bool()
    mass0 = float(np.sum(wl.u0 * (1 - wl.solid)))
    massN = float(u.double().sum().item())
    print(f"geometry4096 5000 steps: J={J:.6e}, max|dJ/dg|={ginf:.3e}, u-mass drift {abs(massN / mass0 - 1):.2e}")
    assert np.isfinite(J) and np.isfinite(ginf) and ginf > 0
    assert bool(torch.isfinite(E).all())
    assert float(E[:, solid_win].abs().max()) == 0.0
    assert abs(massN / mass0 - 1) < 1e-4
