"""Batched problems: one persistent launch per step over all problems' tiles,
replayed as a CUDA graph.  Checked against the oracle per problem, against the
single-problem path and across tile shapes (same per-node formulas, compiled
in other kernels: equal to 1e-13), and across graph replays (bitwise)."""
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


def _mixed(precision=64, N=14, k=5):
    """Uneven sizes, tensors, chemotaxis; one complex-geometry problem."""
    ws = []
    for i, (nx, ny) in enumerate([(40, 24), (64, 16), (33, 47), (48, 48), (20, 28)]):
        w = W.aniso(nx, ny, N, seed=10 + i, precision=precision, ckpt_every=k, chi=-0.02 * (i + 1))
        w.lam_u = w.lam_v = (0.08, 0.08 / (1 + i))
        ws.append(w)
    g = W.geometry(56, 44, N, seed=2, precision=precision, ckpt_every=k, win=24, rmin=3, rmax=7)
    ws.append(g)
    return ws


def _run_batch(ws, tile_x=None, threads=256, rows=None):
    from paper_1908_03876_gb300.batch import Batch

    b = Batch(ws)
    gs = [torch.as_tensor(w.random_control(50 + i, 0.02), dtype=b.dtype, device=b.device) for i, w in enumerate(ws)]
    b.bind(gs)
    if tile_x is not None or rows is not None:
        b.set_tiles(threads, 0, tile_x, rows)
    J, e2, emax = b.gradient()
    b.stream.synchronize()
    b.status()
    fields = [b.fields(i) for i in range(len(ws))]
    torch.cuda.synchronize()
    return b, gs, J.cpu().numpy().copy(), [E.cpu().numpy().copy() for E in b.E], \
        [(u.cpu().numpy(), v.cpu().numpy()) for u, v in fields], e2.cpu().numpy().copy()


def test_batch_fp64_matches_oracle_per_problem():
    ws = _mixed()
    b, gs, J, Es, fields, e2 = _run_batch(ws)
    for i, w in enumerate(ws):
        Jo, Eo, _ = oracle.adjoint(oracle.from_workload(w), gs[i].cpu().numpy())
        eJ = abs(J[i] - Jo) / abs(Jo)
        eE = np.linalg.norm(Es[i] - Eo) / np.linalg.norm(Eo)
        print(f"problem {i} ({w.nx}x{w.ny}): J rel {eJ:.1e}, dJ/dg rel L2 {eE:.1e}")
        assert eJ < 1e-12 and eE < 1e-12
        assert abs(e2[i] - np.sum(Eo * Eo)) <= 1e-12 * np.sum(Eo * Eo)


def _close(a, b, tol=1e-13):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) <= tol * np.linalg.norm(b)


def test_batch_equals_single_problem():
    from paper_1908_03876_gb300.problem import Problem

    ws = _mixed(N=9, k=4)
    b, gs, J, Es, fields, _ = _run_batch(ws)
    for i, w in enumerate(ws):
        p = Problem(w)
        Jp, Ep = p.gradient(gs[i])
        u, v = p.fields()
        assert _close(Es[i], Ep.cpu().numpy())
        assert _close(fields[i][0], u.cpu().numpy()) and _close(fields[i][1], v.cpu().numpy())
        assert abs(Jp.item() - J[i]) <= 1e-14 * abs(J[i])


def test_batch_tile_shapes_and_replay():
    ws = _mixed(N=9, k=4)
    _, _, J1, E1, F1, _ = _run_batch(ws, tile_x=[32] * len(ws), threads=256)
    _, _, J2, E2, F2, _ = _run_batch(ws, tile_x=[64, 128, 32, 64, 32, 128], threads=128, rows=[1, 3, 16, 2, 5, 1])
    b, gs, J3, E3, F3, _ = _run_batch(ws)
    J4, _, _ = b.gradient()  # graph replay
    b.stream.synchronize()
    for a, c in zip(E1, E2):
        assert _close(a, c)
    for a, c in zip(E1, E3):
        assert _close(a, c)
    for (u1, v1), (u2, v2) in zip(F1, F2):
        assert _close(u1, u2) and _close(v1, v2)
    assert np.allclose(J1, J2, rtol=1e-13, atol=0)
    assert np.array_equal(J3, J4.cpu().numpy())  # replaying the captured graph is deterministic


def test_batch_fp32_against_fp64_oracle():
    ws = _mixed(precision=32, N=30, k=8)
    b, gs, J, Es, fields, _ = _run_batch(ws)
    for i, w in enumerate(ws):
        Jo, Eo, _ = oracle.adjoint(oracle.from_workload(w), gs[i].double().cpu().numpy())
        eJ = abs(J[i] - Jo) / abs(Jo)
        eE = np.linalg.norm(Es[i] - Eo) / np.linalg.norm(Eo)
        print(f"fp32 problem {i}: J rel {eJ:.1e}, dJ/dg rel L2 {eE:.1e}")
        assert eJ < 1e-4 and eE < 1e-3


def test_autotuner_picks_admissible_config(tmp_path):
    """cx_batch_autotune: an admissible choice, applied to the batch, results
    unchanged by it (the probe's overwritten state is recomputed), and the
    cached line reused by a second batch of the same size classes."""
    from paper_1908_03876_gb300 import autotune
    from paper_1908_03876_gb300.batch import Batch

    ws = [W.aniso(nx, ny, 8, seed=3, precision=32, ckpt_every=4) for nx, ny in [(64, 64), (128, 64), (64, 128)]]
    b = Batch(ws)
    b.bind(b.zeros_controls())
    J0 = b.forward().cpu().numpy().copy()
    cache = tmp_path / "tune.txt"
    cfg = autotune.autotune(b, probe_steps=6, cache_path=cache)
    assert cfg["threads"] in (128, 256) and cfg["ms"] > 0
    for nx, tx in cfg["tile_x"].items():
        assert cfg["threads"] % tx == 0 and cfg["threads"] // tx <= 8 and tx >= 32
        assert cfg["rows"][nx] in (4, 8, 16, 32)
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and len(lines[0].split("\t")) == 4
    J1 = b.forward().cpu().numpy()
    assert np.allclose(J0, J1, rtol=1e-6)
    J2, gsq, _ = (x.cpu().numpy().copy() for x in b.gradient())
    b2 = Batch(ws)
    b2.bind(b2.zeros_controls())
    again = autotune.autotune(b2, probe_steps=6, cache_path=cache)
    assert again["tile_x"] == cfg["tile_x"] and again["rows"] == cfg["rows"] and again["threads"] == cfg["threads"]
    assert len(cache.read_text().splitlines()) == 1
    J3, gsq3, _ = (x.cpu().numpy() for x in b2.gradient())
    assert np.allclose(J2, J3, rtol=1e-6) and np.allclose(gsq, gsq3, rtol=1e-5)
    b.close()
    b2.close()


def test_batch_step_matches_oracle_gd():
    """Batched Armijo iterations (one trial forward over the problems still
    searching) against the oracle's per-problem iterations: J, step length,
    trials and the updated control after each of three steps."""
    from paper_1908_03876_gb300.batch import Batch

    ws = _mixed(N=12, k=5)
    b = Batch(ws)
    gs = b.zeros_controls()
    b.bind(gs)
    go = [np.zeros(w.ctrl_shape) for w in ws]
    lam_prev = [None] * len(ws)
    for it in range(3):
        info, st = b.step()
        assert all(s == 0 for s in st), st
        for i, w in enumerate(ws):
            go[i], io = oracle.gd_step(oracle.from_workload(w), go[i], lam_prev=lam_prev[i])
            lam_prev[i] = io["lam"]
            assert abs(info[i]["J0"] - io["J0"]) <= 1e-12 * abs(io["J0"]), (it, i)
            assert abs(info[i]["J"] - io["J"]) <= 1e-12 * abs(io["J"]), (it, i)
            assert info[i]["trials"] == io["trials"] and abs(info[i]["lam"] - io["lam"]) <= 1e-14 * io["lam"]
            err = np.linalg.norm(gs[i].cpu().numpy() - go[i]) / np.linalg.norm(go[i])
            assert err < 1e-12, (it, i, err)


def test_batch_windowed_and_switched_off():
    """Windowed controls in the batch (gradients against the oracle), and a
    switched-off problem: its control and gradient buffers are left alone and
    the others step as in a batch without it."""
    from paper_1908_03876_gb300.batch import Batch

    ws = _mixed(N=12, k=5)[:4]
    for w in ws:
        w.windows = 3
    b = Batch(ws)
    gs = [torch.as_tensor(w.random_control(70 + i, 0.02), dtype=b.dtype, device=b.device) for i, w in enumerate(ws)]
    b.bind(gs)
    J, _, _ = b.gradient()
    J = J.cpu().numpy()
    for i, w in enumerate(ws):
        Jo, Eo, _ = oracle.adjoint(oracle.from_workload(w), gs[i].cpu().numpy())
        assert abs(J[i] - Jo) <= 1e-12 * abs(Jo)
        assert np.linalg.norm(b.E[i].cpu().numpy() - Eo) <= 1e-12 * np.linalg.norm(Eo)
    before = [g.cpu().numpy().copy() for g in gs]
    E_off = b.E[2].clone()
    b.set_enabled([True, True, False, True])
    info, st = b.step()
    assert st == [0, 0, 0, 0] and info[2]["trials"] == 0
    assert np.array_equal(gs[2].cpu().numpy(), before[2]) and torch.equal(b.E[2], E_off)
    for i in (0, 1, 3):
        go, io = oracle.gd_step(oracle.from_workload(ws[i]), before[i])
        assert abs(info[i]["J"] - io["J"]) <= 1e-12 * abs(io["J"]) and info[i]["trials"] == io["trials"]
        assert np.linalg.norm(gs[i].cpu().numpy() - go) <= 1e-12 * np.linalg.norm(go)


def test_batch_seeded_adjoint_and_axpy():
    """Seeded AMRT sweep of every problem (the adjoint of u^N given per
    problem) against the oracle's seeded adjoint, then a per-problem axpy of
    the controls, and a step from there (which must restart with a forward)."""
    from paper_1908_03876_gb300.batch import Batch

    ws = _mixed(N=12, k=5)[:3]
    b = Batch(ws)
    gs = [torch.as_tensor(w.random_control(90 + i, 0.02), dtype=b.dtype, device=b.device) for i, w in enumerate(ws)]
    b.bind(gs)
    b.forward()
    rng = np.random.default_rng(5)
    seeds = [torch.as_tensor(rng.standard_normal((w.ny, w.nx)), dtype=b.dtype, device=b.device) for w in ws]
    e2, _ = b.adjoint(seeds)
    e2 = e2.cpu().numpy()
    for i, w in enumerate(ws):
        _, Eo, _ = oracle.adjoint(oracle.from_workload(w), gs[i].cpu().numpy(), seed_u=seeds[i].cpu().numpy())
        assert np.linalg.norm(b.E[i].cpu().numpy() - Eo) <= 1e-12 * np.linalg.norm(Eo), i
        assert abs(e2[i] - np.sum(Eo * Eo)) <= 1e-11 * np.sum(Eo * Eo)
    b.forward()
    b.adjoint(seeds, add_to_cost_seed=True)  # seed = (u^N - u_target) + seeds
    for i, w in enumerate(ws):
        p = oracle.from_workload(w)
        _, uN, _ = oracle.forward(p, gs[i].cpu().numpy())
        _, Eo, _ = oracle.adjoint(p, gs[i].cpu().numpy(), seed_u=uN - w.u_tgt + seeds[i].cpu().numpy())
        assert np.linalg.norm(b.E[i].cpu().numpy() - Eo) <= 1e-12 * np.linalg.norm(Eo), i
    before = [g.cpu().numpy().copy() for g in gs]
    E = [e.cpu().numpy().copy() for e in b.E]
    lam = [0.5, 0.0, 2.0]
    b.axpy(lam)
    torch.cuda.synchronize()
    for i in range(3):
        assert np.abs(gs[i].cpu().numpy() - (before[i] - lam[i] * E[i])).max() <= 1e-14 * (1 + np.abs(before[i]).max())
    info, st = b.step()
    assert st == [0, 0, 0]
    for i, w in enumerate(ws):
        J0o = oracle.forward(oracle.from_workload(w), before[i] - lam[i] * E[i])[0]
        assert abs(info[i]["J0"] - J0o) <= 1e-12 * abs(J0o)


def _aligned(precision=64, N=12, k=5, windows=0):
    """Problems the row-window batched kernel takes (no solid nodes, nx a
    whole number of 16-byte units): uneven sizes, heights that leave partial
    tiles, one problem with its control on a sub-window (g and E staged per
    thread)."""
    ws = []
    for i, (nx, ny) in enumerate([(40, 24), (64, 18), (96, 47), (20, 28), (128, 33)]):
        w = W.aniso(nx, ny, N, seed=30 + i, precision=precision, ckpt_every=k, chi=-0.02 * (i + 1))
        w.lam_u = w.lam_v = (0.08, 0.08 / (1 + i))
        w.windows = windows
        ws.append(w)
    ws[2].window = (8, 5, 60, 30)
    return ws


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("tiles", [None, (256, 32, 4), (128, 64, 3), (256, 128, 16)])
def test_batch_row_windows_bitwise_and_oracle(precision, tiles):
    """The row-window batched kernel (bulk copies of each item's row windows,
    mbarrier per stage) against per-thread staging: J, ||dJ/dg||^2, gradients
    and fields bitwise equal; FP64 gradients against the oracle."""
    ws = _aligned(precision)
    outs = []
    for rows in (True, False):
        from paper_1908_03876_gb300.batch import Batch

        b = Batch(ws)
        b.set_staging(rows)
        gs = [torch.as_tensor(w.random_control(50 + i, 0.02), dtype=b.dtype, device=b.device)
              for i, w in enumerate(ws)]
        b.bind(gs)
        if tiles is not None:
            th, tx, r = tiles
            b.set_tiles(th, 0, [min(tx, th) for _ in ws], [r] * len(ws))
        J, e2, _ = b.gradient()
        b.status()
        fields = [tuple(f.cpu().numpy() for f in b.fields(i)) for i in range(len(ws))]
        outs.append((J.cpu().numpy().copy(), e2.cpu().numpy().copy(), [E.cpu().numpy().copy() for E in b.E],
                     fields, [g.cpu().numpy() for g in gs]))
        b.close()
    (Jr, e2r, Er, Fr, gr), (Jt, e2t, Et, Ft, _) = outs
    assert np.array_equal(Jr, Jt) and np.array_equal(e2r, e2t)
    for i in range(len(ws)):
        assert np.array_equal(Er[i], Et[i]), i
        assert np.array_equal(Fr[i][0], Ft[i][0]) and np.array_equal(Fr[i][1], Ft[i][1]), i
    tol_J, tol_E = (1e-12, 1e-12) if precision == 64 else (1e-4, 1e-3)
    for i, w in enumerate(ws):
        Jo, Eo, _ = oracle.adjoint(oracle.from_workload(w), gr[i].astype(np.float64))
        eJ, eE = abs(Jr[i] - Jo) / abs(Jo), np.linalg.norm(Er[i] - Eo) / np.linalg.norm(Eo)
        print(f"row windows fp{precision} tiles {tiles} problem {i}: J {eJ:.1e} dJ/dg {eE:.1e}")
        assert eJ < tol_J and eE < tol_E


def test_batch_row_windows_steps_and_windows():
    """Armijo steps (line-search trial forwards read g - lam E through the row
    windows) and time-windowed controls with the row-window kernel: controls
    after two steps bitwise equal to per-thread staging, and the windowed
    gradient against the oracle."""
    from paper_1908_03876_gb300.batch import Batch

    ws = _aligned(64, windows=3)
    res = []
    for rows in (True, False):
        b = Batch(ws)
        b.set_staging(rows)
        gs = [torch.as_tensor(w.random_control(80 + i, 0.02), dtype=b.dtype, device=b.device)
              for i, w in enumerate(ws)]
        b.bind(gs)
        J, _, _ = b.gradient()
        J = J.cpu().numpy().copy()
        if rows:
            for i, w in enumerate(ws):
                Jo, Eo, _ = oracle.adjoint(oracle.from_workload(w), gs[i].cpu().numpy())
                assert abs(J[i] - Jo) <= 1e-12 * abs(Jo)
                assert np.linalg.norm(b.E[i].cpu().numpy() - Eo) <= 1e-12 * np.linalg.norm(Eo), i
        infos = []
        for _ in range(2):
            info, st = b.step()
            assert all(s == 0 for s in st), st
            infos.append([(x["J0"], x["J"], x["lam"], x["trials"]) for x in info])
        res.append((infos, [g.cpu().numpy().copy() for g in gs]))
        b.close()
    assert res[0][0] == res[1][0]
    for a, c in zip(res[0][1], res[1][1]):
        assert np.array_equal(a, c)
