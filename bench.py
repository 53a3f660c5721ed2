"""Benchmark: fwd+adjoint MLUPS of the MRT/AMRT gradient on one GB300.

One step = one gradient evaluation of the anisotropic 1024x1024 D2Q9 FP32
problem (2000 time steps, checkpoint every 100): the forward MRT solve writing
checkpoints, the segment recompute writing the adjoint tape, the AMRT adjoint
sweep with the fused gradient, and the FP64 reductions of J and ||dJ/dg||.
MLUPS = nodes x time steps / seconds per gradient evaluation.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs an independent problem (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="aniso1024", nx=1024, ny=1024, N=2000, k=100)
# algorithmic bytes per node and step (FP32, D2Q9, two species):
#   forward   18 pulls + 18 stores (144) + angle (4) + g (4) + Phi in/out (8)  = 160
#   recompute forward + tape (u, G_x, G_y) store (12)                           = 172
#   adjoint   144 + tape read (12) + angle (4) + sigma in/out (8) + g (4) + dJ/dg (4) = 176
BYTES = dict(forward=160, recompute=172, adjoint=176)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, device_index=0):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9 or f[0] != str(device_index):
                    continue
                try:
                    sm.append(float(f[1]))
                    smax = float(f[2])
                except ValueError:
                    continue
                for nm, val in zip(names, f[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def _traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    from the kernel's sources as they are now; else None."""
    try:
        from paper_1908_03876_gb300.kernel_hash import kernel_source_hash

        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            tr = json.load(fh)
        ent = tr.get(kernel)
        if not ent or ent.get("sources_hash") != kernel_source_hash(kernel):
            return None
        return ent["dram_bytes_per_launch"]
    except Exception:
        return None


def _batch_traffic(nodes, kernel="k_batch_rows"):
    """DRAM bytes of one batched forward launch over `nodes` nodes, from the
    per-node figure of the committed capture of `kernel` (its sources unchanged)."""
    try:
        from paper_1908_03876_gb300.kernel_hash import kernel_source_hash

        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            ent = json.load(fh).get(kernel)
        if not ent or ent.get("sources_hash") != kernel_source_hash(kernel):
            return None
        return ent["forward_dram_bytes_per_node"] * nodes
    except Exception:
        return None


def cpu_baseline(nsteps=8, single_thread=True):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the workload:
    the full 1024x1024 lattice for `nsteps` time steps, forward + adjoint, on
    all host cores (OpenMP over rows) and, if asked, on one core."""
    import oracle
    from paper_1908_03876_gb300 import workloads as W

    oracle.build()
    w = W.aniso(WORKLOAD["nx"], WORKLOAD["ny"], nsteps, seed=1, precision=64, ckpt_every=nsteps)
    p = oracle.from_workload(w)
    g = w.random_control(0, 0.01)
    ncpu = os.cpu_count() or 1

    def timed(threads):
        used = oracle.set_threads(threads)
        t0 = time.perf_counter()
        oracle.adjoint(p, g)  # runs the forward and the AMRT sweep
        dt = time.perf_counter() - t0
        return w.nx * w.ny * nsteps / dt / 1e6, dt, used

    mlups, dt, used = timed(ncpu)
    out = {"value": mlups, "unit": "MLUPS", "cores": used, "kind": "oracle", "nproc": ncpu,
           "sample": f"{w.nx}x{w.ny} D2Q9 FP64, {nsteps} of {WORKLOAD['N']} time steps, forward + AMRT adjoint, "
                     f"{dt:.1f} s, C with OpenMP over rows on {used} threads"}
    if single_thread:
        m1, dt1, _ = timed(1)
        out["single_thread"] = {"value": m1, "unit": "MLUPS", "cores": 1, "seconds": dt1}
        oracle.set_threads(ncpu)
    return out


def geometry_block(dev, staging, steps=5, warmup=2, N=20, k=10, size=4096):
    """The complex-geometry workload (4096x4096 D2Q9 FP32, random solid discs,
    20% solid, one-cell solid frame, control on a 256x256 masked window) on
    its full grid: per-launch times of the forward, recompute and adjoint
    kernels from CUDA events over `steps` gradient evaluations of N time steps
    (checkpoint every k), and the HBM fraction at the algorithmic bytes per
    fluid node (populations, angle, node-local scalars, one byte of mask) plus
    the control and gradient bytes of the controlled nodes."""
    import numpy as np
    import torch

    from paper_1908_03876_gb300 import workloads as W
    from paper_1908_03876_gb300.problem import Problem

    w = W.geometry(size, size, N, seed=2, precision=32, ckpt_every=k)
    fluid = int(np.count_nonzero(w.solid == 0))
    ctrl = int(np.count_nonzero(w.cmask))
    prob = Problem(w, device=dev)
    prob.set_staging(staging == "rows")
    g = torch.as_tensor(w.random_control(200, 0.01), dtype=torch.float32, device=dev).contiguous()
    E = torch.empty_like(g)
    for _ in range(warmup):
        prob.gradient(g, out=E)
    torch.cuda.synchronize()
    prob.set_timing(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(prob.stream)
    for _ in range(steps):
        prob.gradient(g, out=E)
    ev1.record(prob.stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    phases = prob.timing()
    prob.set_timing(False)
    J, _, _ = prob.norms()
    prob.close()
    hbm, peak_kind = _peaks()
    # algorithmic bytes per fluid node: 144 (populations) + 4 (angle) + 1 (mask) + node-local scalars
    per_fluid = dict(forward=144 + 4 + 1 + 8, recompute=144 + 4 + 1 + 8 + 12, adjoint=144 + 4 + 1 + 12 + 8)
    per_ctrl = dict(forward=4, recompute=4, adjoint=8)
    out = {}
    for ph in ("forward", "recompute", "adjoint"):
        t, n = phases[ph]
        if n <= 0:
            continue
        us = t * 1e3 / n
        byts = per_fluid[ph] * fluid + per_ctrl[ph] * ctrl
        ach = byts / (us * 1e-6) / 1e9
        out[ph] = {"us_per_launch": us, "launches": n, "bytes_per_launch": byts, "achieved": ach,
                   "frac": ach / hbm, "bytes_per_fluid_node": per_fluid[ph], "bytes_per_ctrl_node": per_ctrl[ph]}
    return {"workload": f"geometry{size}: {size}x{size} D2Q9 FP32, {100 * (1 - fluid / w.nx / w.ny):.1f}% solid discs + "
                        f"frame, control on a 256x256 masked window, {N} steps, checkpoint every {k}",
            "fluid_nodes": fluid, "controlled_nodes": ctrl, "staging": staging, "ms_per_gradient": ms,
            "fluid_mlups": fluid * N / (ms * 1e-3) / 1e6, "kernels": out, "peak": hbm, "peak_source": peak_kind,
            "J": J}


def fp32_error_vs_oracle(dev, nx=128, N=None, k=None):
    """Relative L2 errors of the FP32 GPU path against the FP64 oracle on the
    benchmark's physics and schedule (N steps, checkpoint every k) at a grid
    the oracle finishes in seconds: u^N, v^N, dJ/dg and J."""
    import numpy as np
    import torch

    import oracle
    from paper_1908_03876_gb300 import workloads as W
    from paper_1908_03876_gb300.problem import Problem

    N = N or WORKLOAD["N"]
    k = k or WORKLOAD["k"]
    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)
    w = W.aniso(nx, nx, N, seed=1, precision=32, ckpt_every=k)
    g = w.random_control(100, 0.01)
    p = Problem(w, device=dev)
    J = float(p.forward(g).item())
    E = p.adjoint(g).double().cpu().numpy()
    u, v = p.fields()
    u, v = u.double().cpu().numpy(), v.double().cpu().numpy()
    p.close()
    po = oracle.from_workload(w)
    Jo, uo, vo = oracle.forward(po, g)
    _, Eo, _ = oracle.adjoint(po, g)

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    return {"workload": f"aniso {nx}x{nx} D2Q9 FP32, {N} steps, checkpoint every {k} (the benchmark's physics "
                        "and schedule at a size the oracle finishes in seconds)",
            "u": rel(u, uo), "v": rel(v, vo), "dJdg": rel(E, Eo), "J": abs(J - Jo) / abs(Jo),
            "tolerance": {"fields": 1e-4, "dJdg": 1e-3}}


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle timed on this machine's host cores."""
    if rank != 0:
        return
    steps, warm = max(1, args.steps), max(0, args.warmup)
    nsteps = 4
    times = []
    base = None
    for i in range(warm + steps):
        b = cpu_baseline(nsteps, single_thread=False)
        if i >= warm:
            times.append(b)
        base = b
    val = statistics.mean(t["value"] for t in times)
    base["value"] = val
    base.pop("single_thread", None)
    line = {"metric": "fwd+adjoint MLUPS", "value": val, "unit": "MLUPS", "n_gpus": args.gpus, "steps": steps,
            "warmup": warm, "ms_per_step": WORKLOAD["nx"] * WORKLOAD["ny"] * WORKLOAD["N"] / val / 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)", "impl": "reference",
            "config": {"workload": "aniso1024: 1024x1024 D2Q9, 2000 steps, k=100 (oracle timed on a "
                                   f"{nsteps}-step sample per bench step)", "l2": "inputs larger than L2"},
            "cpu_baseline": base,
            "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batch_block(dev, problems=256, N=1000, steps=2, warmup=1, staging="thread", profile=False, rank=0, world=1,
                dist=None):
    """Many independent problems in one persistent launch per step, replayed
    as a CUDA graph (problems {64..512}^2, N steps, checkpoint every 100),
    sharded over ranks with no collective on the data path: aggregate MLUPS of
    gradient evaluations, the HBM fraction of all lattice launches, and the
    per-problem FP32 gradient error against the FP64 oracle on a sample."""
    import numpy as np
    import torch

    from paper_1908_03876_gb300 import autotune, sharding
    from paper_1908_03876_gb300 import workloads as W
    from paper_1908_03876_gb300.batch import Batch

    if profile:  # small profiling case: 20 steps, k = 10, default tiles
        allw = W.batch_workloads(problems, N=20, seed=3, ckpt_every=10)
    else:
        allw = W.batch_workloads(problems, N=N, seed=3)
    mine = sharding.my_problems(allw, rank, world)
    b = Batch(mine, device=dev)
    b.set_staging(staging == "rows")
    # seeded controls drawn on the device (N x nodes values per problem)
    gs = []
    for i, w in enumerate(mine):
        gen = torch.Generator(device=dev).manual_seed(500 + i)
        gs.append(0.01 * torch.randn(w.ctrl_shape, generator=gen, dtype=torch.float32, device=dev))
    b.bind(gs)
    t0 = time.perf_counter()
    if profile:
        cfg = {"threads": 256, "tile_x": {s: 256 for s in (64, 128, 256, 512)}, "rows": {}}
        autotune.apply(b, cfg)
    else:
        cfg = autotune.autotune(b, probe_steps=12)
    t_tune = time.perf_counter() - t0
    nodes = sum(w.nx * w.ny for w in mine)
    Nn = mine[0].N
    for _ in range(warmup):
        b.gradient()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    for _ in range(steps):
        b.gradient()
    e1.record(b.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    b.status()
    ms, all_nodes = sharding.aggregate(ms, float(nodes))
    mlups = all_nodes * Nn / (ms * 1e-3) / 1e6
    hbm, peak_kind = _peaks()
    k = mine[0].ckpt_every
    byts = all_nodes * (Nn * BYTES["forward"] + (Nn - k) * BYTES["recompute"] + Nn * BYTES["adjoint"])
    ach = byts / (ms * 1e-3) / world / 1e9
    b.close()
    del gs
    torch.cuda.empty_cache()
    err = [float("nan")]
    if rank == 0 and not profile:
        err = []
        import oracle

        oracle.build()
        sample = [W.batch_workloads(problems, N=6, seed=3, ckpt_every=3)[i] for i in (0, 1, 2, 3, 5, 8)]
        sb = Batch(sample, device=dev)
        sg = [torch.as_tensor(w.random_control(700 + i, 0.01), dtype=torch.float32, device=dev)
              for i, w in enumerate(sample)]
        sb.bind(sg)
        autotune.apply(sb, {"threads": cfg["threads"], "tile_x": {w.nx: cfg["tile_x"].get(w.nx, 64) for w in sample},
                            "rows": cfg.get("rows", {})})
        sb.gradient()
        torch.cuda.synchronize()
        for i, w in enumerate(sample):
            _, Eo, _ = oracle.adjoint(oracle.from_workload(w), sg[i].double().cpu().numpy())
            E = sb.E[i].double().cpu().numpy()
            err.append(float(np.linalg.norm(E - Eo) / np.linalg.norm(Eo)))
        sb.close()
    kern = "k_batch_rows" if staging == "rows" else "k_batch"
    return {"workload": f"batch: {problems} problems, nx, ny in {{64,128,256,512}}, {Nn} steps, checkpoint every "
                        f"{k}, one persistent launch per step, CUDA graph",
            "mlups": mlups, "ms_per_gradient": ms, "nodes": all_nodes, "steps": steps, "warmup": warmup,
            "tiles": cfg, "autotune_s": t_tune, "staging": staging,
            "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                         "traffic": _batch_traffic(all_nodes / world, kern),
                         "kernel": kern + " (all lattice launches of the step)", "peak_source": peak_kind},
            "per_problem_grad_rel_err_fp32_vs_oracle": {"sample": "6 problems, 6 steps", "max": max(err),
                                                        "values": err},
            "gpu_launches": steps * (Nn + len(mine) + 1 + 1 + max(0, Nn // k - 2) + (Nn - k) + Nn + 1)}


def run_batch(args, rank, world, local):
    """The batched workload (batch_block) as its own bench line."""
    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1908_03876_gb300.build import build

    if rank == 0:
        build()
    if dist:
        dist.barrier()
    clocks = Clocks()
    if rank == 0:
        clocks.start()
    res = batch_block(dev, problems=args.problems, steps=args.steps, warmup=args.warmup,
                      staging=args.staging or "thread", profile=args.profile, rank=rank, world=world, dist=dist)
    clk = clocks.stop(local) if rank == 0 else None
    if rank == 0:
        line = {
            "metric": "fwd+adjoint MLUPS (batched)", "value": res["mlups"], "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_gradient"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 reductions)",
            "data": "synthetic (seeded)",
            "config": {"workload": res["workload"], "nodes": res["nodes"], "tiles": res["tiles"],
                       "autotune_s": res["autotune_s"], "staging": res["staging"], "l2": "inputs larger than L2"},
            "roofline": res["roofline"],
            "per_problem_grad_rel_err_fp32_vs_oracle": res["per_problem_grad_rel_err_fp32_vs_oracle"],
            "clocks": clk, "e2e": None,
            # per gradient: N forward + one final per problem + finalize, zero sigma, S-2 Phi restores,
            # N-k recompute, N adjoint, finalize
            "gpu_launches": res["gpu_launches"],
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_warmstart(args, rank, world, local):
    """Learned warm start against the plain method on held-out problems.

    Data: args.ws_train seeded problems solved by the plain batched Armijo
    descent from g = 0 to convergence (warmstart.descend); the
    U-Net is trained on (inputs, g*) with the library's BF16 kernels.  On
    args.ws_test held-out problems the plain run from g = 0 defines J*; then
    the warm start (U-Net proposal + descent) and the cold start (descent from
    g = 0) are timed until each problem's cost is <= J* (1 + 1e-6).
    """
    import numpy as np
    import torch

    if rank != 0:  # independent replicas only; rank 0 reports
        return
    torch.cuda.set_device(local)
    from paper_1908_03876_gb300.build import build

    build()
    from paper_1908_03876_gb300 import warmstart as WS

    def log(m):
        print(m, file=sys.stderr, flush=True)

    size, N, win = args.ws_size, args.ws_steps, 8
    k = max(8, N // 4)
    if args.profile:  # three U-Net training steps on random inputs of --ws-size (profiling case)
        model = WS.Surrogate()
        x = torch.randn((16, 6, size, size), device="cuda").to(torch.bfloat16)
        t = torch.randn((16, 1, size, size), device="cuda")
        for _ in range(3):
            model.net.train_step(x, t)
        torch.cuda.synchronize()
        print(json.dumps({"profile": f"U-Net training steps, batch 16, {size}x{size}"}))
        return
    t0 = time.perf_counter()
    train = WS.problems(args.ws_train, 10_000, size=size, N=N, windows=win, ckpt_every=k)
    test = WS.problems(args.ws_test, 900_000, size=size, N=N, windows=win, ckpt_every=k)
    ref_tr = WS.descend(train, max_iter=200, log=log, want_residual=True)
    t_data = time.perf_counter() - t0
    log(f"data: {t_data:.1f} s, iterations mean {ref_tr['iters'].mean():.1f}")
    X = WS.features(train)
    D = np.stack([r - r0 for r, r0 in zip(ref_tr["residual"], ref_tr["residual_init"])])
    model = WS.Surrogate()
    bs = 16
    steps_per_epoch = len(X) // bs
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t1 = time.perf_counter()
    e0.record()
    losses = model.fit(X, np.stack(ref_tr["residual_init"]), D, epochs=args.ws_epochs, batch_size=bs, lr=2e-3,
                       log=log)
    e1.record()
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    train_ms = e0.elapsed_time(e1)
    flops = model.net.flops(bs, size, size) * steps_per_epoch * args.ws_epochs
    tf = flops / (train_ms * 1e-3) / 1e12
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        peak, pk_kind = float(pk["bf16_tflops_sustained"]), "measured (sustained bf16)"
    except Exception:
        peak, pk_kind = 1700.0, "fallback"
    ref_te = WS.descend(test, max_iter=200, log=log, want_residual=True)
    clocks = Clocks()
    clocks.start()
    ev = WS.evaluate(model, test, ref_te, log=log)
    clk = clocks.stop(local)
    line = {
        "metric": "wall time to the plain optimum cost (1e-6 rel), learned warm start",
        "value": ev["warm_seconds"], "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 0,
        "ms_per_step": ev["warm_seconds"] * 1e3, "higher_is_better": False, "scaling": "replicas only",
        "vs_baseline": None, "dtype": "f32 lattice (FP64 reductions), bf16 U-Net (FP32 accumulation)",
        "data": "synthetic (seeded)",
        "config": {"workload": f"warm start: {args.ws_train} training + {args.ws_test} held-out problems, "
                               f"{size}x{size} D2Q9 FP32, {N} steps, control constant over {win} windows, "
                               "random chi, eigenvalue ratio and angle",
                   "alpha": train[0].alpha, "descent": "Armijo steepest descent, converged at ||E||/||E0|| < 1e-4 "
                   "or a relative J decrease < 1e-7 over 5 iterations, at most 200 iterations (J*); "
                   "timed runs stop at J <= J* (1 + 1e-6)",
                   "unet": "4 levels, 32-256 channels, additive skips; from (u0, chi, ratio, angle, r0) predicts d* = u^N(g*) - u^N(0), "
                           "proposal G0 = -S(0)^T (r0 + d_hat) / (2 alpha L) by one forward and one seeded AMRT sweep",
                   "epochs": args.ws_epochs,
                   "batch": bs, "l2": "batched lattices larger than L2"},
        "cold_seconds": ev["cold_seconds"], "speedup_vs_plain": ev["cold_seconds"] / ev["warm_seconds"],
        "eval": ev, "datagen_seconds": t_data, "train_seconds": t_train, "train_loss": losses[-1],
        "roofline": {"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                     "traffic": None, "kernel": "U-Net training (all convolution launches)",
                     "peak_source": pk_kind},
        "clocks": clk, "e2e": None,
    }
    print(json.dumps(line), flush=True)


def cg_block():
    """Nonlinear CG (Polak-Ribiere, Wolfe-Powell search) and steepest descent
    with the linearised (sensitivity) line search against Armijo steepest
    descent on one problem (256x256 D2Q9 FP32, 200 steps, control constant
    over 8 windows): wall time and iterations until J <= J* (1 + 1e-6),
    J* = the lowest cost any method reaches in its iteration budget."""
    import torch

    from paper_1908_03876_gb300 import workloads as W
    from paper_1908_03876_gb300._lib import CxError
    from paper_1908_03876_gb300.problem import Problem

    w = W.aniso(256, 256, 200, seed=1, precision=32, ckpt_every=50)
    w.windows = 8

    def run(method, n_iter, target=None):
        p = Problem(w)
        g = p.zeros_control()
        Js, t_hit, it_hit = [], None, None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(n_iter):
            try:
                info = p.cg_step(g, "PR") if method == "cg" else (p.lma_step(g) if method == "lma" else p.step(g))
            except CxError as e:  # no acceptable step: converged to the FP32 resolution of J
                if e.code != 6:
                    raise
                break
            Js.append(info["J"])
            if target is not None and info["J"] <= target:
                t_hit, it_hit = time.perf_counter() - t0, k + 1
                break
        torch.cuda.synchronize()
        p.close()
        return Js, t_hit, it_hit

    Jcg, _, _ = run("cg", 150)
    Jsd, _, _ = run("sd", 600)
    Jlm, _, _ = run("lma", 600)
    Jstar = min(min(Jcg), min(Jsd), min(Jlm))
    target = Jstar * (1 + 1e-6)
    _, t_cg, it_cg = run("cg", 150, target)
    _, t_sd, it_sd = run("sd", 600, target)
    _, t_lm, it_lm = run("lma", 600, target)
    return {"workload": "aniso 256x256 D2Q9 FP32, 200 steps, k = 50, control constant over 8 windows",
            "J_star": Jstar, "iteration_budgets": {"cg": 150, "steepest_descent": 600, "lma": 600},
            "cg_seconds": t_cg, "cg_iterations": it_cg, "steepest_descent_seconds": t_sd,
            "steepest_descent_iterations": it_sd, "lma_seconds": t_lm, "lma_iterations": it_lm,
            "speedup_vs_steepest_descent": None if (t_cg is None or t_sd is None) else t_sd / t_cg,
            "J_final": {"cg": Jcg[-1], "steepest_descent": Jsd[-1], "lma": Jlm[-1]}}


def run_cg(args, rank, world, local):
    """The CG comparison of cg_block as its own bench line."""
    import torch

    if rank != 0:
        return
    torch.cuda.set_device(local)
    from paper_1908_03876_gb300.build import build

    build()
    if args.profile:  # one forward, sensitivity pass and continuous adjoint (profiling case)
        from paper_1908_03876_gb300 import workloads as W
        from paper_1908_03876_gb300.problem import Problem

        w = W.aniso(256, 256, 200, seed=1, precision=32, ckpt_every=50)
        w.windows = 8
        p = Problem(w)
        g = p.zeros_control()
        p.forward(g)
        p.tlm(g, torch.ones_like(g))
        p.forward(g)
        p.cadjoint(g)
        torch.cuda.synchronize()
        print(json.dumps({"profile": "aniso 256x256, 200 steps: forward, sensitivity, continuous adjoint"}))
        return
    cg = cg_block()
    line = {
        "metric": "wall time to J* (1e-6 rel): nonlinear CG (Polak-Ribiere, Wolfe-Powell) vs Armijo steepest descent",
        "value": cg["cg_seconds"], "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 0,
        "ms_per_step": None if cg["cg_seconds"] is None else cg["cg_seconds"] * 1e3, "higher_is_better": False,
        "scaling": "replicas only", "vs_baseline": None, "dtype": "f32 (FP64 reductions)",
        "data": "synthetic (seeded)", "config": {"workload": cg["workload"]}, **cg,
    }
    print(json.dumps(line), flush=True)


def run_fp64(args, rank, world, local):
    """FP64 lattices on the GPU (not a target: the FP64 pipe of a GB300 is far
    narrower than its FP32 pipe): the 64x64 D2Q5 problem (L2-resident, time per
    step) and the 1024x1024 D2Q9 anisotropic problem for 200 steps, k = 20
    (fwd+adjoint MLUPS and the per-phase launch times, HBM fraction at FP64
    bytes); J of the small problem against the FP64 oracle."""
    import torch

    if rank != 0:
        return
    torch.cuda.set_device(local)
    from paper_1908_03876_gb300.build import build

    build()
    import oracle

    oracle.build()
    from paper_1908_03876_gb300 import workloads as W
    from paper_1908_03876_gb300.problem import Problem

    hbm, peak_kind = _peaks()
    out = {}
    for name, w, reps in [("plain64 (64x64 D2Q5, N=200)", W.plain64(), 20),
                          ("aniso1024 (1024x1024 D2Q9, N=200, k=20)",
                           W.aniso(1024, 1024, 200, seed=1, precision=64, ckpt_every=20), 3)]:
        p = Problem(w)
        g = torch.as_tensor(w.random_control(100, 0.01), dtype=torch.float64, device="cuda").contiguous()
        E = torch.empty_like(g)
        for _ in range(2):
            p.gradient(g, out=E)
        torch.cuda.synchronize()
        p.set_timing(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(p.stream)
        for _ in range(reps):
            J, _ = p.gradient(g, out=E)
        e1.record(p.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        phases = p.timing()
        p.set_timing(False)
        nodes = w.nx * w.ny
        ent = {"ms_per_gradient": ms, "us_per_step": ms * 1e3 / w.N, "mlups": nodes * w.N / (ms * 1e-3) / 1e6}
        if w.Q == 9:
            for ph in ("forward", "recompute", "adjoint"):
                t, n = phases[ph]
                if n > 0:
                    us = t * 1e3 / n
                    gbs = 2 * BYTES[ph] * nodes / (us * 1e-6) / 1e9
                    ent[ph] = {"us_per_launch": us, "GB/s (FP64 bytes)": gbs, "hbm_frac": gbs / hbm}
        if nodes <= 4096:  # the oracle's J for the small problem (the large one is checked by the tests)
            Jo, _, _ = oracle.forward(oracle.from_workload(w), g.cpu().numpy())
            ent["J_rel_err_vs_oracle"] = abs(float(J.item()) - Jo) / abs(Jo)
        out[name] = ent
        p.close()
    line = {"metric": "FP64 lattices: fwd+adjoint MLUPS", "value": out["aniso1024 (1024x1024 D2Q9, N=200, k=20)"]["mlups"],
            "unit": "MLUPS", "n_gpus": 1, "higher_is_better": True, "dtype": "f64", "data": "synthetic (seeded)",
            "peak_hbm_gbs": hbm, "peak_source": peak_kind, "results": out}
    print(json.dumps(line), flush=True)


# algorithmic bytes per node and step of the three-species kernels (FP32, D2Q9):
#   forward   27 pulls + 27 stores (216) + angle (4) + g (4) + Phi in/out for 3 species (24) = 248
#   recompute forward + tape (u, v, G_v, G_w) store (24)                                       = 272
#   adjoint   216 + tape read (24) + angle (4) + sigma in/out (24) + g (4) + dJ/dg (4)         = 276
BYTES3 = dict(forward=248, recompute=272, adjoint=276)


def run_arc(args, rank, world, local):
    """Three-species attraction-repulsion chemotaxis (logistic source) on the
    1024x1024 D2Q9 FP32 lattice, 2000 steps, checkpoint every 100: gradient
    evaluations (forward + recompute + exact discrete adjoint) with per-phase
    kernel times and HBM fractions, FP32 error against the FP64 oracle on a
    reduced-size run, and the CPU oracle on a bounded sample."""
    import numpy as np
    import torch

    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1908_03876_gb300.build import build

    build()
    from paper_1908_03876_gb300 import workloads as W
    from paper_1908_03876_gb300.arc import ArcProblem

    nx = ny = 1024
    N, k = (20, 10) if args.profile else (2000, 100)  # profiling case: the full grid, 20 steps (about 1.3 GB)
    w = W.arc(nx, ny, N, seed=5, precision=32, ckpt_every=k)
    p = ArcProblem(w, device=dev)
    g = torch.as_tensor(w.random_control(100, 0.01), dtype=torch.float32, device=dev).contiguous()
    E = torch.empty_like(g)
    for _ in range(args.warmup):
        p.gradient(g, out=E)
    torch.cuda.synchronize()
    if args.profile:
        print(json.dumps({"profile": f"arc {nx}x{ny}, {N} steps: gradient evaluations"}))
        return
    clocks = Clocks()
    clocks.start()
    p.set_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(p.stream)
    for _ in range(args.steps):
        p.gradient(g, out=E)
    e1.record(p.stream)
    torch.cuda.synchronize()
    clk = clocks.stop(local)
    ms = e0.elapsed_time(e1) / args.steps
    phases = p.timing()
    p.set_timing(False)
    J, gsq, _ = p.norms()
    nodes = nx * ny
    hbm, peak_kind = _peaks()
    kern = {}
    for ph in ("forward", "recompute", "adjoint"):
        t, n = phases[ph]
        if n > 0:
            us = t * 1e3 / n
            ach = BYTES3[ph] * nodes / (us * 1e-6) / 1e9
            kern[ph] = {"us_per_launch": us, "achieved": ach, "frac": ach / hbm, "launches": n,
                        "bytes_per_node": BYTES3[ph]}
    dom = max(kern, key=lambda q: kern[q]["us_per_launch"] * kern[q]["launches"])
    kname = {"forward": "k3_forward_rows", "recompute": "k3_forward_rows", "adjoint": "k3_adjoint"}[dom]
    roof = {"bound": "hbm", "achieved": kern[dom]["achieved"], "peak": hbm, "unit": "GB/s",
            "frac": kern[dom]["frac"], "traffic": _traffic(kname), "kernel": kname, "peak_source": peak_kind,
            "bytes_per_launch": BYTES3[dom] * nodes}
    # FP32 against the FP64 oracle at the same horizon on a 64x64 grid
    err = None
    try:
        import oracle

        oracle.build()
        ws = W.arc(64, 64, N, seed=5, precision=32, ckpt_every=k)
        ps = ArcProblem(ws, device=dev)
        gs = ws.random_control(101, 0.01)
        Js, Es = ps.gradient(gs)
        fs = [t.cpu().numpy() for t in ps.fields()]
        po = oracle.from_workload3(ws)
        Jo, uvw = oracle.forward3(po, gs)
        _, Eo, _ = oracle.adjoint3(po, gs)
        rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
        err = {"grid": "64x64", "steps": N, "u": rel(fs[0], uvw[0]), "v": rel(fs[1], uvw[1]), "w": rel(fs[2], uvw[2]),
               "dJdg": rel(Es.cpu().numpy(), Eo), "J": abs(float(Js.item()) - Jo) / abs(Jo)}
        ps.close()
    except Exception as exc:
        err = {"error": str(exc)[:200]}
    line = {"metric": "fwd+adjoint MLUPS (three species)", "value": nodes * N / (ms * 1e-3) / 1e6, "unit": "MLUPS",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "replicas only", "vs_baseline": None, "dtype": "f32 (FP64 reductions)",
            "data": "synthetic (seeded)",
            "config": {"workload": f"arc{nx}: {nx}x{ny} D2Q9 FP32, three species (attraction to v, repulsion "
                                   f"from w, logistic growth), {N} steps, checkpoint every {k}",
                       "step": "one gradient evaluation (forward + recompute + exact discrete adjoint)",
                       "l2": "inputs larger than L2 (8.4 GB control per step)"},
            "roofline": roof, "kernels": kern, "fp32_err_vs_oracle": err, "clocks": clk,
            "gpu_launches": (3 * N - k + 3) * args.steps, "J": J, "grad_norm": float(np.sqrt(gsq))}
    print(json.dumps(line), flush=True)


# algorithmic bytes per node and step of the D3Q19 kernels (FP32, two species):
#   forward   38 pulls + 38 stores (304) + g (4) + Phi in/out (8)                       = 316
#   recompute forward + tape (u, G_x, G_y, G_z) store (16)                               = 332
#   adjoint   304 + tape read (16) + sigma in/out (8) + g (4) + dJ/dg (4)                = 336
BYTES3D = dict(forward=316, recompute=332, adjoint=336)


def run_d3q19(args, rank, world, local):
    """The two-species problem on a 128^3 D3Q19 lattice (FP32, 500 steps,
    checkpoint every 50, constant rotated tensors, shear convection):
    gradient evaluations with per-phase kernel times and HBM fractions, and
    the FP32 error against the FP64 oracle on a 24^3 run of the same physics."""
    import numpy as np
    import torch

    if rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1908_03876_gb300.build import build

    build()
    from paper_1908_03876_gb300 import workloads as W
    from paper_1908_03876_gb300.d3 import D3Problem

    n = 128
    N, k = (10, 5) if args.profile else (500, 50)
    w = W.aniso3d(n, N, seed=6, precision=32, ckpt_every=k)
    p = D3Problem(w, device=dev)
    g = torch.as_tensor(w.random_control(100, 0.01), dtype=torch.float32, device=dev).contiguous()
    E = torch.empty_like(g)
    for _ in range(args.warmup):
        p.gradient(g, out=E)
    torch.cuda.synchronize()
    if args.profile:
        print(json.dumps({"profile": f"d3q19 {n}^3, {N} steps: gradient evaluations"}))
        return
    clocks = Clocks()
    clocks.start()
    p.set_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(p.stream)
    for _ in range(args.steps):
        p.gradient(g, out=E)
    e1.record(p.stream)
    torch.cuda.synchronize()
    clk = clocks.stop(local)
    ms = e0.elapsed_time(e1) / args.steps
    phases = p.timing()
    p.set_timing(False)
    J, gsq, _ = p.norms()
    nodes = n ** 3
    hbm, peak_kind = _peaks()
    kern = {}
    for ph in ("forward", "recompute", "adjoint"):
        t, c = phases[ph]
        if c > 0:
            us = t * 1e3 / c
            ach = BYTES3D[ph] * nodes / (us * 1e-6) / 1e9
            kern[ph] = {"us_per_launch": us, "achieved": ach, "frac": ach / hbm, "launches": c,
                        "bytes_per_node": BYTES3D[ph]}
    dom = max(kern, key=lambda q: kern[q]["us_per_launch"] * kern[q]["launches"])
    kname = {"forward": "k3d_forward", "recompute": "k3d_forward", "adjoint": "k3d_adjoint"}[dom]
    roof = {"bound": "hbm", "achieved": kern[dom]["achieved"], "peak": hbm, "unit": "GB/s",
            "frac": kern[dom]["frac"], "traffic": _traffic(kname), "kernel": kname, "peak_source": peak_kind,
            "bytes_per_launch": BYTES3D[dom] * nodes}
    err = None
    try:
        import oracle

        oracle.build()
        ws = W.aniso3d(24, 100, seed=6, precision=32, ckpt_every=25)
        ps = D3Problem(ws, device=dev)
        gs = ws.random_control(101, 0.01)
        Js, Es = ps.gradient(gs)
        us, vs = (t.cpu().numpy() for t in ps.fields())
        po = oracle.from_workload3d(ws)
        Jo, uo, vo = oracle.forward3d(po, gs)
        _, Eo, _ = oracle.adjoint3d(po, gs)
        rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
        err = {"grid": "24^3", "steps": 100, "u": rel(us, uo), "v": rel(vs, vo), "dJdg": rel(Es.cpu().numpy(), Eo),
               "J": abs(float(Js.item()) - Jo) / abs(Jo)}
        ps.close()
    except Exception as exc:
        err = {"error": str(exc)[:200]}
    line = {"metric": "fwd+adjoint MLUPS (D3Q19)", "value": nodes * N / (ms * 1e-3) / 1e6, "unit": "MLUPS",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "replicas only", "vs_baseline": None, "dtype": "f32 (FP64 reductions)",
            "data": "synthetic (seeded)",
            "config": {"workload": f"aniso3d{n}: {n}^3 D3Q19 FP32, two species, {N} steps, checkpoint every {k}, "
                                   "rotated constant tensors, shear convection, chi = -0.1",
                       "step": "one gradient evaluation (forward + recompute + exact discrete adjoint)",
                       "l2": "inputs larger than L2 (4.2 GB control per step)"},
            "roofline": roof, "kernels": kern, "fp32_err_vs_oracle": err, "clocks": clk,
            "gpu_launches": (3 * N - k + 3) * args.steps, "J": J, "grad_norm": float(np.sqrt(gsq))}
    print(json.dumps(line), flush=True)


def run_unet_layers(args, rank, world, local):
    """Forward time of each 3x3 layer shape of the 4-level U-Net at 128x128,
    batch 16, on the tcgen05 kernel and on the mma.sync kernel (same packed
    weights; CUDA events, 20 launches after 3 warm-up launches)."""
    import ctypes

    import torch

    if rank != 0:
        return
    torch.cuda.set_device(local)
    from paper_1908_03876_gb300.build import build

    build()
    from paper_1908_03876_gb300 import _lib

    lib = _lib.load()
    BF = torch.bfloat16

    def p(t):
        return ctypes.c_void_p(t.data_ptr())

    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    shapes = [(6, 32, 128), (32, 32, 128), (32, 64, 64), (64, 64, 64), (64, 128, 32), (128, 128, 32),
              (128, 256, 16), (256, 256, 16), (256, 128, 32), (128, 64, 64), (64, 32, 128)]
    B = 16
    out = []
    for cin, cout, hw in shapes:
        x = torch.randn(B, cin, hw, hw, device="cuda").to(BF)
        w = (0.05 * torch.randn(cout, cin, 3, 3, device="cuda")).to(BF)
        wf = torch.empty(lib.cx_nn_packed_weights(cout, cin, 3, 0), dtype=BF, device="cuda")
        wb = torch.empty(lib.cx_nn_packed_weights(cout, cin, 3, 1), dtype=BF, device="cuda")
        _lib.check(lib.cx_nn_pack_weights(p(w), cout, cin, 3, p(wf), p(wb), s), "pack")
        bias = torch.zeros(cout, device="cuda")
        y = torch.empty(B, cout, hw, hw, dtype=BF, device="cuda")
        yf = torch.empty(B, cout, hw, hw, dtype=torch.float32, device="cuda")
        res = {}
        for name, fn in (("tcgen05", lambda: lib.cx_nn_conv_forward_tc(p(x), p(wf), p(bias), p(y), B, cin, cout, hw,
                                                                         hw, 3, 1, None, s)),
                         ("mma_sync", lambda: lib.cx_nn_conv_forward_f32(p(x), p(wf), p(bias), p(yf), B, cin, cout,
                                                                          hw, hw, 3, s))):
            for _ in range(3):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(20):
                fn()
            e1.record()
            torch.cuda.synchronize()
            res[name] = e0.elapsed_time(e1) / 20 * 1e3
        # weight gradient of the same layer (dY random), both kernels, the splits the surrogate uses
        dy = torch.randn(B, cout, hw, hw, device="cuda").to(BF)
        wg = {}
        ntiles = B * ((hw + 7) // 8) ** 2
        for name, base in (("wgrad_tcgen05", ((cin + 15) // 16) * ((cout + 127) // 128)),
                           ("wgrad_mma_sync", ((cin + 15) // 16) * ((cout + 63) // 64))):
            splits = int(max(1, min(ntiles, -(-304 // base))))
            scr = torch.empty(lib.cx_nn_conv_backward_weight_scratch(B, cin, cout, hw, hw, 3, splits) // 4 + 1,
                              device="cuda")
            dw = torch.empty(cout, cin, 3, 3, device="cuda")
            db = torch.empty(cout, device="cuda")
            if name == "wgrad_tcgen05":
                fn = lambda: lib.cx_nn_conv_backward_weight_tc(p(x), p(dy), p(dw), p(db), p(scr), splits, B, cin,
                                                               cout, hw, hw, 3, None, s)
            else:
                fn = lambda: lib.cx_nn_conv_backward_weight(p(x), p(dy), p(dw), p(db), p(scr), splits, B, cin, cout,
                                                            hw, hw, 3, s)
            for _ in range(3):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(20):
                fn()
            e1.record()
            torch.cuda.synchronize()
            wg[name] = e0.elapsed_time(e1) / 20 * 1e3
        res.update(wg)
        fl = 2 * B * hw * hw * cout * cin * 9
        out.append({"layer": f"{cin}->{cout}@{hw}", **{k + "_us": round(v, 1) for k, v in res.items()},
                    **{k + "_tflops": round(fl / v / 1e6, 1) for k, v in res.items()}})
    print(json.dumps({"unet_layers": out}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="aniso1024",
                    choices=["aniso1024", "batch", "warmstart", "cg", "unetlayers", "fp64", "geometry4096", "arc", "d3q19"],
                    help="aniso1024 (default bench line) or batch: 256 independent problems, sizes {64..512}^2, "
                         "1000 steps, one persistent launch per step replayed as a CUDA graph")
    ap.add_argument("--staging", default=None, choices=["rows", "thread"],
                    help="bulk row-window staging or per-thread copies (default: rows for aniso1024, "
                         "thread for batch, the faster of each)")
    ap.add_argument("--threads", type=int, default=256, choices=[128, 256],
                    help="aniso1024: threads per block of the persistent lattice kernels")
    ap.add_argument("--problems", type=int, default=256)
    ap.add_argument("--ws-train", type=int, default=2000)
    ap.add_argument("--ws-test", type=int, default=200)
    ap.add_argument("--ws-size", type=int, default=256)
    ap.add_argument("--no-cg", action="store_true", help="leave the CG comparison out of the default bench line")
    ap.add_argument("--no-batch", action="store_true",
                    help="leave the batched workload (256 problems) out of the default bench line")
    ap.add_argument("--opt-iters", type=int, default=20,
                    help="Armijo steepest-descent iterations of the default workload's optimisation leg (0: skip)")
    ap.add_argument("--ws-steps", type=int, default=256)
    ap.add_argument("--ws-epochs", type=int, default=40)
    ap.add_argument("--profile", action="store_true",
                    help="small profiling case: the same lattices (batch: --problems of them), 20 time steps, "
                         "k = 10, one warm-up and one timed gradient evaluation, no CPU baseline or e2e leg")
    args = ap.parse_args()
    if args.profile:
        WORKLOAD.update(N=20, k=10)
        args.steps, args.warmup, args.no_cpu_baseline = 1, 1, True

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batch":
        run_batch(args, rank, world, local)
        return
    if args.workload == "warmstart":
        run_warmstart(args, rank, world, local)
        return
    if args.workload == "cg":
        run_cg(args, rank, world, local)
        return
    if args.workload == "fp64":
        return run_fp64(args, rank, world, local)
    if args.workload == "arc":
        run_arc(args, rank, world, local)
        return
    if args.workload == "d3q19":
        run_d3q19(args, rank, world, local)
        return
    if args.workload == "unetlayers":
        run_unet_layers(args, rank, world, local)
        return
    if args.workload == "geometry4096":
        if rank != 0:
            return
        import torch

        torch.cuda.set_device(local)
        from paper_1908_03876_gb300.build import build

        build()
        geo = geometry_block(torch.device("cuda", local), args.staging or "rows", steps=args.steps,
                             warmup=args.warmup, size=2048 if args.profile else 4096)
        print(json.dumps({"metric": "fluid MLUPS (complex geometry)", "value": geo["fluid_mlups"], "unit": "MLUPS",
                          "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                          "geometry4096": geo}), flush=True)
        return

    import numpy as np
    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1908_03876_gb300.build import build

    if rank == 0:
        build()
    if dist:
        dist.barrier()
    from paper_1908_03876_gb300 import workloads as W
    from paper_1908_03876_gb300.problem import Problem

    wl = WORKLOAD
    w = W.aniso(wl["nx"], wl["ny"], wl["N"], seed=1 + rank, precision=32, ckpt_every=wl["k"])
    prob = Problem(w, device=dev)
    args.staging = args.staging or "rows"
    prob.set_staging(args.staging == "rows")
    if args.threads != 256:
        prob.set_launch(args.threads, 0)
    g = torch.as_tensor(w.random_control(100 + rank, 0.01), dtype=torch.float32, device=dev).contiguous()
    E = torch.empty_like(g)
    nodes = w.nx * w.ny

    def grad_step():
        prob.gradient(g, out=E)

    for _ in range(args.warmup):
        grad_step()
    torch.cuda.synchronize()

    # ---- timed region (device events on the problem's stream)
    clocks = Clocks()
    if rank == 0:
        clocks.start()
    prob.set_timing(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    stream = prob.stream
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        grad_step()
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms_total = ev0.elapsed_time(ev1)
    phases = prob.timing()
    prob.set_timing(False)
    J, gsq, ginf = prob.norms()
    clk = clocks.stop(local) if rank == 0 else None
    t = torch.tensor([ms_total], dtype=torch.float64, device=dev)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_step = float(t.item()) / args.steps
    mlups = world * nodes * w.N / (ms_step * 1e-3) / 1e6

    # ---- roofline of the kernels, from the same timed region
    hbm, peak_kind = _peaks()
    roof = {}
    for ph in ("forward", "recompute", "adjoint"):
        ms, launches = phases[ph]
        if launches <= 0:
            continue
        per_launch_s = ms * 1e-3 / launches
        traffic = BYTES[ph] * nodes
        ach = traffic / per_launch_s / 1e9
        roof[ph] = {"achieved": ach, "frac": ach / hbm, "ms_total": ms, "launches": launches,
                    "us_per_launch": per_launch_s * 1e6, "bytes_per_node": BYTES[ph]}
    dom = max(roof, key=lambda k: roof[k]["ms_total"]) if roof else "forward"
    if args.staging == "rows":
        kern = {"forward": "k_forward_rows", "recompute": "k_forward_rows (tape)", "adjoint": "k_adjoint_rows"}[dom]
    else:
        kern = {"forward": "k_forward", "recompute": "k_forward (tape)", "adjoint": "k_adjoint"}[dom]
    roofline = {"bound": "hbm", "achieved": roof[dom]["achieved"], "peak": hbm, "unit": "GB/s",
                "frac": roof[dom]["frac"], "traffic": _traffic(kern.split()[0]), "kernel": kern,
                "peak_source": peak_kind, "bytes_per_launch": BYTES[dom] * nodes}

    # ---- end to end: host control in, host gradient and cost out, every step
    e2e = None
    if rank == 0 and not args.profile:
        try:
            g_host = torch.empty(g.shape, dtype=g.dtype, pin_memory=True)
            g_host.copy_(g.cpu())
            E_host = torch.empty_like(g_host, pin_memory=True)
            torch.cuda.synchronize()
            # the host link as this process sees it (the whole pinned buffers,
            # one copy each way, alone), so that a slow link shows beside the
            # figure: the rate of these buffers' pages can differ from a short
            # probe's
            link = {}
            for name, dst, src in (("h2d_gbs", g, g_host), ("d2h_gbs", E_host, E)):
                la, lb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                la.record()
                dst.copy_(src, non_blocking=True)
                lb.record()
                torch.cuda.synchronize()
                link[name] = g.numel() * g.element_size() / (la.elapsed_time(lb) * 1e-3) / 1e9
            g.copy_(g_host, non_blocking=True)
            torch.cuda.synchronize()
            # Every step goes through the C ABI's host-buffer call
            # (cx_gradient_host): the control is copied in chunk by chunk, each
            # forward step waiting only for its own chunk, and the gradient
            # leaves chunk by chunk during the reverse sweep; the call returns
            # with J and dJ/dg in host memory.
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ne = max(1, args.steps)
            ea.record(stream)
            for _ in range(ne):
                prob.gradient_host(g_host, E_host, g, E)
            eb.record(stream)
            torch.cuda.synchronize()
            ms_e2e = ea.elapsed_time(eb) / ne
            e2e = {"value": nodes * w.N / (ms_e2e * 1e-3) / 1e6, "unit": "MLUPS",
                   "h2d_bytes_per_step": g.numel() * g.element_size(),
                   "d2h_bytes_per_step": E.numel() * E.element_size() + 36, "ms_per_step": ms_e2e,
                   "call": "cx_gradient_host (host control in, host gradient and cost out)",
                   "host_link": {k: round(v, 1) for k, v in link.items()},
                   "overlap": "control copied in 32 chunks, each forward step waiting for its own chunk; "
                              "gradient chunks read back during the reverse sweep"}
        except Exception as exc:  # pinned memory can fail on small hosts
            e2e = {"value": None, "unit": "MLUPS", "error": str(exc)[:200]}

    # ---- the optimisation leg of the same workload: plain steepest descent
    # from g = 0 with the Armijo rule (one gradient and >= 1 trial forward
    # solves per iteration), timed on the problem's stream
    opt = None
    if rank == 0 and not args.profile and args.opt_iters > 0:
        g.zero_()
        oa, ob = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        oa.record(stream)
        its = [prob.step(g, E) for _ in range(args.opt_iters)]
        ob.record(stream)
        torch.cuda.synchronize()
        trials = sum(it["trials"] for it in its)
        sec = oa.elapsed_time(ob) * 1e-3
        opt = {"iterations": len(its), "J0": its[0]["J0"], "J": its[-1]["J"],
               "J_ratio": its[-1]["J"] / its[0]["J0"], "trial_forward_solves": trials,
               "grad_norm_ratio": float(np.sqrt(its[-1]["grad_sq"] / its[0]["grad_sq"])),
               "seconds": sec, "ms_per_iteration": sec * 1e3 / len(its),
               "J_per_iteration": [it["J"] for it in its]}

    launches_per_step = 3 * w.N - wl["k"] + 3
    if rank == 0:
        def guarded(fn, *a):  # a block that fails reports its error; the bench line still prints
            try:
                return fn(*a)
            except Exception as exc:
                return {"error": str(exc)[:200]}

        cpu = None if args.no_cpu_baseline else guarded(cpu_baseline)
        fp32_err = None if args.profile else guarded(fp32_error_vs_oracle, dev)
        geom = None if args.profile else guarded(geometry_block, dev, args.staging)
        bb = None
        if not args.profile and not args.no_batch:
            try:
                bb = batch_block(dev)
            except Exception as exc:
                bb = {"error": str(exc)[:200]}
        cgb = None
        if not args.profile and not args.no_cg:
            try:
                cgb = cg_block()
            except Exception as exc:
                cgb = {"error": str(exc)[:200]}
        line = {
            "metric": "fwd+adjoint MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (FP64 reductions)", "data": "synthetic (seeded)",
            "config": {"workload": "aniso1024: 1024x1024 D2Q9 FP32, 2000 steps, checkpoint every 100, "
                                   "rotated anisotropic D_u = D_v, shear convection, chemotaxis chi=-0.1",
                       "step": "one gradient evaluation (forward + recompute + AMRT adjoint + FP64 reductions)",
                       "l2": "inputs larger than L2 (8.4 GB control, 1.5 GB checkpoints per step)",
                       "staging": args.staging, "threads_per_block": args.threads,
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline,
            "kernels": roof,
            "cpu_baseline": cpu,
            "fp32_err_vs_oracle": fp32_err,
            "geometry4096": geom,
            "optimise": opt,
            "cg256": cgb,
            "batch256": bb,
            "clocks": clk,
            "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps,
            "J": J, "grad_norm": float(np.sqrt(gsq)),
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
