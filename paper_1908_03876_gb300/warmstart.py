"""Learned warm start for the optimal-control problem.

The paper's method (Sec. 3.2.1: forward MRT solve, AMRT adjoint, gradient,
Armijo step) solves each control problem from g = 0.  Here a U-Net
(surrogate.UNet) trained on optimal controls that the method itself computed
proposes g0 for a new problem, and the same gradient descent refines it.
Plain descent from g = 0 stays the fallback and the judge: the warm-started
run counts as done when its cost reaches the plain optimum J* to within a
relative 1e-6.

Problems: square periodic D2Q9 grids with constant rotated anisotropic
tensors (random eigenvalue ratio and angle), random chemotactic sensitivity,
seeded initial bumps u0 and a fixed centred target; the control acts on v
everywhere and is piecewise constant over W time windows (the network's W
output channels).  Network inputs per node: u0, chi, lambda2/lambda1,
cos 2 theta, sin 2 theta.

All solves run batched (batch.Batch: one persistent launch per time step
over every problem, captured graphs, one batched Armijo trial per
line-search round); problems that are done are switched off and cost no
lattice work.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import workloads as W
from .batch import Batch
from .surrogate import UNet


def problems(n, seed0, size=128, N=200, windows=8, ckpt_every=50, precision=32):
    """n seeded problems (seeds seed0 .. seed0 + n - 1)."""
    out = []
    for i in range(n):
        seed = seed0 + i
        rng = np.random.default_rng(seed)
        chi = -float(rng.uniform(0.2, 2.0)) / 20.0
        ratio = float(rng.uniform(1.0, 8.0))
        ang = float(rng.uniform(0.0, np.pi))
        sig = size / 16.0
        u0 = W.bumps(size, size, seed, sig)
        u_tgt = 1.0 + 0.2 * W._periodic_gauss(size, size, size / 2, size / 2, 2 * sig)
        lam = (0.08, 0.08 / ratio)
        out.append(W.Workload(name=f"ws{seed}", nx=size, ny=size, N=N, Q=9, precision=precision,
                              aniso="rotated", lam_u=lam, lam_v=lam, theta=np.full((size, size), ang), chi=chi,
                              u0=u0, v0=np.zeros((size, size)), u_tgt=u_tgt, alpha=1e-3,
                              ckpt_every=ckpt_every, windows=windows,
                              extra=dict(ratio=ratio, angle=ang, seed=seed)))
    return out


def features(ws):
    """U-Net inputs [n, 5, ny, nx] (float32): scaled u0, chi, 1/ratio, cos 2t, sin 2t."""
    X = np.zeros((len(ws), 5, ws[0].ny, ws[0].nx), dtype=np.float32)
    for i, w in enumerate(ws):
        X[i, 0] = (w.u0 - 1.0) / 0.2
        X[i, 1] = -20.0 * w.chi
        X[i, 2] = 1.0 / w.extra["ratio"]
        X[i, 3] = np.cos(2 * w.extra["angle"])
        X[i, 4] = np.sin(2 * w.extra["angle"])
    return X


def descend(ws, g0=None, max_iter=200, grad_tol=1e-4, J_target=None, device="cuda", chunk=256, log=None):
    """Batched Armijo gradient descent (the paper's algorithm) on every
    problem from g0 (list of arrays, None: zero controls).

    A problem stops when ||E|| / ||E_0|| < grad_tol (E_0: its gradient at the
    start), or, when J_target is given, as soon as its cost is <= J_target[i]
    (the cost is checked at the start and after every accepted step), or
    after max_iter steps.  Returns dict(g, J, iters, reached, seconds,
    history) where seconds is the wall time of the descent (device work,
    synchronised) and history[i] lists J after each step.
    """
    n = len(ws)
    g_out = [None] * n
    J_out = np.zeros(n)
    J_init = np.full(n, np.nan)
    iters = np.zeros(n, dtype=np.int64)
    reached = np.zeros(n, dtype=bool)
    history = [[] for _ in range(n)]
    seconds = 0.0
    for c0 in range(0, n, chunk):
        idx = list(range(c0, min(n, c0 + chunk)))
        b = Batch([ws[i] for i in idx], device=device)
        if g0 is None:
            gs = b.zeros_controls()
        else:
            gs = [torch.as_tensor(np.asarray(g0[i]), dtype=b.dtype, device=b.device).contiguous() for i in idx]
        b.bind(gs)
        active = np.ones(len(idx), dtype=bool)
        e0 = np.full(len(idx), np.nan)
        torch.cuda.synchronize(b.device)
        t0 = time.perf_counter()
        if J_target is not None:
            Jc = b.forward().cpu().numpy()
            for k, i in enumerate(idx):
                J_out[i] = J_init[i] = Jc[k]
                if Jc[k] <= J_target[i]:
                    active[k] = False
                    reached[i] = True
            b.set_enabled(active)
        for it in range(max_iter):
            if not active.any():
                break
            info, st = b.step()
            for k, i in enumerate(idx):
                if not active[k]:
                    continue
                if st[k] != 0:  # line search failed or non-finite: stop this problem
                    active[k] = False
                    continue
                if np.isnan(e0[k]):
                    e0[k] = np.sqrt(info[k]["grad_sq"])
                    J_init[i] = info[k]["J0"]
                iters[i] += 1
                J_out[i] = info[k]["J"]
                history[i].append(info[k]["J"])
                if J_target is not None:
                    if info[k]["J"] <= J_target[i]:
                        active[k] = False
                        reached[i] = True
                elif e0[k] > 0 and np.sqrt(info[k]["grad_sq"]) < grad_tol * e0[k]:
                    active[k] = False
                    reached[i] = True
            b.set_enabled(active)
            if log and it % 20 == 0:
                log(f"  descend chunk {c0}: it {it} active {int(active.sum())}")
        torch.cuda.synchronize(b.device)
        seconds += time.perf_counter() - t0
        for k, i in enumerate(idx):
            g_out[i] = gs[k].detach().cpu().numpy()
        b.close()
        del b
    return dict(g=g_out, J=J_out, J_init=J_init, iters=iters, reached=reached, seconds=seconds, history=history)


class Surrogate:
    """U-Net proposal of the windowed control from a problem's inputs."""

    def __init__(self, windows=8, chans=(32, 64, 128, 256), seed=0, device="cuda"):
        self.net = UNet(cin=5, cout=windows, chans=chans, seed=seed, device=device)
        self.device = self.net.device
        self.scale = 1.0

    def fit(self, X, G, epochs=30, batch_size=16, lr=2e-3, seed=0, log=None):
        """Train on inputs X [n, 5, H, W] and optimal controls G [n, W, H, W].
        Returns the per-epoch mean training loss (on the scaled targets)."""
        self.scale = float(np.sqrt(np.mean(np.square(G)))) or 1.0
        Xd = torch.as_tensor(X, dtype=torch.bfloat16, device=self.device)
        Yd = torch.as_tensor(G / self.scale, dtype=torch.float32, device=self.device)
        rng = np.random.default_rng(seed)
        n = len(X)
        losses = []
        step = 0
        total = epochs * max(1, n // batch_size)
        for ep in range(epochs):
            perm = rng.permutation(n)
            acc = []
            for s in range(0, n - batch_size + 1, batch_size):
                sel = torch.as_tensor(perm[s:s + batch_size], device=self.device)
                # cosine decay of the learning rate
                lr_t = 0.5 * lr * (1 + np.cos(np.pi * step / total))
                loss = self.net.train_step(Xd[sel].contiguous(), Yd[sel].contiguous(), lr=lr_t)
                acc.append(loss)
                step += 1
            ep_loss = float(torch.cat(acc).mean()) if acc else float("nan")
            losses.append(ep_loss)
            if log:
                log(f"  epoch {ep}: loss {ep_loss:.4e}")
        return losses

    def propose(self, X, batch_size=32):
        """g0 [n, W, H, W] (float32, unscaled) for inputs X."""
        out = []
        for s in range(0, len(X), batch_size):
            x = torch.as_tensor(X[s:s + batch_size], dtype=torch.bfloat16, device=self.device)
            y = self.net.forward(x)
            out.append(y.float() * self.scale)
        return torch.cat(out).cpu().numpy()


def evaluate(model: Surrogate, ws, ref, max_iter=200, device="cuda", log=None):
    """Warm vs cold on held-out problems.  ref: descend(...) result from g = 0
    (defines J*).  Both timed runs stop each problem at J <= J* (1 + 1e-6)."""
    Jstar = ref["J"]
    target = Jstar * (1.0 + 1e-6)
    X = features(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g0 = model.propose(X)
    torch.cuda.synchronize()
    t_inf = time.perf_counter() - t0
    warm = descend(ws, g0=g0, max_iter=max_iter, J_target=target, device=device, log=log)
    cold = descend(ws, g0=None, max_iter=max_iter, J_target=target, device=device, log=log)
    gstar = np.stack(ref["g"])
    err = np.linalg.norm((g0 - gstar).reshape(len(ws), -1), axis=1) / np.maximum(
        np.linalg.norm(gstar.reshape(len(ws), -1), axis=1), 1e-300)
    return dict(
        problems=len(ws),
        warm_seconds=warm["seconds"] + t_inf, warm_inference_seconds=t_inf, cold_seconds=cold["seconds"],
        warm_iters_mean=float(warm["iters"].mean()), cold_iters_mean=float(cold["iters"].mean()),
        warm_iters_median=float(np.median(warm["iters"])), cold_iters_median=float(np.median(cold["iters"])),
        warm_reached=int(warm["reached"].sum()), cold_reached=int(cold["reached"].sum()),
        warm_zero_iters=int((warm["iters"] == 0).sum()),
        g0_rel_err_mean=float(err.mean()), g0_rel_err_median=float(np.median(err)),
        J_excess_at_g0_median=float(np.median((warm["J_init"] - Jstar) / Jstar)),
        J_excess_at_zero_median=float(np.median((cold["J_init"] - Jstar) / Jstar)),
    )
