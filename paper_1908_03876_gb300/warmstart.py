"""Learned warm start for the optimal-control problem.

The paper's method (Sec. 3.2.1: forward MRT solve, AMRT adjoint, gradient,
Armijo step) solves each control problem from g = 0.  Here a U-Net
(surrogate.UNet) trained on optimal solutions that the method itself computed
proposes g0 for a new problem, and the same gradient descent refines it.
Plain descent from g = 0 stays the fallback and the reference: the
warm-started run counts as done when its cost reaches the plain optimum J*
to within a relative 1e-6.

What the network predicts.  At the optimum the gradient vanishes:
S(g*)^T r* + 2 alpha L G* = 0, with r* = u^N(g*) - u_target the terminal
residual, S the sensitivity of u^N to the window controls G and L = N/W the
window length.  Write r* = r0 + d*, with r0 = u^N(0) - u_target the residual
without control (one forward solve gives it exactly) and d* = u^N(g*) -
u^N(0) the change the optimal control makes to the terminal state.  The
network predicts d* (one smooth field), and the proposal is
G0 = -S(0)^T (r0 + d_hat) / (2 alpha L): one forward solve at g = 0 and one
AMRT sweep seeded with r0 + d_hat.  Like G*, the proposal lies in the range
of S^T, so its error sits in the directions that steepest descent corrects
quickly; a network that outputs G directly leaves error in the directions
that barely affect u^N, where only the penalty curvature acts and descent is
slow (measured: no gain over the plain method).  Predicting r* itself fails
the other way: r* is mostly the part of the mismatch no control can remove,
and S^T amplifies the network's error relative to the small controllable
part.  Besides the problem parameters the network sees r0 itself, which the
proposal's forward solve provides before the network runs.

Problems: square periodic D2Q9 grids with constant rotated anisotropic
tensors (random eigenvalue ratio and angle), random chemotactic sensitivity,
seeded initial bumps u0 and a fixed centred target; the control acts on v
everywhere and is piecewise constant over W time windows (the network's W
output channels).  The control weight alpha = 1e-2 (per step) makes the
plain descent converge in J within its iteration cap (with 1e-3 it is still
decreasing after 200 steepest-descent iterations, so its "optimum" would be
an unconverged iterate).  Network inputs per node: u0, chi, lambda2/lambda1,
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


def problems(n, seed0, size=128, N=128, windows=8, ckpt_every=32, precision=32, alpha=1e-2):
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
                              u0=u0, v0=np.zeros((size, size)), u_tgt=u_tgt, alpha=alpha,
                              ckpt_every=ckpt_every, windows=windows,
                              extra=dict(ratio=ratio, angle=ang, seed=seed)))
    return out


def features(ws):
    """Static U-Net inputs [n, 5, ny, nx] (float32): scaled u0, chi, 1/ratio,
    cos 2t, sin 2t (the sixth input, r0, comes from a forward solve)."""
    X = np.zeros((len(ws), 5, ws[0].ny, ws[0].nx), dtype=np.float32)
    for i, w in enumerate(ws):
        X[i, 0] = (w.u0 - 1.0) / 0.2
        X[i, 1] = -20.0 * w.chi
        X[i, 2] = 1.0 / w.extra["ratio"]
        X[i, 3] = np.cos(2 * w.extra["angle"])
        X[i, 4] = np.sin(2 * w.extra["angle"])
    return X


def descend(ws, g0=None, max_iter=200, grad_tol=1e-4, stall_tol=1e-7, stall_window=5, J_target=None,
            device="cuda", chunk=256, log=None, init=None, want_residual=False):
    """Batched Armijo gradient descent (the paper's algorithm) on every
    problem from g0 (list of arrays, None: zero controls).

    A problem stops when it has converged: ||E|| / ||E_0||
    < grad_tol (E_0: its gradient at the start), or J fell by less than a
    relative stall_tol over the last stall_window steps (the FP32 lattice
    resolves J to about 1e-7, below which the gradient is rounding noise and
    further steps only random-walk the control in flat directions).  With
    J_target it also stops as soon as its cost is <= J_target[i] (checked at
    the start and after every accepted step; reached = True), and the
    gradient test is not used.  Either way at most max_iter steps.
    init(batch, idx) may set the bound controls (batch.g) inside the timed
    region.  want_residual: also return r = u^N - u_target at the final
    controls (residual) and at the starting controls (residual_init).  Returns dict(g, J, iters, reached, seconds,
    history) where seconds is the wall time of the descent (device work,
    synchronised) and history[i] lists J after each step.
    """
    n = len(ws)
    g_out = [None] * n
    J_out = np.zeros(n)
    J_init = np.full(n, np.nan)
    iters = np.zeros(n, dtype=np.int64)
    reached = np.zeros(n, dtype=bool)
    grad_ratio = np.full(n, np.nan)  # ||E|| / ||E_0|| at the last step
    history = [[] for _ in range(n)]
    resid = [None] * n
    resid0 = [None] * n
    seconds = 0.0
    for c0 in range(0, n, chunk):
        idx = list(range(c0, min(n, c0 + chunk)))
        b = Batch([ws[i] for i in idx], device=device)
        if g0 is None:
            gs = b.zeros_controls()
        else:
            gs = [torch.as_tensor(np.asarray(g0[i]), dtype=b.dtype, device=b.device).contiguous() for i in idx]
        b.bind(gs)
        b.prepare()  # graph capture stays out of the timed region
        active = np.ones(len(idx), dtype=bool)
        e0 = np.full(len(idx), np.nan)
        if want_residual:
            b.forward()
            for k, i in enumerate(idx):
                u, _ = b.fields(k)
                resid0[i] = u.double().cpu().numpy() - ws[i].u_tgt
        torch.cuda.synchronize(b.device)
        t0 = time.perf_counter()
        if init is not None:
            init(b, idx)
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
                if e0[k] > 0:
                    grad_ratio[i] = np.sqrt(info[k]["grad_sq"]) / e0[k]
                J_out[i] = info[k]["J"]
                history[i].append(info[k]["J"])
                stalled = len(history[i]) > stall_window and \
                    history[i][-1 - stall_window] - history[i][-1] < stall_tol * abs(history[i][-1])
                if J_target is not None:
                    if info[k]["J"] <= J_target[i]:
                        active[k] = False
                        reached[i] = True
                    elif stalled:  # converged elsewhere, above the target
                        active[k] = False
                elif (e0[k] > 0 and np.sqrt(info[k]["grad_sq"]) < grad_tol * e0[k]) or stalled:
                    active[k] = False
                    reached[i] = True
            b.set_enabled(active)
            if log and it % 20 == 0:
                log(f"  descend chunk {c0}: it {it} active {int(active.sum())}")
        torch.cuda.synchronize(b.device)
        seconds += time.perf_counter() - t0
        for k, i in enumerate(idx):
            g_out[i] = gs[k].detach().cpu().numpy()
        if want_residual:
            b.set_enabled(None)
            b.forward()
            for k, i in enumerate(idx):
                u, _ = b.fields(k)
                resid[i] = u.double().cpu().numpy() - ws[i].u_tgt
        b.close()
        del b
    return dict(g=g_out, J=J_out, J_init=J_init, iters=iters, reached=reached, seconds=seconds, history=history,
                grad_ratio=grad_ratio, residual=resid, residual_init=resid0)


class Surrogate:
    """U-Net prediction of the optimal control's effect on the terminal state,
    d* = u^N(g*) - u^N(0), from the problem parameters and the uncontrolled
    residual r0, turned into a proposed control by one seeded AMRT sweep."""

    def __init__(self, chans=(32, 64, 128, 256), seed=0, device="cuda"):
        self.net = UNet(cin=6, cout=1, chans=chans, seed=seed, device=device)
        self.device = self.net.device
        self.scale = 1.0     # of d*
        self.r0_scale = 1.0  # of r0

    def _inputs(self, Xs, R0):
        x = torch.as_tensor(Xs, dtype=torch.float32, device=self.device)
        r0 = torch.as_tensor(R0, dtype=torch.float32, device=self.device)[:, None] / self.r0_scale
        return torch.cat([x, r0], dim=1).to(torch.bfloat16).contiguous()

    def fit(self, X, R0, D, epochs=30, batch_size=16, lr=2e-3, seed=0, log=None):
        """Train on static inputs X [n, 5, H, W], uncontrolled residuals R0
        [n, H, W] and terminal-state changes D [n, H, W].  Returns the
        per-epoch mean training loss (on the scaled targets)."""
        D = np.asarray(D)[:, None]
        self.scale = float(np.sqrt(np.mean(np.square(D)))) or 1.0
        self.r0_scale = float(np.sqrt(np.mean(np.square(R0)))) or 1.0
        Xd = self._inputs(X, np.asarray(R0))
        Yd = torch.as_tensor(D / self.scale, dtype=torch.float32, device=self.device)
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

    def predict(self, Xs, R0, batch_size=32):
        """d_hat [n, H, W] (device FP32, unscaled) from static inputs and r0."""
        x = self._inputs(Xs, R0)
        out = []
        for s in range(0, len(x), batch_size):
            out.append(self.net.forward(x[s:s + batch_size].contiguous(), out_f32=True)[:, 0] * self.scale)
        return torch.cat(out)

    def initializer(self, ws, D=None):
        """init hook for descend(): the bound controls of the chunk become
        G0 = -S(0)^T (r0 + d) / (2 alpha L), d = the network's prediction
        (or the given D, for diagnostics)."""
        X = features(ws)
        if D is None:
            return proposal_init(ws, lambda idx, r0: self.predict(X[idx], r0))
        return proposal_init(ws, lambda idx, r0: torch.as_tensor(np.stack([D[i] for i in idx]),
                                                                 dtype=torch.float32, device=self.device))


def proposal_init(ws, d_of):
    """init hook: G0 = -S(0)^T (r0 + d) / (2 alpha L), d = d_of(idx, r0) [len(idx), H, W]."""

    def init(b, idx):
        b.forward()                                                   # state and r0 at g = 0
        r0 = torch.stack([b.fields(k)[0] for k in range(len(idx))]).float() - torch.as_tensor(
            np.stack([ws[i].u_tgt for i in idx]), dtype=torch.float32, device=b.device)
        d = d_of(idx, r0).to(b.dtype)
        b.adjoint([d[k] for k in range(len(idx))], add_to_cost_seed=True)  # E = S(0)^T (r0 + d)
        lam = [1.0 / (2.0 * ws[i].alpha * (ws[i].N // (ws[i].windows or ws[i].N))) for i in idx]
        b.axpy(lam)                                                   # G0 = 0 - lam E

    return init


def evaluate(model: Surrogate, ws, ref, max_iter=200, device="cuda", log=None, stall_tol=1e-9, repeats=3):
    """Warm vs cold on held-out problems.  ref: descend(...) result from g = 0
    (defines J*).  Both timed runs stop each problem at J <= J* (1 + 1e-6);
    the warm run's time includes the network, the forward at g = 0 and the
    seeded sweep that make its proposal.  A warm-started problem that stops
    improving (relative J decrease < stall_tol over 5 steps) above the target
    falls back to the plain method from g = 0, and that time is added.  The
    timed runs are repeated (deterministic: same iterations) and the median
    wall times reported."""
    Jstar = ref["J"]
    target = Jstar * (1.0 + 1e-6)
    model.predict(features(ws[:1]), np.zeros((1, ws[0].ny, ws[0].nx)))  # module loading stays out of the timing
    warm_s, cold_s = [], []
    for rep in range(repeats):
        warm = descend(ws, init=model.initializer(ws), max_iter=max_iter, J_target=target, device=device, log=log,
                       stall_tol=stall_tol)
        # fallback: problems whose warm-started descent converged above the
        # target are solved again by the plain method from g = 0
        failed = [i for i in range(len(ws)) if not warm["reached"][i]]
        fb_seconds, fb_iters = 0.0, 0
        if failed:
            fb = descend([ws[i] for i in failed], g0=None, max_iter=max_iter, J_target=target[failed],
                         device=device, stall_tol=stall_tol)
            fb_seconds, fb_iters = fb["seconds"], int(fb["iters"].sum())
        warm_s.append(warm["seconds"] + fb_seconds)
        cold = descend(ws, g0=None, max_iter=max_iter, J_target=target, device=device, log=log, stall_tol=stall_tol)
        cold_s.append(cold["seconds"])
    # the proposal itself, against g*; and the proposal from the exact d*
    n = len(ws)
    gstar = np.stack(ref["g"])

    def rel_err(g):
        g = np.stack(g)
        return np.linalg.norm((g - gstar).reshape(n, -1), axis=1) / np.maximum(
            np.linalg.norm(gstar.reshape(n, -1), axis=1), 1e-300)

    err = rel_err(descend(ws, init=model.initializer(ws), max_iter=0, device=device)["g"])
    Dstar = [r - r0 for r, r0 in zip(ref["residual"], ref["residual_init"])]
    err_exact = rel_err(descend(ws, init=model.initializer(ws, D=Dstar), max_iter=0, device=device)["g"])
    Dh = model.predict(features(ws), np.stack(ref["residual_init"])).double().cpu().numpy()
    Ds = np.stack(Dstar)
    d_err = float(np.median(np.linalg.norm((Dh - Ds).reshape(n, -1), axis=1) /
                            np.linalg.norm(Ds.reshape(n, -1), axis=1)))
    return dict(
        problems=n,
        warm_seconds=float(np.median(warm_s)), cold_seconds=float(np.median(cold_s)),
        warm_seconds_all=warm_s, cold_seconds_all=cold_s, fallback_problems=len(failed),
        fallback_final_excess=[float(warm["J"][i] / Jstar[i] - 1.0) for i in failed],
        warm_iters_total=int(warm["iters"].sum()) + fb_iters, cold_iters_total=int(cold["iters"].sum()),
        warm_iters_mean=float(warm["iters"].mean()), cold_iters_mean=float(cold["iters"].mean()),
        warm_iters_median=float(np.median(warm["iters"])), cold_iters_median=float(np.median(cold["iters"])),
        warm_reached=int(warm["reached"].sum()), cold_reached=int(cold["reached"].sum()),
        warm_zero_iters=int((warm["iters"] == 0).sum()),
        g0_rel_err_mean=float(err.mean()), g0_rel_err_median=float(np.median(err)),
        g0_from_exact_d_rel_err_median=float(np.median(err_exact)), d_rel_err_median=d_err,
        J_excess_at_g0_median=float(np.median((warm["J_init"] - Jstar) / Jstar)),
        J_excess_at_zero_median=float(np.median((cold["J_init"] - Jstar) / Jstar)),
    )
