"""The optimisation loop around the library's descent iterations, with a
JSON-lines log and checkpoint/resume of the control.

Every iteration runs in the CUDA library: one forward solve, the AMRT adjoint
sweep and the line search (the gradient algorithm of Sec. 2.3 and the
optimisation process of Sec. 3.2.1) through ``Problem.step`` (Armijo),
``Problem.lma_step`` (linearised step length) or ``Problem.cg_step``
(nonlinear conjugate gradients).  This module only repeats them, decides when
to stop, writes one JSON object per iteration and saves or restores the
control between runs.  It does no arithmetic of the method.

Resuming restores the control and the iteration count.  The line search's
memory (the previous step length, the conjugate direction) stays inside the
library object that ran the iterations, so a resumed run starts its first
line search afresh, from min(1, 1/||E||_inf), and a resumed CG run restarts
from the steepest-descent direction; from there on it is the same descent.
"""
from __future__ import annotations

import json
import math
import os
import time

import torch

METHODS = ("armijo", "lma", "cg-FR", "cg-PR", "cg-HS", "cg-DY")


def _one_iteration(problem, g, method, E):
    if method == "armijo":
        return problem.step(g, E)
    if method == "lma":
        return problem.lma_step(g, E)
    if method.startswith("cg-"):
        return problem.cg_step(g, method[3:])
    raise ValueError(f"unknown method {method!r}; one of {METHODS}")


def descend(problem, g, iters, method="armijo", target=None, grad_ratio=None, log=None, checkpoint=None,
            checkpoint_every=0, start=0):
    """Run iterations start, start + 1, ... < iters on the control g (a device
    tensor of the problem's control shape, updated in place).

    Stops early once J <= target, or once ||E|| / ||E_0|| < grad_ratio with
    E_0 the gradient at the first iteration of this call.
    log: path of a JSON-lines file, one object appended per iteration (iter,
    method, J0, J, lam, trials, grad_norm, grad_inf when the method reports
    it, seconds, stop).
    checkpoint: path written with torch.save every checkpoint_every iterations
    (0: only at the end): the control (on the host), the next iteration's
    index, the method and the last record.
    Returns the list of records."""
    if method not in METHODS:
        raise ValueError(f"unknown method {method!r}; one of {METHODS}")
    E = torch.empty_like(g) if method in ("armijo", "lma") else None
    records = []
    g0_norm = None
    fh = open(log, "a") if log else None
    try:
        k = start
        while k < iters:
            t0 = time.perf_counter()
            info = _one_iteration(problem, g, method, E)
            dt = time.perf_counter() - t0
            gnorm = math.sqrt(max(info["grad_sq"], 0.0))
            if g0_norm is None:
                g0_norm = gnorm
            stop = None
            if target is not None and info["J"] <= target:
                stop = "target"
            elif grad_ratio is not None and g0_norm > 0 and gnorm / g0_norm < grad_ratio:
                stop = "grad_ratio"
            elif k + 1 >= iters:
                stop = "iters"
            rec = {"iter": k, "method": method, "J0": info["J0"], "J": info["J"], "lam": info["lam"],
                   "trials": info["trials"], "grad_norm": gnorm, "seconds": dt, "stop": stop}
            if "grad_inf" in info:
                rec["grad_inf"] = info["grad_inf"]
            records.append(rec)
            if fh:
                fh.write(json.dumps(rec) + "\n")
                fh.flush()
            k += 1
            if checkpoint and (stop or (checkpoint_every and k % checkpoint_every == 0)):
                save_checkpoint(checkpoint, g, k, method, rec)
            if stop:
                break
    finally:
        if fh:
            fh.close()
    return records


def save_checkpoint(path, g, next_iter, method, last=None):
    """The control (copied to the host), the index of the next iteration, the
    method and the last record, written atomically."""
    tmp = f"{path}.{os.getpid()}.tmp"
    torch.save({"g": g.detach().to("cpu"), "next_iter": int(next_iter), "method": method, "last": last}, tmp)
    os.replace(tmp, path)


def resume(path, problem):
    """(g, next_iter, method, last record) from a checkpoint, with g on the
    problem's device in its control dtype."""
    ck = torch.load(path, map_location="cpu")
    g = ck["g"].to(device=problem.device, dtype=problem.dtype).contiguous()
    return g, ck["next_iter"], ck["method"], ck["last"]
