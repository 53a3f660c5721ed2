"""Tile-shape and schedule autotuner for the batched launch.

Tunables: threads per block (128, 256) and, per size class (problems with the
same nx), the tile width tx and the rows r each thread updates per tile (tile
= tx x r threads/tx nodes).  The tuner times a short probe batch (the same
problems with a few time steps): first the best of a few uniform shapes (the
same width and rows for every class), then coordinate descent from it: for
each class try the other row counts, then the other admissible widths, while
the rest stay fixed, keeping the fastest.  The probe is a gradient evaluation (forward,
segment recompute and adjoint: the kernels differ in their best tiles), not
a forward alone.  Results are cached in a JSON file keyed by the device,
lattice, precision and the size-class histogram.
"""
from __future__ import annotations

import json
import os
from dataclasses import replace

import torch

from .batch import Batch

WIDTHS = (32, 64, 128, 256)
ROWS = (4, 8, 16, 32)
UNIFORM = ((32, 8), (64, 8), (64, 16), (128, 16), (32, 16))


def _signature(workloads, device):
    from collections import Counter

    hist = Counter(w.nx for w in workloads)
    name = torch.cuda.get_device_name(device)
    w0 = workloads[0]
    return f"{name}|Q{w0.Q}|fp{w0.precision}|" + ",".join(f"{k}:{v}" for k, v in sorted(hist.items()))


def _admissible(threads, nx):
    return [t for t in WIDTHS if t <= threads and threads % t == 0 and threads // t <= 8 and t <= max(32, 2 * nx)]


def _time_gradient(b: Batch, reps=2):
    b.gradient()
    b.stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    for _ in range(reps):
        b.gradient()
    e1.record(b.stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def autotune(workloads, probe_steps=24, threads_options=(128, 256), cache_path=None, device="cuda"):
    """Returns {"threads": T, "blocks": 0, "tile_x": {nx: tx}, "rows": {nx: r}, "ms": best probe time}."""
    sig = _signature(workloads, device)
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as fh:
            cache = json.load(fh)
        if sig in cache:
            got = cache[sig]
            got["tile_x"] = {int(k): v for k, v in got["tile_x"].items()}
            got["rows"] = {int(k): v for k, v in got.get("rows", {}).items()}
            return got
    probe = [replace(w, N=probe_steps, ckpt_every=max(1, probe_steps // 2)) for w in workloads]
    b = Batch(probe, device=device)
    b.bind([None] * len(probe), None)
    classes = sorted(set(w.nx for w in probe))
    best = None
    for threads in threads_options:
        def run(ch, rw):
            b.set_tiles(threads, 0, [ch[w.nx] for w in probe], [rw[w.nx] for w in probe])
            return _time_gradient(b)

        t_best, choice, rows = None, None, None
        for tx, r in UNIFORM:
            ch = {nx: min(tx, max(_admissible(threads, nx))) for nx in classes}
            if any(c not in _admissible(threads, nx) for nx, c in ch.items()):
                continue
            rw = {nx: r for nx in classes}
            t = run(ch, rw)
            if t_best is None or t < t_best:
                t_best, choice, rows = t, ch, rw
        for nx in classes:
            for r in ROWS:
                if r == rows[nx]:
                    continue
                trial = dict(rows)
                trial[nx] = r
                t = run(choice, trial)
                if t < t_best:
                    t_best, rows = t, trial
            for tx in _admissible(threads, nx):
                if tx == choice[nx]:
                    continue
                trial = dict(choice)
                trial[nx] = tx
                t = run(trial, rows)
                if t < t_best:
                    t_best, choice = t, trial
        if best is None or t_best < best["ms"]:
            best = {"threads": threads, "blocks": 0, "tile_x": dict(choice), "rows": dict(rows), "ms": t_best}
    b.close()
    if cache_path:
        cache = {}
        if os.path.exists(cache_path):
            with open(cache_path) as fh:
                cache = json.load(fh)
        cache[sig] = {**best, "tile_x": {str(k): v for k, v in best["tile_x"].items()},
                      "rows": {str(k): v for k, v in best["rows"].items()}}
        with open(cache_path, "w") as fh:
            json.dump(cache, fh, indent=1)
    return best


def apply(batch: Batch, cfg):
    rows = cfg.get("rows", {})
    batch.set_tiles(cfg["threads"], cfg.get("blocks", 0), [cfg["tile_x"][w.nx] for w in batch.ws_list],
                    [rows.get(w.nx, 2) for w in batch.ws_list])
