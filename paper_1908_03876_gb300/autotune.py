"""Tile-shape autotuner for the batched launch (binding of cx_batch_autotune).

The search runs in the library: per size class (problems with the same nx)
the tile width and the rows each thread updates per tile, for 128 and 256
threads per block, timed on a short probe of the batch's own gradient
evaluation (forward, segment recompute, AMRT adjoint); the winner is applied
to the batch.  Results are cached in a text file keyed by the device,
lattice, precision and the size-class histogram.
"""
from __future__ import annotations

import ctypes

from . import _lib
from .batch import Batch


def autotune(batch: Batch, probe_steps=24, cache_path=None):
    """Tunes and applies the tiles of `batch` (initial state set, controls
    and gradient outputs bound).  Returns {"threads", "blocks": 0,
    "tile_x": {nx: tx}, "rows": {nx: r}, "ms": probe time}.  The probe
    overwrites the forward state, so the next evaluation recomputes it."""
    n = batch.count
    threads = ctypes.c_int(0)
    tx = (ctypes.c_int * n)()
    rows = (ctypes.c_int * n)()
    ms = ctypes.c_double(0.0)
    path = None if cache_path is None else str(cache_path).encode()
    batch._enter()
    _lib.check(batch.lib.cx_batch_autotune(batch.h, int(probe_steps), path, ctypes.byref(threads), tx, rows,
                                           ctypes.byref(ms)), "cx_batch_autotune")
    batch._leave()
    return {"threads": threads.value, "blocks": 0,
            "tile_x": {w.nx: tx[i] for i, w in enumerate(batch.ws_list)},
            "rows": {w.nx: rows[i] for i, w in enumerate(batch.ws_list)}, "ms": ms.value}


def apply(batch: Batch, cfg):
    """Applies a tuned configuration (for example one tuned on another batch
    with the same size classes)."""
    rows = cfg.get("rows", {})
    batch.set_tiles(cfg["threads"], cfg.get("blocks", 0), [cfg["tile_x"][w.nx] for w in batch.ws_list],
                    [rows.get(w.nx, 2) for w in batch.ws_list])
