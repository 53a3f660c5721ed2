"""Many independent control problems advanced together on one GPU.

Thin binding over the cx_batch_* calls of include/cxlbm.h: one persistent
launch per time step covers every problem's tiles, and the launch sequence of
a forward or gradient evaluation is a captured CUDA graph replayed on each
call.  PyTorch provides the memory and a (non-default) stream.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from .problem import _ptr, make_desc


def _vp_array(ts):
    arr = (ctypes.c_void_p * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = None if t is None else t.data_ptr()
    return arr


class Batch:
    def __init__(self, workloads, device="cuda", stream: torch.cuda.Stream | None = None):
        self.lib = _lib.load()
        self.ws_list = list(workloads)
        w0 = self.ws_list[0]
        self.count = len(self.ws_list)
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.precision = w0.precision
        self.dtype = torch.float64 if self.precision == 64 else torch.float32
        # graph capture needs a stream other than the legacy default stream
        self.stream = stream or torch.cuda.Stream(self.device)
        descs = (_lib.Desc * self.count)()
        self._keep = []
        for i, w in enumerate(self.ws_list):
            d, keep = make_desc(w, self.device, self.precision)
            descs[i] = d
            self._keep.append(keep)
        self.descs = descs
        nbytes = ctypes.c_size_t(0)
        _lib.check(self.lib.cx_batch_workspace_size(descs, self.count, ctypes.byref(nbytes)), "cx_batch_workspace_size")
        self.workspace_bytes = nbytes.value
        self.ws = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
        h = ctypes.c_void_p()
        _lib.check(self.lib.cx_batch_create(descs, self.count, _ptr(self.ws), nbytes.value,
                                            ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)),
                   "cx_batch_create")
        self.h = h
        self._keep = None  # cx_batch_create synchronised: the descriptor arrays were read
        u0 = [torch.as_tensor(w.u0, dtype=self.dtype, device=self.device).contiguous() for w in self.ws_list]
        v0 = [torch.as_tensor(w.v0, dtype=self.dtype, device=self.device).contiguous() for w in self.ws_list]
        _lib.check(self.lib.cx_batch_set_initial(self.h, _vp_array(u0), _vp_array(v0)), "cx_batch_set_initial")
        self.stream.synchronize()
        self.out = torch.zeros(3 * self.count, dtype=torch.float64, device=self.device)
        self.g = None
        self.E = None

    def zeros_controls(self):
        return [torch.zeros(w.ctrl_shape, dtype=self.dtype, device=self.device) for w in self.ws_list]

    def bind(self, g, E=None):
        """Controls g[i] and gradient outputs E[i] (lists of device tensors)."""
        self.g = [None if x is None else x.contiguous() for x in g]
        self.E = E if E is not None else [torch.empty(w.ctrl_shape, dtype=self.dtype, device=self.device)
                                         for w in self.ws_list]
        torch.cuda.synchronize(self.device)
        _lib.check(self.lib.cx_batch_bind(self.h, _vp_array(self.g), _vp_array(self.E)), "cx_batch_bind")

    def set_tiles(self, threads=256, blocks=0, tile_x=None, rows=None):
        """Tile width and rows per thread of every problem (None: defaults)."""
        arr = None if tile_x is None else (ctypes.c_int * self.count)(*tile_x)
        rws = None if rows is None else (ctypes.c_int * self.count)(*rows)
        _lib.check(self.lib.cx_batch_set_tiles(self.h, threads, blocks, arr, rws), "cx_batch_set_tiles")

    def set_staging(self, row_windows=True):
        """Bulk row-window staging (True, the default) or per-thread copies
        everywhere (False); results are identical."""
        _lib.check(self.lib.cx_batch_set_staging(self.h, 1 if row_windows else 0), "cx_batch_set_staging")

    def _enter(self):
        # inputs written on the caller's stream are visible to the batch's stream
        self.stream.wait_stream(torch.cuda.current_stream(self.device))

    def _leave(self):
        # results are visible to work the caller queues next on its stream
        torch.cuda.current_stream(self.device).wait_stream(self.stream)

    def forward(self):
        """J of every problem (device FP64 [count])."""
        self._enter()
        _lib.check(self.lib.cx_batch_forward(self.h, _ptr(self.out)), "cx_batch_forward")
        self._leave()
        return self.out[: self.count]

    def gradient(self):
        """(J, ||dJ/dg||^2, max |dJ/dg|) per problem; gradients land in self.E."""
        self._enter()
        _lib.check(self.lib.cx_batch_gradient(self.h, _ptr(self.out)), "cx_batch_gradient")
        self._leave()
        return self.out[: self.count], self.out[self.count: 2 * self.count], self.out[2 * self.count:]

    def adjoint(self, seeds=None, add_to_cost_seed=False):
        """Seeded AMRT sweep (seeds: list of [ny, nx] device tensors, the
        adjoint of u^N, or additions to u^N - u_target) after forward();
        gradients land in self.E.  Returns (||dJ/dg||^2, max |dJ/dg|) per
        problem."""
        self._seeds = None if seeds is None else [s.contiguous() for s in seeds]
        arr = None if seeds is None else _vp_array(self._seeds)
        self._enter()
        _lib.check(self.lib.cx_batch_adjoint(self.h, arr, 1 if add_to_cost_seed else 0, _ptr(self.out)),
                   "cx_batch_adjoint")
        self._leave()
        return self.out[self.count: 2 * self.count], self.out[2 * self.count:]

    def prepare(self):
        """Capture every launch sequence as a CUDA graph now (not on first use)."""
        self._enter()
        _lib.check(self.lib.cx_batch_prepare(self.h), "cx_batch_prepare")
        self._leave()

    def axpy(self, lam):
        """g[i] <- g[i] - lam[i] E[i] (lam: per-problem floats)."""
        arr = (ctypes.c_double * self.count)(*[float(x) for x in lam])
        self._enter()
        _lib.check(self.lib.cx_batch_axpy(self.h, arr), "cx_batch_axpy")
        self._leave()

    def step(self):
        """One Armijo gradient-descent iteration of every enabled problem: the
        bound controls are updated in place, self.E holds the gradients at the
        incoming controls.  Returns (info, status): per-problem dicts (J0, J,
        lam, grad_sq, grad_inf, trials) and cx_status codes."""
        info = (_lib.StepInfo * self.count)()
        st = (ctypes.c_int * self.count)()
        self._enter()
        _lib.check(self.lib.cx_batch_step(self.h, info, st), "cx_batch_step")
        self._leave()
        out = [dict(J0=x.J0, J=x.J, lam=x.lam, grad_sq=x.grad_sq, grad_inf=x.grad_inf, trials=x.trials)
               for x in info]
        return out, list(st)

    def set_enabled(self, mask=None):
        """Switch problems on/off (sequence of bools, None: all on)."""
        arr = None if mask is None else (ctypes.c_int * self.count)(*[1 if m else 0 for m in mask])
        self._enter()
        _lib.check(self.lib.cx_batch_set_enabled(self.h, arr), "cx_batch_set_enabled")

    def fields(self, i):
        w = self.ws_list[i]
        u = torch.empty((w.ny, w.nx), dtype=self.dtype, device=self.device)
        v = torch.empty_like(u)
        self._enter()
        _lib.check(self.lib.cx_batch_get_fields(self.h, i, _ptr(u), _ptr(v)), "cx_batch_get_fields")
        self._leave()
        return u, v

    def status(self):
        _lib.check(self.lib.cx_batch_get_status(self.h), "cx_batch_get_status")

    def close(self):
        if getattr(self, "h", None):
            self.lib.cx_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
