"""Python handle on one three-species problem (include/cxarc.h): the
attraction-repulsion chemotaxis model with a logistic source.

Argument marshalling only: PyTorch provides the workspace, the descriptor's
device fields and the stream; the forward MRT solve, the exact discrete
adjoint with the fused gradient and the Armijo search run in the library.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from .workloads import Workload3


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def make_desc3(w: Workload3, dev, precision=None):
    """cx3_desc for a workload; returns (desc, device arrays it points to)."""
    f64 = lambda a: None if a is None else torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    keep = {}
    d = _lib.Desc3()
    d.nx, d.ny, d.n_steps = w.nx, w.ny, w.N
    d.precision = precision or w.precision
    d.ckpt_every = w.ckpt_every or w.N
    d.tau = 1.0
    d.aniso = {"const": _lib.CX_ANISO_CONST, "rotated": _lib.CX_ANISO_ROTATED, "field": _lib.CX_ANISO_FIELD}[w.aniso]
    d.D_u = (ctypes.c_double * 3)(*w.D_u_const)
    d.D_v = (ctypes.c_double * 3)(*w.D_v_const)
    d.D_w = (ctypes.c_double * 3)(*w.D_w_const)
    d.lam_u = (ctypes.c_double * 2)(*w.lam_u)
    d.lam_v = (ctypes.c_double * 2)(*w.lam_v)
    d.lam_w = (ctypes.c_double * 2)(*w.lam_w)
    if w.aniso == "rotated":
        keep["theta"] = f64(w.theta)
        d.theta = _ptr(keep["theta"])
    if w.aniso == "field":
        keep["Du"], keep["Dv"], keep["Dw"] = f64(w.D_u_field), f64(w.D_v_field), f64(w.D_w_field)
        d.D_u_field, d.D_v_field, d.D_w_field = _ptr(keep["Du"]), _ptr(keep["Dv"]), _ptr(keep["Dw"])
    for k in ("d", "chi1", "chi2", "a1", "a2", "b1", "b2", "b3", "c1", "c2", "alpha"):
        setattr(d, k, float(getattr(w, k)))
    d.ctrl_species = w.ctrl_species
    d.adv = {"none": _lib.CX_ADV_NONE, "row": _lib.CX_ADV_ROW, "field": _lib.CX_ADV_FIELD}[w.adv]
    if w.adv == "row":
        keep["a"] = f64(w.a_row)
    elif w.adv == "field":
        keep["a"] = f64(w.a_field)
    d.a = _ptr(keep.get("a"))
    keep["ut"] = f64(w.u_tgt)
    d.u_target = _ptr(keep["ut"])
    d.s = (ctypes.c_double * 7)(*w.s)
    d.source_order = w.source_order
    return d, keep


class ArcProblem:
    """One three-species problem bound to a caller-owned workspace and a stream."""

    def __init__(self, w: Workload3, device="cuda", stream: torch.cuda.Stream | None = None, precision=None):
        self.lib = _lib.load()
        self.w = w
        self.device = torch.device(device)
        if self.device.type == "cuda" and self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.precision = precision or w.precision
        self.dtype = torch.float64 if self.precision == 64 else torch.float32
        self.stream = stream or torch.cuda.current_stream(self.device)
        self.ctrl_shape = w.ctrl_shape
        d, keep = make_desc3(w, self.device, self.precision)
        nbytes = ctypes.c_size_t(0)
        _lib.check(self.lib.cx3_workspace_size(ctypes.byref(d), ctypes.byref(nbytes)), "cx3_workspace_size")
        self.workspace_bytes = nbytes.value
        with torch.cuda.device(self.device):
            self.ws = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=self.device)
        h = ctypes.c_void_p()
        _lib.check(self.lib.cx3_create(ctypes.byref(d), _ptr(self.ws), nbytes.value,
                                       ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)), "cx3_create")
        self.h = h
        del keep  # cx3_create converted every field into the workspace
        self._J = torch.zeros(1, dtype=torch.float64, device=self.device)
        self.set_initial(w.u0, w.v0, w.w0)

    def _t(self, a, shape):
        if a is None:
            return None
        t = torch.as_tensor(a, device=self.device)
        if t.dtype != self.dtype:
            t = t.to(self.dtype)
        t = t.contiguous()
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"expected shape {shape}, got {tuple(t.shape)}")
        return t

    def zeros_control(self):
        return torch.zeros(self.ctrl_shape, dtype=self.dtype, device=self.device)

    def set_initial(self, u0, v0, w0):
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=self.device)
        u, v, w = f(u0), f(v0), f(w0)
        _lib.check(self.lib.cx3_set_initial(self.h, _ptr(u), _ptr(v), _ptr(w)), "cx3_set_initial")
        self._init = (u, v, w)  # read by the queued initial kernel

    def forward(self, g=None):
        """Forward solve; the FP64 cost J as a 1-element device tensor."""
        g = self._t(g, self.ctrl_shape)
        _lib.check(self.lib.cx3_forward(self.h, _ptr(g), _ptr(self._J)), "cx3_forward")
        self._g = g
        return self._J

    def adjoint(self, g=None, seeds=None, penalty=True, out=None):
        """Exact discrete adjoint at the last forward's control g.  seeds:
        None (the cost's terminal term) or a triple of [ny, nx] arrays / None
        (the adjoints of u^N, v^N, w^N)."""
        g = self._t(g, self.ctrl_shape)
        shp = (self.w.ny, self.w.nx)
        s = [None, None, None] if seeds is None else [self._t(x, shp) for x in seeds]
        out = out if out is not None else torch.empty(self.ctrl_shape, dtype=self.dtype, device=self.device)
        _lib.check(self.lib.cx3_adjoint(self.h, _ptr(g), _ptr(s[0]), _ptr(s[1]), _ptr(s[2]), 1 if penalty else 0,
                                        _ptr(out)), "cx3_adjoint")
        self._seeds = s
        return out

    def gradient(self, g=None, out=None):
        g = self._t(g, self.ctrl_shape)
        out = out if out is not None else torch.empty(self.ctrl_shape, dtype=self.dtype, device=self.device)
        _lib.check(self.lib.cx3_gradient(self.h, _ptr(g), _ptr(out), _ptr(self._J)), "cx3_gradient")
        return self._J, out

    def step(self, g, E=None):
        """One Armijo steepest-descent iteration, g updated in place."""
        if g.dtype != self.dtype or not g.is_contiguous() or g.device != self.device or \
                tuple(g.shape) != tuple(self.ctrl_shape):
            raise ValueError("g must be a contiguous device tensor of the problem's dtype")
        E = E if E is not None else torch.empty_like(g)
        info = _lib.StepInfo()
        _lib.check(self.lib.cx3_step(self.h, _ptr(g), _ptr(E), ctypes.byref(info)), "cx3_step")
        return dict(J0=info.J0, J=info.J, lam=info.lam, grad_sq=info.grad_sq, grad_inf=info.grad_inf,
                    trials=info.trials)

    def fields(self):
        u = torch.empty((self.w.ny, self.w.nx), dtype=self.dtype, device=self.device)
        v, w = torch.empty_like(u), torch.empty_like(u)
        _lib.check(self.lib.cx3_get_fields(self.h, _ptr(u), _ptr(v), _ptr(w)), "cx3_get_fields")
        return u, v, w

    def norms(self):
        J, e2, einf = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _lib.check(self.lib.cx3_get_norms(self.h, ctypes.byref(J), ctypes.byref(e2), ctypes.byref(einf)),
                   "cx3_get_norms")
        return J.value, e2.value, einf.value

    def set_staging(self, mode=1):
        """1: the forward in the row-window kernel where it pays (default);
        0: per-thread kernels only; 2: row-window forward and adjoint for
        every eligible step (tests)."""
        _lib.check(self.lib.cx3_set_staging(self.h, int(mode)), "cx3_set_staging")

    def set_timing(self, on=True):
        _lib.check(self.lib.cx3_set_timing(self.h, 1 if on else 0), "cx3_set_timing")

    def timing(self):
        ms = (ctypes.c_double * 3)()
        cnt = (ctypes.c_longlong * 3)()
        _lib.check(self.lib.cx3_get_timing(self.h, ms, cnt), "cx3_get_timing")
        return {n: (ms[i], cnt[i]) for i, n in enumerate(("forward", "recompute", "adjoint"))}

    def close(self):
        if getattr(self, "h", None):
            self.lib.cx3_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
