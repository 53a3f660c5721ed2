"""Python handle on one D3Q19 problem (include/cx3d.h): the two-species
chemotaxis control problem on a periodic three-dimensional lattice.

Argument marshalling only: PyTorch provides the workspace, the descriptor's
device fields and the stream; the forward MRT solve, the exact discrete
adjoint with the fused gradient and the Armijo search run in the library.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from .workloads import Workload3D


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def make_desc3d(w: Workload3D, dev, precision=None):
    """cx3d_desc for a workload; returns (desc, device arrays it points to)."""
    f64 = lambda a: None if a is None else torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    keep = {}
    d = _lib.Desc3D()
    d.nx, d.ny, d.nz, d.n_steps = w.nx, w.ny, w.nz, w.N
    d.precision = precision or w.precision
    d.ckpt_every = w.ckpt_every or w.N
    d.tau = 1.0
    d.aniso = {"const": _lib.CX_ANISO_CONST, "field": _lib.CX_ANISO_FIELD}[w.aniso]
    d.D_u = (ctypes.c_double * 6)(*w.D_u_const)
    d.D_v = (ctypes.c_double * 6)(*w.D_v_const)
    if w.aniso == "field":
        keep["Du"], keep["Dv"] = f64(w.D_u_field), f64(w.D_v_field)
        d.D_u_field, d.D_v_field = _ptr(keep["Du"]), _ptr(keep["Dv"])
    for k in ("d_u", "d_v", "chi", "r_vu", "r_vv", "alpha"):
        setattr(d, k, float(getattr(w, k)))
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


class D3Problem:
    """One D3Q19 problem bound to a caller-owned workspace and a stream."""

    def __init__(self, w: Workload3D, device="cuda", stream: torch.cuda.Stream | None = None, precision=None):
        self.lib = _lib.load()
        self.w = w
        self.device = torch.device(device)
        if self.device.type == "cuda" and self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.precision = precision or w.precision
        self.dtype = torch.float64 if self.precision == 64 else torch.float32
        self.stream = stream or torch.cuda.current_stream(self.device)
        self.ctrl_shape = w.ctrl_shape
        d, keep = make_desc3d(w, self.device, self.precision)
        nbytes = ctypes.c_size_t(0)
        _lib.check(self.lib.cx3d_workspace_size(ctypes.byref(d), ctypes.byref(nbytes)), "cx3d_workspace_size")
        self.workspace_bytes = nbytes.value
        with torch.cuda.device(self.device):
            self.ws = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=self.device)
        h = ctypes.c_void_p()
        _lib.check(self.lib.cx3d_create(ctypes.byref(d), _ptr(self.ws), nbytes.value,
                                        ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)), "cx3d_create")
        self.h = h
        del keep  # converted into the workspace by cx3d_create
        self._J = torch.zeros(1, dtype=torch.float64, device=self.device)
        self.set_initial(w.u0, w.v0)

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

    def set_initial(self, u0, v0):
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=self.device)
        u, v = f(u0), f(v0)
        _lib.check(self.lib.cx3d_set_initial(self.h, _ptr(u), _ptr(v)), "cx3d_set_initial")
        self._init = (u, v)

    def forward(self, g=None):
        g = self._t(g, self.ctrl_shape)
        _lib.check(self.lib.cx3d_forward(self.h, _ptr(g), _ptr(self._J)), "cx3d_forward")
        self._g = g
        return self._J

    def adjoint(self, g=None, seed_u=None, seed_v=None, penalty=True, out=None):
        g = self._t(g, self.ctrl_shape)
        shp = (self.w.nz, self.w.ny, self.w.nx)
        su, sv = self._t(seed_u, shp), self._t(seed_v, shp)
        out = out if out is not None else torch.empty(self.ctrl_shape, dtype=self.dtype, device=self.device)
        _lib.check(self.lib.cx3d_adjoint(self.h, _ptr(g), _ptr(su), _ptr(sv), 1 if penalty else 0, _ptr(out)),
                   "cx3d_adjoint")
        self._seeds = (su, sv)
        return out

    def gradient(self, g=None, out=None):
        g = self._t(g, self.ctrl_shape)
        out = out if out is not None else torch.empty(self.ctrl_shape, dtype=self.dtype, device=self.device)
        _lib.check(self.lib.cx3d_gradient(self.h, _ptr(g), _ptr(out), _ptr(self._J)), "cx3d_gradient")
        return self._J, out

    def step(self, g, E=None):
        if g.dtype != self.dtype or not g.is_contiguous() or g.device != self.device or \
                tuple(g.shape) != tuple(self.ctrl_shape):
            raise ValueError("g must be a contiguous device tensor of the problem's dtype")
        E = E if E is not None else torch.empty_like(g)
        info = _lib.StepInfo()
        _lib.check(self.lib.cx3d_step(self.h, _ptr(g), _ptr(E), ctypes.byref(info)), "cx3d_step")
        return dict(J0=info.J0, J=info.J, lam=info.lam, grad_sq=info.grad_sq, grad_inf=info.grad_inf,
                    trials=info.trials)

    def fields(self):
        u = torch.empty((self.w.nz, self.w.ny, self.w.nx), dtype=self.dtype, device=self.device)
        v = torch.empty_like(u)
        _lib.check(self.lib.cx3d_get_fields(self.h, _ptr(u), _ptr(v)), "cx3d_get_fields")
        return u, v

    def norms(self):
        J, e2, einf = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _lib.check(self.lib.cx3d_get_norms(self.h, ctypes.byref(J), ctypes.byref(e2), ctypes.byref(einf)),
                   "cx3d_get_norms")
        return J.value, e2.value, einf.value

    def set_timing(self, on=True):
        _lib.check(self.lib.cx3d_set_timing(self.h, 1 if on else 0), "cx3d_set_timing")

    def timing(self):
        ms = (ctypes.c_double * 3)()
        cnt = (ctypes.c_longlong * 3)()
        _lib.check(self.lib.cx3d_get_timing(self.h, ms, cnt), "cx3d_get_timing")
        return {n: (ms[i], cnt[i]) for i, n in enumerate(("forward", "recompute", "adjoint"))}

    def close(self):
        if getattr(self, "h", None):
            self.lib.cx3d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
