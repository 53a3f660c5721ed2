"""Python handle on one optimal-control problem of the CUDA library.

Thin binding over include/cxlbm.h: PyTorch provides device memory (the
workspace and the per-problem fields) and the current CUDA stream; every step
of the method runs in the library's kernels.  Calls follow the paper's
statement of the problem and its discrete-adjoint algorithm (Sec. 3.2.1):
``set_initial`` (initial lattices), ``forward(g)``, ``adjoint(g)`` (AMRT sweep
with the gradient assembled in the same kernel), ``gradient(g)`` and ``step``
(one steepest-descent iteration with Armijo backtracking).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from .workloads import Workload


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Problem:
    """One lattice problem bound to a caller-owned workspace and a stream."""

    def __init__(self, w: Workload, device="cuda", stream: torch.cuda.Stream | None = None, precision=None):
        self.lib = _lib.load()
        self.w = w
        self.device = torch.device(device)
        if self.device.type == "cuda" and self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.precision = precision or w.precision
        self.dtype = torch.float64 if self.precision == 64 else torch.float32
        self.stream = stream or torch.cuda.current_stream(self.device)
        self.N = w.N
        self.ctrl_shape = w.ctrl_shape
        dev = self.device
        d, keep = make_desc(w, dev, self.precision)
        self.desc = d
        self._desc_arrays = keep  # the descriptor's device arrays stay valid with the Problem
        nbytes = ctypes.c_size_t(0)
        _lib.check(self.lib.cx_workspace_size(ctypes.byref(d), ctypes.byref(nbytes)), "cx_workspace_size")
        self.workspace_bytes = nbytes.value
        with torch.cuda.device(dev):
            self.ws = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=dev)
        h = ctypes.c_void_p()
        _lib.check(self.lib.cx_create(ctypes.byref(d), _ptr(self.ws), nbytes.value,
                                      ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)), "cx_create")
        self.h = h
        self.generation = 0  # counts forward solves (the checkpoints belong to the latest one)
        self._J = torch.zeros(1, dtype=torch.float64, device=dev)
        self.set_initial(w.u0, w.v0)

    # ------------------------------------------------------------ helpers
    def _t(self, a, shape=None):
        """Device tensor of the problem's dtype (numpy or torch input)."""
        if a is None:
            return None
        t = torch.as_tensor(a, device=self.device)
        if t.dtype != self.dtype:
            t = t.to(self.dtype)
        t = t.contiguous()
        if shape is not None and tuple(t.shape) != tuple(shape):
            raise ValueError(f"expected shape {shape}, got {tuple(t.shape)}")
        return t

    def zeros_control(self):
        return torch.zeros(self.ctrl_shape, dtype=self.dtype, device=self.device)

    # ------------------------------------------------------------ calls
    def set_initial(self, u0, v0):
        u0 = self._t(u0, (self.w.ny, self.w.nx))
        v0 = self._t(v0, (self.w.ny, self.w.nx))
        _lib.check(self.lib.cx_set_initial(self.h, _ptr(u0), _ptr(v0)), "cx_set_initial")
        self._keep_init = (u0, v0)

    def forward(self, g=None):
        """Forward solve; returns the FP64 cost J as a 1-element device tensor."""
        g = self._t(g, self.ctrl_shape)
        _lib.check(self.lib.cx_forward(self.h, _ptr(g), _ptr(self._J)), "cx_forward")
        self._g_fwd = g
        self.generation += 1
        return self._J

    def adjoint(self, g=None, seed_u=None, seed_v=None, out=None):
        """AMRT adjoint sweep; returns dJ/dg (device tensor, control shape)."""
        g = self._t(g, self.ctrl_shape)
        su = self._t(seed_u, (self.w.ny, self.w.nx))
        sv = self._t(seed_v, (self.w.ny, self.w.nx))
        out = out if out is not None else torch.empty(self.ctrl_shape, dtype=self.dtype, device=self.device)
        _lib.check(self.lib.cx_adjoint(self.h, _ptr(g), _ptr(su), _ptr(sv), _ptr(out)), "cx_adjoint")
        self._keep_adj = (g, su, sv)  # inputs stay alive until the queued work has read them
        return out

    def vjp(self, g=None, seed_u=None, seed_v=None, out=None):
        """Vector-Jacobian product (du^N/dg)^T seed_u + (dv^N/dg)^T seed_v of
        the last forward's solve (no penalty term; None seeds are zero)."""
        g = self._t(g, self.ctrl_shape)
        su = self._t(seed_u, (self.w.ny, self.w.nx))
        sv = self._t(seed_v, (self.w.ny, self.w.nx))
        out = out if out is not None else torch.empty(self.ctrl_shape, dtype=self.dtype, device=self.device)
        _lib.check(self.lib.cx_adjoint_vjp(self.h, _ptr(g), _ptr(su), _ptr(sv), _ptr(out)), "cx_adjoint_vjp")
        self._keep_adj = (g, su, sv)
        return out

    def gradient(self, g=None, out=None):
        g = self._t(g, self.ctrl_shape)
        out = out if out is not None else torch.empty(self.ctrl_shape, dtype=self.dtype, device=self.device)
        _lib.check(self.lib.cx_gradient(self.h, _ptr(g), _ptr(out), _ptr(self._J)), "cx_gradient")
        self.generation += 1
        return self._J, out

    def gradient_host(self, g_host, out_host, g_dev=None, E_dev=None):
        """J and dJ/dg with the control and the gradient in host memory
        (cx_gradient_host): g_host and out_host are CPU tensors of the control's
        shape and dtype (pinned for the copies to overlap the kernels); g_dev
        and E_dev are the device buffers the call works in (allocated here
        when not given).  Returns J (float)."""
        for t in (g_host, out_host):
            if t.device.type != "cpu" or t.dtype != self.dtype or not t.is_contiguous() or \
                    tuple(t.shape) != tuple(self.ctrl_shape):
                raise ValueError("host buffers must be contiguous CPU tensors of the control's shape and dtype")
        g_dev = g_dev if g_dev is not None else torch.empty(self.ctrl_shape, dtype=self.dtype, device=self.device)
        E_dev = E_dev if E_dev is not None else torch.empty(self.ctrl_shape, dtype=self.dtype, device=self.device)
        J = ctypes.c_double(0.0)
        _lib.check(self.lib.cx_gradient_host(self.h, ctypes.c_void_p(g_host.data_ptr()),
                                             ctypes.c_void_p(out_host.data_ptr()), ctypes.byref(J), _ptr(g_dev),
                                             _ptr(E_dev)), "cx_gradient_host")
        self.generation += 1
        return J.value

    def step(self, g, E=None):
        """One Armijo steepest-descent iteration, g updated in place."""
        if g.dtype != self.dtype or not g.is_contiguous() or g.device != self.device or \
                tuple(g.shape) != tuple(self.ctrl_shape):
            raise ValueError("g must be a contiguous device tensor of the problem's dtype")
        E = E if E is not None else torch.empty_like(g)
        info = _lib.StepInfo()
        _lib.check(self.lib.cx_step(self.h, _ptr(g), _ptr(E), ctypes.byref(info)), "cx_step")
        self.generation += 1
        return dict(J0=info.J0, J=info.J, lam=info.lam, grad_sq=info.grad_sq, grad_inf=info.grad_inf,
                    trials=info.trials)

    def cg_step(self, g, variant="PR"):
        """One nonlinear conjugate-gradient iteration (Wolfe-Powell search), g
        updated in place; the iteration state (gradients, direction) stays in
        a work buffer of this object until cg_reset()."""
        if g.dtype != self.dtype or not g.is_contiguous() or g.device != self.device or \
                tuple(g.shape) != tuple(self.ctrl_shape):
            raise ValueError("g must be a contiguous device tensor of the problem's dtype")
        if getattr(self, "_cg_work", None) is None:
            self._cg_work = torch.empty((4,) + tuple(self.ctrl_shape), dtype=self.dtype, device=self.device)
        info = _lib.CGInfo()
        _lib.check(self.lib.cx_cg_step(self.h, _ptr(g), _ptr(self._cg_work), _lib.CG_VARIANTS[variant],
                                       ctypes.byref(info)), "cx_cg_step")
        self.generation += 1
        return dict(J0=info.J0, J=info.J, lam=info.lam, grad_sq=info.grad_sq, r=info.beta, trials=info.trials,
                    restarted=bool(info.restarted))

    def tlm(self, g, dg):
        """Sensitivity (du^N, dv^N, ||du^N||^2) of the last forward's trajectory
        (control g) along the direction dg."""
        g = None if g is None else self._t(g, self.ctrl_shape)
        dg = self._t(dg, self.ctrl_shape)
        du = torch.empty((self.w.ny, self.w.nx), dtype=self.dtype, device=self.device)
        dv = torch.empty_like(du)
        sq = ctypes.c_double()
        _lib.check(self.lib.cx_tlm(self.h, _ptr(g), _ptr(dg), _ptr(du), _ptr(dv), ctypes.byref(sq)), "cx_tlm")
        return du, dv, sq.value

    def cadjoint(self, g, out=None):
        """Continuous-adjoint gradient (time-reversed MRT solve of the adjoint
        PDE) at the control of the last forward."""
        g = None if g is None else self._t(g, self.ctrl_shape)
        out = out if out is not None else torch.empty(self.ctrl_shape, dtype=self.dtype, device=self.device)
        _lib.check(self.lib.cx_cadjoint(self.h, _ptr(g), _ptr(out)), "cx_cadjoint")
        return out

    def lma_step(self, g, E=None):
        """One steepest-descent iteration with the linearised (sensitivity)
        line search, g updated in place."""
        if g.dtype != self.dtype or not g.is_contiguous() or g.device != self.device or \
                tuple(g.shape) != tuple(self.ctrl_shape):
            raise ValueError("g must be a contiguous device tensor of the problem's dtype")
        E = E if E is not None else torch.empty_like(g)
        info = _lib.StepInfo()
        _lib.check(self.lib.cx_lma_step(self.h, _ptr(g), _ptr(E), ctypes.byref(info)), "cx_lma_step")
        self.generation += 1
        return dict(J0=info.J0, J=info.J, lam=info.lam, grad_sq=info.grad_sq, grad_inf=info.grad_inf,
                    trials=info.trials)

    def cg_reset(self):
        _lib.check(self.lib.cx_cg_reset(self.h), "cx_cg_reset")

    def fields(self):
        u = torch.empty((self.w.ny, self.w.nx), dtype=self.dtype, device=self.device)
        v = torch.empty_like(u)
        _lib.check(self.lib.cx_get_fields(self.h, _ptr(u), _ptr(v)), "cx_get_fields")
        return u, v

    def psi0(self):
        out = torch.empty((2, self.w.Q, self.w.ny, self.w.nx), dtype=self.dtype, device=self.device)
        _lib.check(self.lib.cx_get_psi0(self.h, _ptr(out)), "cx_get_psi0")
        return out

    def norms(self):
        J, e2, einf = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _lib.check(self.lib.cx_get_norms(self.h, ctypes.byref(J), ctypes.byref(e2), ctypes.byref(einf)),
                   "cx_get_norms")
        return J.value, e2.value, einf.value

    def set_launch(self, bx, by):
        _lib.check(self.lib.cx_set_launch(self.h, bx, by), "cx_set_launch")

    def set_staging(self, row_windows=True):
        """Bulk row-window staging of the lattice kernels (True, the default)
        or per-thread copies everywhere (False); results are identical."""
        _lib.check(self.lib.cx_set_staging(self.h, 1 if row_windows else 0), "cx_set_staging")

    def set_timing(self, on=True):
        _lib.check(self.lib.cx_set_timing(self.h, 1 if on else 0), "cx_set_timing")

    def timing(self):
        ms = (ctypes.c_double * 4)()
        cnt = (ctypes.c_longlong * 4)()
        _lib.check(self.lib.cx_get_timing(self.h, ms, cnt), "cx_get_timing")
        names = ("forward", "recompute", "adjoint", "other")
        return {n: (ms[i], cnt[i]) for i, n in enumerate(names)}

    def close(self):
        if getattr(self, "h", None):
            self.lib.cx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_desc(w: Workload, dev, precision=None):
    """cx_problem_desc for a workload; returns (desc, device arrays it points to).

    The arrays must stay alive while the library may read them (until cx_create
    or the static forward's queued work has run)."""
    precision = precision or w.precision
    f64 = lambda a: None if a is None else torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    u8 = lambda a: None if a is None else torch.as_tensor(np.ascontiguousarray(a, dtype=np.uint8), device=dev)
    keep = {}
    d = _lib.Desc()
    d.nx, d.ny, d.n_steps, d.lattice = w.nx, w.ny, w.N, w.Q
    d.precision = precision
    d.ckpt_every = w.ckpt_every or w.N
    d.tau = 1.0
    d.aniso = {"const": _lib.CX_ANISO_CONST, "rotated": _lib.CX_ANISO_ROTATED, "field": _lib.CX_ANISO_FIELD}[w.aniso]
    d.D_u = (ctypes.c_double * 3)(*w.D_u_const)
    d.D_v = (ctypes.c_double * 3)(*w.D_v_const)
    d.lam_u = (ctypes.c_double * 2)(*w.lam_u)
    d.lam_v = (ctypes.c_double * 2)(*w.lam_v)
    if w.aniso == "rotated":
        keep["theta"] = f64(w.theta)
        d.theta = _ptr(keep["theta"])
    if w.aniso == "field":
        keep["Du"], keep["Dv"] = f64(w.D_u_field), f64(w.D_v_field)
        d.D_u_field, d.D_v_field = _ptr(keep["Du"]), _ptr(keep["Dv"])
    d.d_u, d.d_v = w.d_u, w.d_v
    d.chi, d.r_vu, d.r_vv = w.chi, w.r_vu, w.r_vv
    d.adv = {"none": _lib.CX_ADV_NONE, "row": _lib.CX_ADV_ROW, "field": _lib.CX_ADV_FIELD}[w.adv]
    if w.adv == "row":
        keep["a"] = f64(w.a_row)
    elif w.adv == "field":
        keep["a"] = f64(w.a_field)
    d.a = _ptr(keep.get("a"))
    if w.solid is not None:
        keep["solid"] = u8(w.solid)
        d.solid = _ptr(keep["solid"])
    if w.window is not None:
        d.ctrl_x0, d.ctrl_y0, d.ctrl_nx, d.ctrl_ny = w.window
    if w.cmask is not None:
        keep["cmask"] = u8(w.cmask)
        d.ctrl_mask = _ptr(keep["cmask"])
    keep["ut"] = f64(w.u_tgt)
    d.u_target = _ptr(keep["ut"])
    d.alpha = w.alpha
    d.s = (ctypes.c_double * 7)(*w.s)
    d.source_order = w.source_order
    d.ctrl_windows = w.windows
    d.halo = w.halo
    return d, keep
