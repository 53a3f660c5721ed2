"""Domain decomposition of one control problem over 2-D blocks.

Collision is local and streaming reaches only the nearest neighbours (Sec. 3.1;
the adjoint of Sec. 3.2.1 streams the other way), so the lattice splits into
px x py blocks, one per rank, that exchange one-node halos before every step.
Each block is a library problem over its lx x ly interior plus a one-node frame
(descriptor field halo = 1); the library calls back after every lattice step
and the callback here packs the crossing populations with the library's
kernels, moves the slots between ranks, and unpacks them into the frame.

Transport: torch.distributed point-to-point (NCCL with device buffers; gloo
with host buffers, as in the tests); a rank that is its own neighbour (one
block along an axis) copies the slot to itself.  Messages carry the direction
as their tag, and every rank posts its sends and receives in direction order,
so they also pair up in order where tags are ignored.

Sums over blocks (the cost, ||dJ/dg||^2) are FP64 all-reduces, the maximum
|dJ/dg| a max-reduce; the Armijo iteration of cx_step runs here on those
global values (the library's own cx_step would use one block's cost).

Only argument marshalling and data movement run in Python; every step of the
method runs in the library's kernels.
"""
from __future__ import annotations

import ctypes
from dataclasses import replace

import numpy as np
import torch

from . import _lib
from .problem import Problem, _ptr
from .workloads import Workload

# D2Q9 velocities e_1..e_8 (E, N, W, S, NE, NW, SW, SE): the neighbour directions
DIRS = {1: (1, 0), 2: (0, 1), 3: (-1, 0), 4: (0, -1), 5: (1, 1), 6: (-1, 1), 7: (-1, -1), 8: (1, -1)}
OPP = {1: 3, 2: 4, 3: 1, 4: 2, 5: 7, 6: 8, 7: 5, 8: 6}


class Partition:
    """px x py blocks of an nx x ny periodic grid; rank = by * px + bx.
    Block sizes differ by at most one node along each axis."""

    def __init__(self, nx: int, ny: int, px: int, py: int):
        if px < 1 or py < 1 or nx < px or ny < py:
            raise ValueError("every block needs at least one node along each axis")
        self.nx, self.ny, self.px, self.py = nx, ny, px, py
        self.xs = [nx * i // px for i in range(px + 1)]
        self.ys = [ny * j // py for j in range(py + 1)]

    @property
    def size(self):
        return self.px * self.py

    def coords(self, rank):
        return rank % self.px, rank // self.px

    def block(self, rank):
        """(x0, y0, lx, ly): the block's interior in global coordinates."""
        bx, by = self.coords(rank)
        return self.xs[bx], self.ys[by], self.xs[bx + 1] - self.xs[bx], self.ys[by + 1] - self.ys[by]

    def neighbour(self, rank, d):
        """Rank of the block at offset e_d (periodic)."""
        bx, by = self.coords(rank)
        dx, dy = DIRS[d]
        return ((by + dy) % self.py) * self.px + (bx + dx) % self.px


def _frame(a, x0, y0, lx, ly):
    """The block's interior and one-node frame of a global per-node array
    ([ny][nx][...]), with periodic images at the grid's edges."""
    ny, nx = a.shape[:2]
    ys = (np.arange(y0 - 1, y0 + ly + 1) % ny)[:, None]
    xs = (np.arange(x0 - 1, x0 + lx + 1) % nx)[None, :]
    return np.ascontiguousarray(a[ys, xs])


def block_workload(w: Workload, part: Partition, rank: int) -> Workload:
    """The sub-problem of block `rank`: (lx + 2) x (ly + 2) nodes whose frame is
    a halo, every per-node field taken over the interior and frame, and the
    control window the part of the global window inside the interior (local
    control shape [W][lcny][lcnx]).  A block without controlled nodes gets a
    one-node window on a frame corner, which is never controlled."""
    x0, y0, lx, ly = part.block(rank)
    f = lambda a: None if a is None else _frame(a, x0, y0, lx, ly)
    wx0, wy0, wcx, wcy = w.win
    cx0, cx1 = max(wx0, x0), min(wx0 + wcx, x0 + lx)
    cy0, cy1 = max(wy0, y0), min(wy0 + wcy, y0 + ly)
    if cx1 > cx0 and cy1 > cy0:
        window = (cx0 - x0 + 1, cy0 - y0 + 1, cx1 - cx0, cy1 - cy0)
        cmask = None if w.cmask is None else np.ascontiguousarray(w.cmask[cy0 - wy0:cy1 - wy0, cx0 - wx0:cx1 - wx0])
        ctrl = (cx0 - wx0, cy0 - wy0, cx1 - cx0, cy1 - cy0)  # the slice of the global control array
    else:
        window, cmask, ctrl = (0, 0, 1, 1), None, None
    a_row = None if w.a_row is None else np.ascontiguousarray(w.a_row[np.arange(y0 - 1, y0 + ly + 1) % w.ny])
    sub = replace(w, name=f"{w.name}[block {rank}]", nx=lx + 2, ny=ly + 2, theta=f(w.theta),
                  D_u_field=f(w.D_u_field), D_v_field=f(w.D_v_field), a_row=a_row, a_field=f(w.a_field),
                  solid=f(w.solid), u0=f(w.u0), v0=f(w.v0), u_tgt=f(w.u_tgt), window=window, cmask=cmask,
                  halo=1, extra=dict(w.extra, block=(x0, y0, lx, ly), ctrl_slice=ctrl))
    return sub


class HaloExchange:
    """The library's exchange callback for one block: pack (library kernel),
    move the eight slots to and from the neighbouring ranks, unpack (library
    kernel) into the frame, all ordered on the block's stream."""

    def __init__(self, prob: Problem, part: Partition, rank: int, group=None):
        self.prob, self.part, self.rank, self.group = prob, part, rank, group
        self.lib = prob.lib
        if part.size > 1 and not torch.distributed.is_initialized():
            raise RuntimeError("a partition of several blocks needs an initialised torch.distributed group")
        self.dist = torch.distributed if part.size > 1 else None
        self.host = self.dist is not None and self.dist.get_backend(group) == "gloo"
        self.layout = {}
        for kind in (_lib.CX_HALO_FWD, _lib.CX_HALO_ADJ, _lib.CX_HALO_SEED):
            so, ro = (ctypes.c_size_t * 8)(), (ctypes.c_size_t * 8)()
            nb = ctypes.c_size_t()
            _lib.check(self.lib.cx_halo_layout(prob.h, kind, so, ro, ctypes.byref(nb)), "cx_halo_layout")
            self.layout[kind] = (list(so), list(ro), nb.value)
        nbytes = max(v[2] for v in self.layout.values())
        dev = prob.device
        self.send = torch.empty(max(nbytes, 16), dtype=torch.uint8, device=dev)
        self.recv = torch.empty_like(self.send)
        if self.host:
            self.send_h = torch.empty(self.send.shape, dtype=torch.uint8, pin_memory=True)
            self.recv_h = torch.empty_like(self.send_h, pin_memory=True)
        self.error = None
        self._cb = _lib.HALO_FN(self._callback)  # kept alive with the object
        _lib.check(self.lib.cx_set_halo_exchange(prob.h, self._cb, None), "cx_set_halo_exchange")

    def close(self):
        if getattr(self, "prob", None) is not None and self.prob.h:
            self.lib.cx_set_halo_exchange(self.prob.h, None, None)

    def exchange(self, kind: int, field_ptr: int):
        """Fill the frame of the device field at field_ptr (the kind's layout)."""
        p = self.prob
        send_off, recv_off, nbytes = self.layout[kind]
        _lib.check(self.lib.cx_halo_pack(p.h, kind, ctypes.c_void_p(field_ptr), _ptr(self.send)), "cx_halo_pack")
        ends_s = send_off[1:] + [nbytes]
        ends_r = recv_off[1:] + [nbytes]
        if self.dist is None:
            with torch.cuda.stream(p.stream):
                for d in range(1, 9):  # every neighbour is this block itself
                    o = OPP[d]
                    self.recv[recv_off[o - 1]:ends_r[o - 1]].copy_(self.send[send_off[d - 1]:ends_s[d - 1]])
        else:
            if self.host:
                with torch.cuda.stream(p.stream):
                    self.send_h[:nbytes].copy_(self.send[:nbytes], non_blocking=True)
                p.stream.synchronize()
                sbuf, rbuf = self.send_h, self.recv_h
            else:
                p.stream.synchronize()
                sbuf, rbuf = self.send, self.recv
            exchange_slots(sbuf, rbuf, send_off, recv_off, nbytes, self.part, self.rank, self.group)
            if self.host:
                with torch.cuda.stream(p.stream):
                    self.recv[:nbytes].copy_(self.recv_h[:nbytes], non_blocking=True)
        _lib.check(self.lib.cx_halo_unpack(p.h, kind, _ptr(self.recv), ctypes.c_void_p(field_ptr)), "cx_halo_unpack")

    def _callback(self, user, kind, field, stream):
        try:
            self.exchange(kind, field)
            return 0
        except Exception as exc:  # reported to the library as an internal error; kept for the caller
            self.error = exc
            return 8


def exchange_slots(send, recv, send_off, recv_off, nbytes, part: Partition, rank: int, group=None):
    """Send slot d of `send` to the block at e_d and receive, into slot d of
    `recv`, what the block at e_d sent toward this one (its slot opp(d)).
    send / recv: uint8 tensors (host for gloo, device for NCCL); offsets in bytes."""
    dist = torch.distributed
    ends_s = list(send_off[1:]) + [nbytes]
    ends_r = list(recv_off[1:]) + [nbytes]
    reqs = []
    for d in range(1, 9):  # receives first, then sends, both in direction order
        src = part.neighbour(rank, d)
        if src == rank:
            continue
        buf = recv[recv_off[d - 1]:ends_r[d - 1]]
        if buf.numel():
            reqs.append(dist.irecv(buf, src=src, group=group, tag=OPP[d]))
    for d in range(1, 9):
        dst = part.neighbour(rank, d)
        chunk = send[send_off[d - 1]:ends_s[d - 1]]
        if dst == rank:
            o = OPP[d]
            recv[recv_off[o - 1]:ends_r[o - 1]].copy_(chunk)
        elif chunk.numel():
            reqs.append(dist.isend(chunk, dst=dst, group=group, tag=d))
    for r in reqs:
        r.wait()


class DecomposedProblem:
    """One block of a decomposed problem on this rank: forward solve, AMRT
    gradient, vector-Jacobian product and the Armijo iteration over the whole
    problem, with the block's halos exchanged after every step.

    Controls and gradients are the block's part of the global window
    ([W][lcny][lcnx]); fields are the block's interior."""

    def __init__(self, w: Workload, part: Partition, rank: int, device="cuda", group=None):
        self.w_global, self.part, self.rank, self.group = w, part, rank, group
        self.w = block_workload(w, part, rank)
        self.prob = Problem(self.w, device=device)
        self.halo = HaloExchange(self.prob, part, rank, group)
        self.dist = self.halo.dist
        self.device = self.prob.device
        self.dtype = self.prob.dtype
        self.ctrl_shape = self.prob.ctrl_shape
        self.lam_prev = None
        self._J_at_g = None  # global J when the block's forward state is that of the current control

    def _run(self, fn, *args):
        """A library call whose exchanges may fail: re-raise the callback's error."""
        try:
            return fn(*args)
        except _lib.CxError:
            if self.halo.error is not None:
                err, self.halo.error = self.halo.error, None
                raise err
            raise

    def close(self):
        self.halo.close()
        self.prob.close()

    # ---- global reductions (FP64)
    def _sum(self, x: float) -> float:
        if self.dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64)
        if not self.halo.host:
            t = t.to(self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return float(t.item())

    def _max(self, x: float) -> float:
        if self.dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64)
        if not self.halo.host:
            t = t.to(self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return float(t.item())

    def local_control(self, g_global):
        """The block's part of a global control array [W][cny][cnx]."""
        sl = self.w.extra["ctrl_slice"]
        if sl is None:
            return np.zeros(self.ctrl_shape)
        cx, cy, nx, ny = sl
        return np.ascontiguousarray(np.asarray(g_global)[:, cy:cy + ny, cx:cx + nx])

    # ---- calls
    def forward(self, g=None) -> float:
        """Global cost J(g)."""
        self._run(self.prob.forward, g)
        J, _, _ = self.prob.norms()
        self._J_at_g = None
        return self._sum(J)

    def gradient(self, g=None, out=None):
        """(global J, the block's dJ/dg)."""
        _, E = self._run(self.prob.gradient, g, out)
        Jl, _, _ = self.prob.norms()
        self._J_at_g = None
        return self._sum(Jl), E

    def fields(self):
        """u^N, v^N on the block's interior."""
        u, v = self.prob.fields()
        return u[1:-1, 1:-1], v[1:-1, 1:-1]

    def vjp(self, g, seed_u=None, seed_v=None):
        """(du^N/dg)^T seed_u + (dv^N/dg)^T seed_v for interior seeds [ly][lx]
        (None: zero), after forward(g)."""
        seeds = []
        for s in (seed_u, seed_v):
            if s is None:
                seeds.append(None)
                continue
            full = torch.zeros((self.w.ny, self.w.nx), dtype=self.dtype, device=self.device)
            full[1:-1, 1:-1] = torch.as_tensor(s, dtype=self.dtype, device=self.device)
            with torch.cuda.stream(self.prob.stream):
                self.halo.exchange(_lib.CX_HALO_SEED, full.data_ptr())
            seeds.append(full)
        return self._run(self.prob.vjp, g, seeds[0], seeds[1])

    def step(self, g: torch.Tensor, E: torch.Tensor | None = None, c1=1e-4, max_trials=30):
        """One Armijo steepest-descent iteration over the whole problem (the rule
        of cx_step on the global J, ||E||^2 and max |E|); g updated in place."""
        lib, h = self.prob.lib, self.prob.h
        E = E if E is not None else torch.empty_like(g)
        if self._J_at_g is not None:  # the accepted trial's forward state is the control's: adjoint only
            J0 = self._J_at_g
            self._run(self.prob.adjoint, g, None, None, E)
        else:
            J0, _ = self.gradient(g, out=E)
        _, e2, einf = self.prob.norms()
        e2, einf = self._sum(e2), self._max(einf)
        lam = 2.0 * self.lam_prev if self.lam_prev else min(1.0, 1.0 / einf if einf > 0 else 1.0)
        Jd = torch.zeros(1, dtype=torch.float64, device=self.device)
        for t in range(max_trials):
            self._run(lambda: _lib.check(lib.cx_forward_trial(h, _ptr(g), _ptr(E), lam, _ptr(Jd)),
                                         "cx_forward_trial"))
            Jl, _, _ = self.prob.norms()
            Jt = self._sum(Jl)
            if np.isfinite(Jt) and Jt <= J0 - c1 * lam * e2:
                _lib.check(lib.cx_control_axpy(h, _ptr(g), _ptr(E), lam), "cx_control_axpy")
                self.lam_prev = lam
                self._J_at_g = Jt
                return dict(J0=J0, J=Jt, lam=lam, grad_sq=e2, grad_inf=einf, trials=t + 1)
            lam *= 0.5
        self._J_at_g = None
        raise _lib.CxError(6, "decomposed step")
