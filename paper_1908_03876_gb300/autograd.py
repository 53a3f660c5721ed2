"""The MRT forward solve as a differentiable PyTorch function of the control.

``MRTSolve.apply(g, problem)`` returns (u^N, v^N).  Its backward is the AMRT
adjoint sweep (Sec. 3.2.1) seeded with the incoming gradients of u^N and v^N:
the reverse-time pass recomputes each checkpointed forward segment, so the
memory held between forward and backward is the problem's O(N/k) checkpoint
lattices, not the trajectory.  Both passes run in the CUDA library.

The library's seeded adjoint returns the gradient of
sum(seed_u u^N + seed_v v^N) + alpha ||g||^2; the penalty part 2 alpha g is
removed here so that the backward is the plain vector-Jacobian product of the
solve.
"""
from __future__ import annotations

import numpy as np
import torch

from .problem import Problem


def controlled_mask(problem: Problem) -> torch.Tensor:
    """1 on controlled nodes of the control window (window & mask & fluid)."""
    w = problem.w
    x0, y0, cnx, cny = w.win
    m = np.ones((cny, cnx))
    if w.cmask is not None:
        m = m * w.cmask
    if w.solid is not None:
        m = m * (1 - w.solid[y0:y0 + cny, x0:x0 + cnx])
    return torch.as_tensor(m, dtype=problem.dtype, device=problem.device)


class MRTSolve(torch.autograd.Function):
    """(u^N, v^N) = F(g) with F the coupled MRT forward solve."""

    @staticmethod
    def forward(ctx, g: torch.Tensor, problem: Problem):
        g = g.detach().to(problem.dtype).contiguous()
        problem.forward(g)
        u, v = problem.fields()
        ctx.problem = problem
        ctx.generation = problem.generation
        ctx.save_for_backward(g)
        return u, v

    @staticmethod
    def backward(ctx, grad_u, grad_v):
        (g,) = ctx.saved_tensors
        p: Problem = ctx.problem
        if p.generation != ctx.generation:
            # another forward ran on this problem since: restore its checkpoints
            p.forward(g)
        su = None if grad_u is None else grad_u.contiguous()
        sv = None if grad_v is None else grad_v.contiguous()
        if su is None:
            su = torch.zeros((p.w.ny, p.w.nx), dtype=p.dtype, device=p.device)
        E = p.adjoint(g, seed_u=su, seed_v=sv)
        if p.w.alpha:
            E = E - (2.0 * p.w.alpha) * g * controlled_mask(p)[None]
        return E, None


def solve(g: torch.Tensor, problem: Problem):
    """(u^N, v^N) as differentiable functions of g."""
    return MRTSolve.apply(g, problem)
