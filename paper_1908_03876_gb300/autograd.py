"""The MRT forward solve as a differentiable PyTorch function of the control.

``MRTSolve.apply(g, problem)`` returns (u^N, v^N).  Its backward is the AMRT
adjoint sweep (Sec. 3.2.1) seeded with the incoming gradients of u^N and v^N:
the reverse-time pass recomputes each checkpointed forward segment, so the
memory held between forward and backward is the problem's O(N/k) checkpoint
lattices, not the trajectory.  Both passes run in the CUDA library.

The backward calls the library's vector-Jacobian product (cx_adjoint_vjp):
the seeded AMRT sweep without the control-penalty term, summed over each
window's steps for time-windowed controls.  No arithmetic of the method runs
here.
"""
from __future__ import annotations

import torch

from .problem import Problem


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
        return p.vjp(g, seed_u=su, seed_v=sv), None


def solve(g: torch.Tensor, problem: Problem):
    """(u^N, v^N) as differentiable functions of g."""
    return MRTSolve.apply(g, problem)
