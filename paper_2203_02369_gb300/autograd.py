"""torch.autograd face of the HAMLET potential.

``logpost(problem, w, d)`` returns Psi(w, d) (eq. Psi) as a 0-d float64
tensor; its backward pass returns the hand-derived adjoint gradient that
libhamlet computes in the same call (no second pass, no tape).
"""
from __future__ import annotations

import torch


class HamletLogPost(torch.autograd.Function):
    """forward(w, d, problem) -> Psi; backward -> (g * dPsi/dw, g * dPsi/dd)."""

    @staticmethod
    def forward(ctx, w, d, problem):
        psi, gw, gd = problem.logpost_grad(w.detach(), d.detach())
        ctx.save_for_backward(gw.to(w.dtype), gd.to(d.dtype))
        return psi

    @staticmethod
    def backward(ctx, grad_out):
        gw, gd = ctx.saved_tensors
        g = grad_out.to(torch.float64)
        return (g.to(gw.dtype) * gw if ctx.needs_input_grad[0] else None,
                g.to(gd.dtype) * gd if ctx.needs_input_grad[1] else None,
                None)


def logpost(problem, w, d):
    return HamletLogPost.apply(w, d, problem)
