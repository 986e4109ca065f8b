"""torch.autograd.Function over the library: u, grad u = path(u_hat, x), with the
adjoint entry point (bspline_spread_adjoint) as the backward.

Gradient convention for the complex half spectrum: dL/dRe + i dL/dIm, the
one PyTorch uses for its real-to-complex transforms.  Argument marshalling
only; both directions run in the library's CUDA kernels.
"""
from __future__ import annotations

import torch

from .bspline import Plan


class BSplineInterp(torch.autograd.Function):
    """apply(u_hat, x, plan) -> (u [P, 3], grad [P, 3, 3])."""

    @staticmethod
    def forward(ctx, u_hat, x, plan: Plan):
        coef = plan.coeffs(u_hat.contiguous())
        u, g = plan.interp(coef, x.contiguous())
        ctx.plan = plan
        ctx.save_for_backward(x, coef)
        return u, g

    @staticmethod
    def backward(ctx, g_u, g_grad):
        x, coef = ctx.saved_tensors
        plan = ctx.plan
        need_uhat, need_x = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (need_uhat or need_x):
            return None, None, None
        g_u = g_u.contiguous() if g_u is not None else None
        g_grad = g_grad.contiguous() if g_grad is not None else None
        g_u_hat, g_x, _ = plan.spread_adjoint(x.contiguous(), g_u, g_grad, coef=coef if need_x else None,
                                              u_hat_grad=need_uhat)
        return g_u_hat, g_x, None


def interpolate(u_hat, x, plan: Plan):
    """Differentiable u, grad u at x of the B-spline interpolant of the field u_hat."""
    return BSplineInterp.apply(u_hat, x, plan)
