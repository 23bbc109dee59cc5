"""torch.autograd binding of the structure-factor loss.

`structure_factor_loss(points, plan)` returns L (Eq. 2) as a differentiable scalar: its forward
is fresco_forward (sort, spread, FFT, deconvolve, loss: the type-1 half) and its hand-written
backward is fresco_backward (inverse FFT and interpolation: the type-2 half of Eq. 4), scaled by
the incoming gradient on the device. Torch only routes the call; all arithmetic runs in
libfresco. A plan holds the gradient coefficients of its last forward, so each forward must be
followed by its backward before the plan evaluates again.
"""

from __future__ import annotations

import torch


class StructureFactorLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, points, plan):
        loss = plan.forward(points.contiguous())
        ctx.plan = plan
        ctx.points_shape = points.shape
        return loss

    @staticmethod
    def backward(ctx, grad_out):
        grad = ctx.plan.backward(grad_out)
        return grad.reshape(ctx.points_shape), None


def structure_factor_loss(points: torch.Tensor, plan) -> torch.Tensor:
    """L(points) for a fresco.Plan built for points.shape[0] points; differentiable in points."""
    return StructureFactorLoss.apply(points, plan)
