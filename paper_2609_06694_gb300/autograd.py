"""torch.autograd.Function wrappers pairing each sweep with its hand-written adjoint.

StencilSweep.apply(x, plan, steps)         y = A^steps x        (STENCIL_CONST plans)
VarStencilSweep.apply(x, plan, steps, *w)  y = A(w)^steps x     (STENCIL_VAR / DIVKGRAD plans)
The backward pass applies the transposed sweep (offsets flipped; for VAR the coefficient is
gathered at the shifted cell) to the incoming gradient.  Gradients with respect to the
coefficients are not provided.
"""
from __future__ import annotations

import torch

from . import api


class StencilSweep(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, plan, steps=1):
        ctx.plan, ctx.steps = plan, int(steps)
        y = torch.empty_like(x)
        api.stencil_apply(plan, x.contiguous(), y, ctx.steps)
        return y

    @staticmethod
    def backward(ctx, gy):
        gx = torch.empty_like(gy)
        api.stencil_apply_adjoint(ctx.plan, gy.contiguous(), gx, ctx.steps)
        return gx, None, None


class VarStencilSweep(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, plan, steps, *w):
        ctx.plan, ctx.steps = plan, int(steps)
        ctx.save_for_backward(*w)
        y = torch.empty_like(x)
        api.stencil_apply_var(plan, x.contiguous(), list(w), y, ctx.steps)
        return y

    @staticmethod
    def backward(ctx, gy):
        w = ctx.saved_tensors
        gx = torch.empty_like(gy)
        api.stencil_apply_adjoint_var(ctx.plan, gy.contiguous(), list(w), gx, ctx.steps)
        return (gx, None, None) + (None,) * len(w)
