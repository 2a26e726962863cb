"""PyTorch autograd wrapper of the batched solve and its hand-written adjoint.

    Y = abm_solve(plan, alpha, h, N, params, y0)   # (M, max(N)+1, d), FP64, CUDA
    loss(Y).backward()                             # params.grad, y0.grad via abm_adjoint

The backward pass calls abm_adjoint (reverse-time transposed history
convolution, Jacobians of f recomputed from the stored states); nothing is
differentiated by autograd inside the solver.  Rows of Y beyond N[i] are zero
and receive no gradient.
"""
from __future__ import annotations

import numpy as np
import torch

from . import abm as _abm


class _ABMSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, y0, plan, alpha, h, N):
        alpha = np.ascontiguousarray(alpha, dtype=np.float64)
        h = np.ascontiguousarray(h, dtype=np.float64)
        N = np.ascontiguousarray(N, dtype=np.int32)
        params = params.detach().contiguous()
        y0 = y0.detach().contiguous()
        ldY = int(N.max()) + 1
        Y = torch.zeros(len(alpha), ldY, plan.d, dtype=torch.float64, device=params.device)
        YP = torch.zeros_like(Y)
        plan.solve_batched(alpha, h, N, params, y0, Y=Y, YP=YP, ldY=ldY)
        ctx.plan, ctx.alpha, ctx.h, ctx.N = plan, alpha, h, N
        ctx.save_for_backward(params, y0, Y, YP)
        return Y

    @staticmethod
    def backward(ctx, dY):
        params, y0, Y, YP = ctx.saved_tensors
        dp, dy0 = ctx.plan.adjoint(ctx.alpha, ctx.h, ctx.N, params, y0, Y, YP, dY.contiguous())
        return dp, dy0, None, None, None, None


def abm_solve(plan, alpha, h, N, params: torch.Tensor, y0: torch.Tensor) -> torch.Tensor:
    """Differentiable batched solve: gradients flow to params and y0."""
    return _ABMSolve.apply(params, y0, plan, alpha, h, N)
