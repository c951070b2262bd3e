"""torch.autograd binding of the compressed operator: the forward is the
library's apply, the backward its adjoint (conjugate-transpose) apply, both
through the C ABI (marshalling only; no arithmetic here).

For a real loss L of complex inputs PyTorch propagates dL/dz* (the conjugate
Wirtinger derivative); for Y = C X that is dL/dX* = C^H dL/dY*, which is
what bem_op_apply with transpose = 1 computes (Eq. (3.15) transposed).
"""
from __future__ import annotations

import torch

from . import BEM_APPLY_BATCHED, BEM_APPLY_CONTRACTED, Operator


class OperatorApply(torch.autograd.Function):
    """Y = C(s_k) X_k for all k (BATCHED, Y: K x n_rows x 3) or
    y = sum_k C(s_k) X_k (CONTRACTED, y: n_rows x 3); X: K x n_cols x 3,
    complex of the operator's precision on its device."""

    @staticmethod
    def forward(ctx, X: torch.Tensor, op: Operator, mode: int = BEM_APPLY_BATCHED) -> torch.Tensor:
        X = X.contiguous()
        t = op.tree
        shape = (op.K, t.n_rows, 3) if mode == BEM_APPLY_BATCHED else (t.n_rows, 3)
        Y = torch.empty(shape, dtype=X.dtype, device=X.device)
        op.apply(X, Y, mode)
        ctx.op = op
        ctx.mode = mode
        ctx.xshape = X.shape
        return Y

    @staticmethod
    def backward(ctx, gY: torch.Tensor):
        op = ctx.op
        gX = torch.empty(ctx.xshape, dtype=gY.dtype, device=gY.device)
        op.apply_adjoint(gY.contiguous(), gX, ctx.mode)
        return gX, None, None


def apply(op: Operator, X: torch.Tensor, mode: int = BEM_APPLY_BATCHED) -> torch.Tensor:
    """Differentiable apply of a compressed operator."""
    return OperatorApply.apply(X, op, mode)


__all__ = ["OperatorApply", "apply", "BEM_APPLY_BATCHED", "BEM_APPLY_CONTRACTED"]
