"""torch.autograd binding of the compressed operator: the forward is the
library's apply, the backward its adjoint (conjugate-transpose) apply, both
through the C ABI (marshalling only; no arithmetic here).

For a real loss L of complex inputs PyTorch propagates dL/dz* (the conjugate
Wirtinger derivative); for Y = C X that is dL/dX* = C^H dL/dY*, which is
what bem_op_apply with transpose = 1 computes (Eq. (3.15) transposed).

Wave-speed gradients (the adjoint method): for Y = V(c) X with c = (c_p,
c_s) at fixed density, dL/dc_a = Re <G, dV/dc_a X> with G PyTorch's
gradient of Y; bem_op_inner evaluates it on the compressed derivative
operators (kernels BEM_SL_DCP, BEM_SL_DCS).
"""
from __future__ import annotations

import torch

from . import BEM_APPLY_BATCHED, BEM_APPLY_CONTRACTED, Operator, receiver_energy_grad


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


class WaveSpeedApply(torch.autograd.Function):
    """Y = V(c) X of a single-layer operator, differentiable in X (adjoint
    apply) and in the wave speeds c = (c_p, c_s) (real tensor of shape (2,),
    the speeds the operators were compressed at; its value is not read).
    dops = (dV/dc_p, dV/dc_s): operators of kernels BEM_SL_DCP, BEM_SL_DCS on
    the same mesh, rows and frequencies."""

    @staticmethod
    def forward(ctx, X: torch.Tensor, c: torch.Tensor, op: Operator, dops, mode: int = BEM_APPLY_BATCHED):
        X = X.contiguous()
        t = op.tree
        shape = (op.K, t.n_rows, 3) if mode == BEM_APPLY_BATCHED else (t.n_rows, 3)
        Y = torch.empty(shape, dtype=X.dtype, device=X.device)
        op.apply(X, Y, mode)
        ctx.save_for_backward(X)
        ctx.op, ctx.dops, ctx.mode, ctx.cdev, ctx.cdt = op, dops, mode, c.device, c.dtype
        return Y

    @staticmethod
    def backward(ctx, gY: torch.Tensor):
        (X,) = ctx.saved_tensors
        gY = gY.contiguous()
        gX = gc = None
        if ctx.needs_input_grad[0]:
            gX = torch.empty(X.shape, dtype=gY.dtype, device=gY.device)
            ctx.op.apply_adjoint(gY, gX, ctx.mode)
        if ctx.needs_input_grad[1]:
            gc = torch.tensor([d.inner(gY, X, ctx.mode).real for d in ctx.dops], dtype=ctx.cdt, device=ctx.cdev)
        return gX, gc, None, None, None


def apply_speeds(op: Operator, dops, X: torch.Tensor, c: torch.Tensor,
                 mode: int = BEM_APPLY_BATCHED) -> torch.Tensor:
    """Differentiable apply of V(c) with gradients to X and to c = (c_p, c_s)."""
    return WaveSpeedApply.apply(X, c, op, tuple(dops), mode)


__all__ = ["OperatorApply", "WaveSpeedApply", "apply", "apply_speeds", "BEM_APPLY_BATCHED",
           "BEM_APPLY_CONTRACTED"]


class ReceiverEnergy(torch.autograd.Function):
    """J(g, c) = dt sum_n sum_r |u_n[r]|^2 of the traction-driven Neumann
    problem through CQ (bem_receiver_energy_grad), differentiable in the
    traction samples g (real float64 (N + 1, n_tris, 3) on the device) and
    the wave speeds c = (c_p, c_s) (real tensor of shape (2,), the speeds the
    operators were compressed at; its value is not read).  The library
    computes J and both gradients in one call (forward solve, adjoint
    solve), so the backward only scales them by the incoming gradient."""

    @staticmethod
    def forward(ctx, g: torch.Tensor, c: torch.Tensor, V: Operator, A: Operator, dV, dA, rec, N: int, dt: float,
                tol: float = 1e-8, max_iter: int = 500):
        J, dg, dc, _ = receiver_energy_grad(V, A, g.contiguous(), rec, N, dt, dV=dV, dA=dA, tol=tol,
                                            max_iter=max_iter, grad_g=True)
        ctx.save_for_backward(dg)
        ctx.dc = torch.tensor(dc + [0.0] * (2 - len(dc)), dtype=c.dtype, device=c.device)
        return torch.tensor(J, dtype=torch.float64, device=g.device)

    @staticmethod
    def backward(ctx, gJ: torch.Tensor):
        (dg,) = ctx.saved_tensors
        return gJ * dg, gJ.to(ctx.dc.device) * ctx.dc, None, None, None, None, None, None, None, None, None


def receiver_energy(g: torch.Tensor, c: torch.Tensor, V: Operator, A: Operator, dV, dA, rec, N: int, dt: float,
                    tol: float = 1e-8, max_iter: int = 500) -> torch.Tensor:
    """Differentiable receiver energy (see ReceiverEnergy)."""
    return ReceiverEnergy.apply(g, c, V, A, tuple(dV), tuple(dA), rec, N, dt, tol, max_iter)
