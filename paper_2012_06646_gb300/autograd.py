"""Differentiable spreading and interpolation (torch.autograd.Function).

With W_jk = prod_b phi(t_b - r_b) the weight of point j at node k,
spreading is f = h^-d W^T G and interpolation is U = W u (Eqs. disc-spread,
disc-interp; S* = S^T, Eqs. matrix-interp and matrix-spread).  Hence

  spread:       dL/dG = h^-d W (dL/df)      -> ib_interpolate with IB_ADJOINT
                dL/dX = h^-d D(dL/df, G)    -> ib_pos_grad with IB_SPREAD_GRAD (h^-d applied in C)
  interpolate:  dL/du = W^T (dL/dU)         -> ib_spread with IB_ADJOINT
                dL/dX = D(u, dL/dU)         -> ib_pos_grad, scale = 1

where D(field, v)_{j,b} = sum_a v_{j,a} sum_k field_a[k] dW_jk/dX_{j,b}, the
position derivative of the weights.  Every backward step runs in the CUDA
kernels of libibgb.so.  The backward reuses the forward call's bins when the
plan has not re-binned since and X is the same, unmodified tensor.
"""

from __future__ import annotations

import torch

from .plan import Plan


def _bins_token(plan: Plan, Xc, X):
    """What must be unchanged for the bins of the forward call to serve the backward."""
    return (plan.bin_epoch, Xc.data_ptr(), X._version)


def _ensure_bins(ctx, plan: Plan, Xc, X) -> None:
    """Re-bin X unless the plan still holds the bins the forward call made for the
    same, unmodified positions."""
    if _bins_token(plan, Xc, X) != ctx.bins:
        plan.bin(Xc)


class SpreadFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, G, plan: Plan, compensated: bool = False):
        Xc = X.detach().contiguous()
        f = plan.spread(Xc, G.detach().contiguous(), compensated=compensated)
        ctx.plan = plan
        ctx.bins = _bins_token(plan, Xc, X)
        ctx.save_for_backward(X, G)
        return f

    @staticmethod
    def backward(ctx, gf):
        X, G = ctx.saved_tensors
        plan = ctx.plan
        gf = gf.contiguous()
        Xc = X.detach().contiguous()
        gX = gG = None
        _ensure_bins(ctx, plan, Xc, X)
        if ctx.needs_input_grad[1]:
            gG = plan.interpolate(Xc, gf, reuse_bins=True, adjoint=True)
        if ctx.needs_input_grad[0]:
            gX = plan.pos_grad(Xc, gf, G.detach().contiguous(), reuse_bins=True, spread=True)
        return gX, gG, None, None


class InterpolateFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, u, plan: Plan):
        Xc = X.detach().contiguous()
        U = plan.interpolate(Xc, u.detach().contiguous())
        ctx.plan = plan
        ctx.bins = _bins_token(plan, Xc, X)
        ctx.save_for_backward(X, u)
        return U

    @staticmethod
    def backward(ctx, gU):
        X, u = ctx.saved_tensors
        plan = ctx.plan
        gU = gU.contiguous()
        Xc = X.detach().contiguous()
        gX = gu = None
        _ensure_bins(ctx, plan, Xc, X)
        if ctx.needs_input_grad[1]:
            gu = plan.spread(Xc, gU, reuse_bins=True, adjoint=True)
        if ctx.needs_input_grad[0]:
            gX = plan.pos_grad(Xc, u.detach().contiguous(), gU, scale=1.0, reuse_bins=True)
        return gX, gu, None


def spread(X, G, plan: Plan, compensated: bool = False):
    """Differentiable f = S G on the plan's grid."""
    return SpreadFunction.apply(X, G, plan, compensated)


def interpolate(X, u, plan: Plan):
    """Differentiable U = S* u at the points X."""
    return InterpolateFunction.apply(X, u, plan)
