"""torch.autograd Functions over the library's filter and its hand-written backward.

``ChebFilterFn``: Y = filter(X; V_eff, B_xc, Delta) (gbc_filter forward,
gbc_filter_vjp backward, checkpointing every ``ckpt_every`` degrees).
``EnergyFn``: L = sum_i w_i y_i^H H y_i (gbc_energy_grad).
Gradients follow torch's convention for complex tensors (dL/dRe + i dL/dIm).
Fields are host float64 tensors [E, nq^3]; Delta is a host complex128 tensor of
the concatenated per-atom matrices.  Both are loaded into the context in the
forward pass; every arithmetic step runs in the library's CUDA kernels.
"""
from __future__ import annotations

import numpy as np
import torch


def _load_params(gctx, veff, bx, by, bz, delta):
    gctx.set_fields(veff.detach().cpu().numpy(), bx.detach().cpu().numpy(),
                    by.detach().cpu().numpy(), bz.detach().cpu().numpy())
    if delta is not None and delta.numel():
        gctx.set_delta(delta.detach().cpu().numpy())


class ChebFilterFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, veff, bx, by, bz, delta, gctx, degree, lT, lmax, lmin, ckpt_every=5):
        _load_params(gctx, veff, bx, by, bz, delta)
        Y = X.detach().clone()
        gctx.filter(Y, degree, lT, lmax, lmin)
        ctx.save_for_backward(X.detach())
        ctx.gctx = gctx
        ctx.args = (degree, lT, lmax, lmin, ckpt_every)
        ctx.shapes = (veff.shape, delta.shape if delta is not None else None)
        return Y

    @staticmethod
    def backward(ctx, GY):
        (X,) = ctx.saved_tensors
        degree, lT, lmax, lmin, ck = ctx.args
        GX = torch.empty_like(X)
        gV, gBx, gBy, gBz, gD = ctx.gctx.filter_vjp(X, GY.contiguous().to(X.dtype), GX, degree,
                                                    lT, lmax, lmin, ck)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a))
        gdelta = t(gD) if ctx.shapes[1] is not None else None
        return GX, t(gV), t(gBx), t(gBy), t(gBz), gdelta, None, None, None, None, None, None


class EnergyFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Y, veff, bx, by, bz, delta, gctx, w):
        _load_params(gctx, veff, bx, by, bz, delta)
        GY = torch.empty_like(Y)
        L, gV, gBx, gBy, gBz, gD = gctx.energy_grad(Y.detach(), w, GY)
        ctx.grads = (GY, gV, gBx, gBy, gBz, gD, delta is not None)
        return torch.tensor(L, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gL):
        GY, gV, gBx, gBy, gBz, gD, has_d = ctx.grads
        s = float(gL)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)) * s
        return (GY * s, t(gV), t(gBx), t(gBy), t(gBz), t(gD) if has_d else None, None, None)
