"""torch.autograd bindings of Algorithm 1's H application and of Algorithm 2's Chebyshev
filter with respect to the wavefunctions, the local potential V_loc(r) and the nonlocal
coefficients D.

Forward and backward all run in libchebfi (chebfi_apply_H / chebfi_apply_H_backward,
chebfi_cheb_filter / chebfi_cheb_filter_backward); this module only wires them into
autograd.  The context's V_loc and D are replaced by the values passed in (V through
chebfi_set_vloc, D through chebfi_set_D) before each forward, and set again before each
backward, so several differentiable calls with different V or D may share one context.
"""
from __future__ import annotations

import torch

from .chebfi import ChebFI, fortran

__all__ = ["apply_H", "ApplyH", "cheb_filter", "ChebFilter"]


class ApplyH(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Y, V, D, op: ChebFI):
        op.set_vloc(V.detach())
        op.set_D(D.detach())
        Yf = fortran(Y.detach(), device=Y.device)
        out = op.apply_H(Yf)
        ctx.op = op
        ctx.grid = tuple(V.shape)
        ctx.nD = D.numel()
        ctx.save_for_backward(Yf, V.detach(), D.detach())
        return out

    @staticmethod
    def backward(ctx, G):
        Yf, V, D = ctx.saved_tensors
        op = ctx.op
        op.set_vloc(V)
        op.set_D(D)
        need_y, need_v, need_d = ctx.needs_input_grad[:3]
        Gf = fortran(G, device=Yf.device)
        gY, gV, gD = op.apply_H_backward(Yf, Gf, ctx.grid, ctx.nD, need_y, need_v, need_d)
        return gY, gV, gD, None


def apply_H(op: ChebFI, Y: torch.Tensor, V: torch.Tensor, D: torch.Tensor) -> torch.Tensor:
    """H(V, D) Y, differentiable in Y (complex128, npw x nb), V (float64 grid) and D (float64,
    packed per-atom blocks)."""
    return ApplyH.apply(Y, V, D, op)


class ChebFilter(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Y, V, D, op: ChebFI, degree, lambda_lo, lambda_hi, prec):
        op.set_vloc(V.detach())
        op.set_D(D.detach())
        Y0 = fortran(Y.detach(), device=Y.device)
        out = op.cheb_filter(Y0.clone(memory_format=torch.preserve_format), degree, lambda_lo, lambda_hi, prec)
        ctx.op = op
        ctx.args = (degree, lambda_lo, lambda_hi, prec)
        ctx.grid = tuple(V.shape)
        ctx.nD = D.numel()
        ctx.save_for_backward(Y0, V.detach(), D.detach())
        return out

    @staticmethod
    def backward(ctx, G):
        Y0, V, D = ctx.saved_tensors
        op = ctx.op
        op.set_vloc(V)
        op.set_D(D)
        degree, lo, hi, prec = ctx.args
        need_y, need_v, need_d = ctx.needs_input_grad[:3]
        Gf = fortran(G, device=Y0.device)
        gY, gV, gD = op.cheb_filter_backward(Y0, Gf, degree, lo, hi, ctx.grid, ctx.nD, prec=prec, want_Y=need_y,
                                             want_V=need_v, want_D=need_d)
        return gY, gV, gD, None, None, None, None, None


def cheb_filter(op: ChebFI, Y: torch.Tensor, V: torch.Tensor, D: torch.Tensor, degree: int, lambda_lo: float,
                lambda_hi: float, prec: int = 0) -> torch.Tensor:
    """Algorithm 2's filter of degree ``degree`` on [lambda_lo, lambda_hi] applied to Y, with
    H = H(V, D); differentiable in Y (complex128, npw x nb), V (float64 grid) and D (float64,
    packed per-atom blocks).  prec: 0 FP64, 1 FP32."""
    return ChebFilter.apply(Y, V, D, op, degree, lambda_lo, lambda_hi, prec)
