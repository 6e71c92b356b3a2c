"""torch.autograd binding of Algorithm 1's H application with respect to the
wavefunctions, the local potential V_loc(r) and the nonlocal coefficients D.

Forward and backward both run in libchebfi (chebfi_apply_H, chebfi_apply_H_backward);
this module only wires them into autograd.  The context's V_loc and D are replaced by the
values passed in (V through chebfi_set_vloc, D through chebfi_set_D) before each forward.
"""
from __future__ import annotations

import torch

from .chebfi import ChebFI, fortran

__all__ = ["apply_H", "ApplyH"]


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
        ctx.save_for_backward(Yf)
        return out

    @staticmethod
    def backward(ctx, G):
        (Yf,) = ctx.saved_tensors
        op = ctx.op
        need_y, need_v, need_d = ctx.needs_input_grad[:3]
        Gf = fortran(G, device=Yf.device)
        gY, gV, gD = op.apply_H_backward(Yf, Gf, ctx.grid, ctx.nD, need_y, need_v, need_d)
        return gY, gV, gD, None


def apply_H(op: ChebFI, Y: torch.Tensor, V: torch.Tensor, D: torch.Tensor) -> torch.Tensor:
    """H(V, D) Y, differentiable in Y (complex128, npw x nb), V (float64 grid) and D (float64,
    packed per-atom blocks)."""
    return ApplyH.apply(Y, V, D, op)
