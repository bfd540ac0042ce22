"""torch.autograd.Function wrappers whose backward passes are libcrk's hand-written adjoint kernels.

The forward passes call grav_short and crk_geometry; the backward passes call
grav_short_adjoint and crk_geometry_adjoint, which recompute the pair terms
(nothing per pair is stored).  Gradients flow to the positions (as a (3, n)
tensor) and the masses; h is held fixed and the leaves are treated as
constant (piecewise constant in the positions, so they carry no gradient).

The positions tensor passed in must be the one the leaves were built from; the
kernels read the positions captured by the leaves.
"""
from __future__ import annotations

import torch

from . import api


class GravShort(torch.autograd.Function):
    """a = grav_short(positions, m); backward gives dL/dpositions, dL/dm."""

    @staticmethod
    def forward(fctx, pos3, m, ctx: api.Context, leaves: api.Leaves, gp: api.GravParams):
        a, _ = api.grav_short(ctx, leaves, gp, m.detach().contiguous())
        fctx.save_for_backward(m)
        fctx.crk = (ctx, leaves, gp)
        return a

    @staticmethod
    def backward(fctx, abar):
        (m,) = fctx.saved_tensors
        ctx, leaves, gp = fctx.crk
        gx, gm = api.grav_short_adjoint(ctx, leaves, gp, m.detach().contiguous(), abar.contiguous())
        return gx, gm, None, None, None


class CrkGeometry(torch.autograd.Function):
    """(V, rho) = crk_geometry(positions, m); backward gives dL/dpositions, dL/dm."""

    @staticmethod
    def forward(fctx, pos3, m, ctx: api.Context, leaves: api.Leaves):
        V, rho, _ = api.geometry(ctx, leaves, m.detach().contiguous())
        fctx.save_for_backward(m, V)
        fctx.crk = (ctx, leaves)
        return V, rho

    @staticmethod
    def backward(fctx, Vbar, rhobar):
        m, V = fctx.saved_tensors
        ctx, leaves = fctx.crk
        if rhobar is None:
            rhobar = torch.zeros_like(V)
        gx, gm = api.geometry_adjoint(ctx, leaves, m.detach().contiguous(), V, rhobar.contiguous(),
                                      Vbar.contiguous() if Vbar is not None else None)
        return gx, gm, None, None


def gravity(pos3, m, ctx, leaves, gp):
    return GravShort.apply(pos3, m, ctx, leaves, gp)


def geometry(pos3, m, ctx, leaves):
    return CrkGeometry.apply(pos3, m, ctx, leaves)
