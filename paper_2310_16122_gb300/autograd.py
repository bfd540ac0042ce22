"""torch.autograd.Function wrappers whose backward passes are libcrk's hand-written adjoint kernels.

The forward passes call grav_short, crk_geometry, crk_corrections and
crk_hydro; the backward passes call grav_short_adjoint, crk_geometry_adjoint,
crk_corrections_adjoint and crk_hydro_adjoint, which recompute the pair terms
(nothing per pair is stored).  Chained, geometry -> corrections -> hydro give
the gradient of a loss of dv/dt, du/dt in the positions, masses, velocities
and u.  Gradients flow to the positions (as a (3, n)
tensor) and the masses; h is held fixed and the leaves are treated as
constant (piecewise constant in the positions, so they carry no gradient).

The kernels read the positions captured by the leaves, so every forward
checks the positions tensor passed in against the ones the leaves were built
from: the same storage passes at once; another tensor must hold equal values
(checked on the device), else CRK_ESTATE is raised: leaves built from other
positions would give values and gradients at the wrong positions.
"""
from __future__ import annotations

import torch

from . import api
from . import native as N


def _check_positions(pos3, leaves: api.Leaves) -> None:
    """Refuse positions other than those the leaves were built from (CRK_ESTATE)."""
    src = leaves._keep[:3]
    if pos3.dim() != 2 or pos3.shape[0] != 3 or pos3.shape[1] != leaves.n:
        raise N.CrkError(N.CRK_ESTATE, f"positions must be a (3, {leaves.n}) tensor, got {tuple(pos3.shape)}")
    p = pos3.detach()
    if all(p[c].data_ptr() == src[c].data_ptr() and p[c].stride() == src[c].stride() for c in range(3)):
        return
    if not all(torch.equal(p[c], src[c]) for c in range(3)):
        raise N.CrkError(N.CRK_ESTATE, "positions differ from those the leaves were built from: rebuild the leaves")


class GravShort(torch.autograd.Function):
    """a = grav_short(positions, m); backward gives dL/dpositions, dL/dm."""

    @staticmethod
    def forward(fctx, pos3, m, ctx: api.Context, leaves: api.Leaves, gp: api.GravParams):
        _check_positions(pos3, leaves)
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
        _check_positions(pos3, leaves)
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


class CrkCorrections(torch.autograd.Function):
    """(A, B, gradA, gradB) = crk_corrections(positions, V); backward gives dL/dpositions, dL/dV."""

    @staticmethod
    def forward(fctx, pos3, V, ctx: api.Context, leaves: api.Leaves):
        _check_positions(pos3, leaves)
        A, B, gA, gB, _ = api.corrections(ctx, leaves, V.detach().contiguous())
        fctx.save_for_backward(V)
        fctx.crk = (ctx, leaves)
        return A, B, gA, gB

    @staticmethod
    def backward(fctx, Abar, Bbar, gAbar, gBbar):
        (V,) = fctx.saved_tensors
        ctx, leaves = fctx.crk
        n = V.numel()
        z = lambda t, *shape: t.contiguous() if t is not None else torch.zeros(*shape, device=V.device)
        gx, gV, _ = api.corrections_adjoint(ctx, leaves, V.detach().contiguous(), z(Abar, n), z(Bbar, 3, n),
                                            z(gAbar, 3, n), z(gBbar, 9, n))
        return gx, gV, None, None


class CrkHydro(torch.autograd.Function):
    """(dv, du) = crk_hydro(positions, m, v, u, V, rho, A, B, gradA, gradB); backward gives the
    gradients in every tensor input (the pair terms are recomputed)."""

    @staticmethod
    def forward(fctx, pos3, m, v3, u, V, rho, A, B, gA, gB, ctx: api.Context, leaves: api.Leaves,
                hp: api.HydroParams):
        _check_positions(pos3, leaves)
        ins = [t.detach().contiguous() for t in (m, v3, u, V, rho, A, B, gA, gB)]
        dv, du, _, _ = api.hydro(ctx, leaves, hp, *ins)
        fctx.save_for_backward(*ins)
        fctx.crk = (ctx, leaves, hp)
        return dv, du

    @staticmethod
    def backward(fctx, dvbar, dubar):
        ins = fctx.saved_tensors
        ctx, leaves, hp = fctx.crk
        n = ins[0].numel()
        dvbar = dvbar.contiguous() if dvbar is not None else torch.zeros(3, n, device=ins[0].device)
        dubar = dubar.contiguous() if dubar is not None else torch.zeros(n, device=ins[0].device)
        g = api.hydro_adjoint(ctx, leaves, hp, *ins, dvbar, dubar)
        return (g["x"], g["m"], g["v"], g["u"], g["V"], g["rho"], g["A"], g["B"], g["gA"], g["gB"],
                None, None, None)


def corrections(pos3, V, ctx, leaves):
    return CrkCorrections.apply(pos3, V, ctx, leaves)


def hydro(pos3, m, v3, u, V, rho, A, B, gA, gB, ctx, leaves, hp):
    return CrkHydro.apply(pos3, m, v3, u, V, rho, A, B, gA, gB, ctx, leaves, hp)


def gravity(pos3, m, ctx, leaves, gp):
    return GravShort.apply(pos3, m, ctx, leaves, gp)


def geometry(pos3, m, ctx, leaves):
    return CrkGeometry.apply(pos3, m, ctx, leaves)
