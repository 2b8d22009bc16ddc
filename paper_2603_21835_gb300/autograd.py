"""torch.autograd wrapper of the grid energy E = sum_g w V_g rho_g.

Forward: positions -> neighbour lists (rebuilt on the device when they change), density pass,
float64 energy reduction on the device.  Backward (hand-written, no graph through the
kernels):
    dE/dD    = H          (the local-Hamiltonian pass; D enters through its symmetric part,
                           so this is the gradient for symmetric perturbations of D)
    dE/dV_g  = w rho_g    (the density saved by the forward)
    dE/dR_I  = -F_I       (the local Pulay force pass of the paper's Sec. 3.3.1; orbitals and
                           their gradients are recomputed by the kernel, not stored)
"""
from __future__ import annotations

import torch

from . import gint as G


class GintEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, D_blocks: torch.Tensor, V: torch.Tensor, pos: torch.Tensor, g: "G.Gint", precision: int):
        g.ensure_positions(pos)
        rho = g.rho(D_blocks, precision)
        E = g.grid_dot(V, rho)
        ctx.save_for_backward(D_blocks, V, rho)
        ctx.g = g
        ctx.precision = precision
        return E.reshape(())

    @staticmethod
    def backward(ctx, gE: torch.Tensor):
        D_blocks, V, rho = ctx.saved_tensors
        g, prec = ctx.g, ctx.precision
        gD = gV = gpos = None
        if ctx.needs_input_grad[0]:
            gD = gE * g.vlocal(V, prec)
        if ctx.needs_input_grad[1]:
            gV = (gE * g.weight) * rho.reshape(-1)
        if ctx.needs_input_grad[2]:
            gpos = -gE * g.force(D_blocks, V, prec)
        return gD, gV, gpos, None, None


def grid_energy(g: "G.Gint", D_blocks: torch.Tensor, V: torch.Tensor, pos: torch.Tensor,
                precision: int = G.FP64) -> torch.Tensor:
    """E = sum_g w V rho(D, pos) as a differentiable float64 scalar (device)."""
    return GintEnergy.apply(D_blocks, V, pos, g, precision)
