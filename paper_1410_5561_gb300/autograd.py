"""torch.autograd.Function around the library's forward and adjoint sweeps.

Forward: u_T = A(C)^T u_0 (Listings 2 and 3, T Jacobi steps, Dirichlet halo),
computed by stencil_run_checkpointed with the grid's schedule (blocked when the
grid is tuned so), keeping every k-th state (k = ceil(sqrt(T)) by default).
Backward: stencil_run_adjoint recomputes the states between checkpoints and
runs the transposed operator backwards, accumulating the coefficient gradients
in FP64 (available afterwards as ``grid.last_coef_grad``).

One forward/backward pair per grid at a time: the grid's arrays and workspace
hold the state of the last forward call.
"""
from __future__ import annotations

import torch

from .stencil import Stencil


class StencilSweep(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0: torch.Tensor, coefs: torch.Tensor, grid: Stencil, T: int, ckpt_every: int = 0,
                halo: float = 0.0):
        grid.set_coeffs(arrays=list(coefs.detach()))
        grid.set_field(u0.detach(), halo=halo)
        ws = grid.adjoint_workspace(T, ckpt_every)
        grid.run_checkpointed(T, ckpt_every, ws)
        uT = grid.get_field()
        ctx.grid, ctx.T, ctx.k, ctx.ws = grid, int(T), int(ckpt_every), ws
        ctx.coef_dtype = coefs.dtype
        return uT

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        grid: Stencil = ctx.grid
        lam = grid.new_field_array(zero=True)
        grid.interior_of(lam).copy_(g.to(grid.dtype))
        gu = grid.new_field_array(zero=False)
        gc = [grid.new_grad_array() for _ in range(grid.ncoef)]
        grid.run_adjoint(ctx.T, ctx.k, lam, gu, gc, ctx.ws)
        g_u0 = grid.interior_of(gu).clone()
        g_c = torch.stack([grid.interior_of(x) for x in gc])
        grid.last_coef_grad = g_c
        return g_u0, g_c.to(ctx.coef_dtype), None, None, None, None


def sweep(u0: torch.Tensor, coefs: torch.Tensor, grid: Stencil, T: int, ckpt_every: int = 0, halo: float = 0.0):
    """Differentiable u_T for the variable-coefficient stencils."""
    return StencilSweep.apply(u0, coefs, grid, T, ckpt_every, halo)
