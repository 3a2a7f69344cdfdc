"""PressureSolve: x = A(upper, diag)^-1 b as a torch.autograd.Function.

Forward: one spuma_pcg_solve.  Backward (the adjoint; A is symmetric):
A lambda = dL/dx by the same PCG from lambda = 0, then
dL/db = lambda, dL/dupper_f = -(lambda_l x_u + lambda_u x_l), dL/ddiag = -lambda x,
all on the device (spuma_pcg_adjoint).  The forward's x is kept; no Krylov
history is stored.

LaplacianAssembly: (upper, diag) = assembly(gamma, bgamma) on fixed geometry
(spuma_assemble_laplacian); its backward is spuma_assemble_laplacian_adjoint,
so that a loss on x differentiates down to the face diffusivities.
"""
from __future__ import annotations

import torch

from .core import LduMesh, SolverControls


class PressureSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, upper, diag, b, mesh: LduMesh, controls: SolverControls, adj_controls: SolverControls):
        x, perf = mesh.solve(diag.detach(), upper.detach(), b.detach(), None, controls)
        ctx.mesh, ctx.adj = mesh, adj_controls
        ctx.perf = perf
        ctx.save_for_backward(upper, diag, x)
        return x

    @staticmethod
    def backward(ctx, gx):
        upper, diag, x = ctx.saved_tensors
        dldb, dldu, dldd, _ = ctx.mesh.adjoint(diag.detach(), upper.detach(), x, gx.contiguous(), ctx.adj)
        return dldu, dldd, dldb, None, None, None


def pressure_solve(mesh: LduMesh, upper, diag, b, controls: SolverControls | None = None,
                   adj_controls: SolverControls | None = None):
    c = controls or SolverControls()
    a = adj_controls or SolverControls(precond=c.precond, tolerance=min(c.tolerance, 1e-12))
    return PressureSolve.apply(upper, diag, b, mesh, c, a)


class LaplacianAssembly(torch.autograd.Function):
    @staticmethod
    def forward(ctx, gamma, bgamma, mesh: LduMesh, geometry):
        sf, c, bface_cell, bface_sf, bface_cf, btype = geometry
        upper, diag = mesh.assemble_laplacian(sf, c, gamma.detach(), bface_cell, bface_sf, bface_cf,
                                              None if bgamma is None else bgamma.detach(), btype)
        ctx.mesh, ctx.geometry = mesh, geometry
        return upper, diag

    @staticmethod
    def backward(ctx, gu, gd):
        sf, c, bface_cell, bface_sf, bface_cf, btype = ctx.geometry
        gg, gb = ctx.mesh.assemble_laplacian_adjoint(sf, c, gu, gd, bface_cell, bface_sf, bface_cf, btype)
        return gg, gb, None, None


def assemble_laplacian(mesh: LduMesh, gamma, bgamma, sf, c, bface_cell=None, bface_sf=None, bface_cf=None,
                       btype=None):
    """(upper, diag), differentiable with respect to gamma and bgamma."""
    return LaplacianAssembly.apply(gamma, bgamma, mesh, (sf, c, bface_cell, bface_sf, bface_cf, btype))
