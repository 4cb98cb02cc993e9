"""Differentiable s-step CG solve: x = A(kappa)^-1 b for the cell-centred diffusion stencil,
as a torch.autograd.Function whose backward runs the adjoint solve A lambda = dL/dx with the
same handle (A is SPD, so A^T = A) and assembles dL/dkappa in a CUDA kernel
(sstep_cg_grad_kappa). dL/db = lambda. Marshalling only: both solves and the assembly run in
libsstep_cg.so.
"""
from __future__ import annotations

import torch

from . import abi
from .solver import SStepCG


class SStepSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, kappa: torch.Tensor, b: torch.Tensor, grid: tuple, opts: dict):
        kappa = kappa.detach().contiguous()
        opts = dict(opts)
        ctx.adjoint_tol = opts.pop("adjoint_tol", None)
        sv = SStepCG(grid=grid, kappa=kappa, **opts)
        x, info = sv.solve(b.detach().contiguous(), allow_no_convergence=False)
        ctx.sv = sv
        ctx.save_for_backward(x)
        ctx.info = info
        return x

    @staticmethod
    def backward(ctx, gx: torch.Tensor):
        (x,) = ctx.saved_tensors
        sv = ctx.sv
        if ctx.adjoint_tol is not None:
            abi.sstep_cg_set_tolerance(sv.h, ctx.adjoint_tol, sv.opts.max_outer)
        lam, _ = sv.solve(gx.detach().contiguous(), allow_no_convergence=False)
        gk = torch.empty_like(x)
        abi.sstep_cg_grad_kappa(sv.h, x, lam, gk)
        sv.close()
        return gk, lam, None, None


def solve_diffusion(kappa: torch.Tensor, b: torch.Tensor, grid, **opts) -> torch.Tensor:
    """x = A(kappa)^-1 b, differentiable in kappa and b. `grid` = (nx, ny[, nz]); options as
    for SStepCG (s, nu, tol, bounds_mode, ...); `adjoint_tol` sets the backward solve's
    tolerance (default: tol)."""
    return SStepSolve.apply(kappa, b, tuple(int(v) for v in grid), dict(opts))
