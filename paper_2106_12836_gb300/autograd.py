"""Differentiable SAIT-preconditioned solve: x = A^{-1} b as a torch.autograd.Function.

A is given by its values on a fixed CSR pattern, so gradients flow to whatever
produced those values (for instance a PDE assembly from coefficients written
with torch ops).  Forward: ILU(0), SAIT build of L and U, right-preconditioned
GMRES, all through the C ABI.  Backward (the adjoint method): solve
A^T lambda = dl/dx with GMRES preconditioned by the transposed SAIT apply
(M_U M_L)^T = M_L^T M_U^T on transposed copies made on the GPU, then
dl/db = lambda and dl/dA_ij = -lambda_i x_j on A's pattern.

This module only calls the C ABI; every step runs in the library's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import (Context, sait_build, sait_gmres, sait_ilu0, sait_mat_create_csr, sait_mat_transpose,
               sait_outer_on_pattern, sait_prec_create_sait)

__all__ = ["SolveOptions", "SaitSolve", "sait_solve"]


@dataclass
class SolveOptions:
    m_terms: int = 3
    drop: str = "rowrel"
    tau: float = 1e-3
    store: str = "f64"
    restart: int = 30
    tol: float = 1e-8
    adjoint_tol: float | None = None   # defaults to tol
    maxit: int = 20000


class SaitSolve(torch.autograd.Function):
    @staticmethod
    def forward(fctx, vals, b, rp, ci, ctx: Context, opts: SolveOptions):
        n = b.numel()
        vals_c = vals.detach().contiguous()
        b_c = b.detach().contiguous()
        A = sait_mat_create_csr(ctx, n, rp, ci, vals_c)
        L, U = sait_ilu0(ctx, n, rp, ci, vals_c)
        ML = sait_build(ctx, L, True, opts.m_terms, opts.drop, opts.tau, store=opts.store)
        MU = sait_build(ctx, U, False, opts.m_terms, opts.drop, opts.tau, store=opts.store)
        P = sait_prec_create_sait(ctx, ML, MU)
        x, info, _ = sait_gmres(ctx, A, P, b_c, restart=opts.restart, tol=opts.tol, maxit=opts.maxit)
        fctx.save_for_backward(x)
        fctx.objs = (ctx, A, ML, MU, opts)
        fctx.info = info.as_dict()
        return x

    @staticmethod
    def backward(fctx, gx):
        (x,) = fctx.saved_tensors
        ctx, A, ML, MU, opts = fctx.objs
        AT = sait_mat_transpose(ctx, A)
        PT = sait_prec_create_sait(ctx, sait_mat_transpose(ctx, MU), sait_mat_transpose(ctx, ML))
        tol = opts.adjoint_tol if opts.adjoint_tol is not None else opts.tol
        lam, _, _ = sait_gmres(ctx, AT, PT, gx.detach().contiguous(), restart=opts.restart, tol=tol,
                               maxit=opts.maxit)
        gA = sait_outer_on_pattern(ctx, A, -1.0, lam, x)
        return gA, lam, None, None, None, None


def sait_solve(vals: torch.Tensor, b: torch.Tensor, rp: torch.Tensor, ci: torch.Tensor, ctx: Context,
               opts: SolveOptions | None = None) -> torch.Tensor:
    """x = A(vals)^{-1} b, differentiable with respect to vals and b."""
    return SaitSolve.apply(vals, b, rp, ci, ctx, opts or SolveOptions())
