"""Differentiable block CG solve: X = A(vals)^{-1} B as a torch.autograd.Function.

Forward: one bcg_solve on the handle. Backward (A is symmetric, so the adjoint system A Lambda = dL/dX is
solved by the same handle and kernels): dL/dB = Lambda, and, for every stored CSR entry e = (i, j),
dL/dvals[e] = -Lambda_i . X_j (bcg_grad_values). This follows from dX = -A^{-1} dA X. The paper has no
differentiation; this is the standard adjoint of a linear solve applied to its hot path.

The values are treated as independent parameters, one per stored entry. A symmetric perturbation of the
pair (i, j), (j, i) (which keeps A SPD) therefore has derivative grad[(i, j)] + grad[(j, i)].
"""
from __future__ import annotations

import torch

from . import bcg


class BCGSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, B, solver: "bcg.Solver", tol: float, maxit: int):
        if vals.data_ptr() != solver._keep[2].data_ptr():
            raise ValueError("vals must be the tensor the solver's handle was created with (or passed to "
                             "update_values)")
        X, res = solver.solve(B.detach().contiguous(), tol=tol, maxit=maxit)
        if not res.ok:
            raise bcg.BCGError(res.status, f"forward solve: {bcg.bcg_last_error()}")
        ctx.solver, ctx.tol, ctx.maxit = solver, tol, maxit
        ctx.save_for_backward(X)
        return X

    @staticmethod
    def backward(ctx, gX):
        (X,) = ctx.saved_tensors
        Lam, res = ctx.solver.solve(gX.detach().contiguous(), tol=ctx.tol, maxit=ctx.maxit)
        if not res.ok:
            raise bcg.BCGError(res.status, f"adjoint solve: {bcg.bcg_last_error()}")
        gvals = ctx.solver.grad_values(Lam, X) if ctx.needs_input_grad[0] else None
        gB = Lam if ctx.needs_input_grad[1] else None
        return gvals, gB, None, None, None


def bcg_solve_autograd(vals: torch.Tensor, B: torch.Tensor, solver: "bcg.Solver", tol: float = 1e-10,
                       maxit: int = 20000) -> torch.Tensor:
    """X = A(vals)^{-1} B, differentiable in vals and B. ``solver`` is a CSR Solver created from ``vals``."""
    return BCGSolve.apply(vals, B, solver, tol, maxit)
