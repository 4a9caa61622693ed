"""Differentiable solve: u = A(kappa = exp(m))^-1 f as a torch.autograd.Function.

Forward assembles A from the map and the per-cell coefficient kappa = exp(m),
builds the hierarchy and solves with the library's PCG.  Backward reuses that
hierarchy for the adjoint solve A lambda = dL/du (A is symmetric) and the
per-cell contraction dL/dkappa_e = -lambda_e^T K_e^0 u_e in the library, so
that dL/dm = kappa * dL/dkappa and dL/df = lambda.  Everything runs in
libbmg.so; this module only moves tensors.

The solver object holds the operator of the last forward call: do not reuse
it for another operator between a forward and its backward.
"""
from __future__ import annotations

import torch

from . import binding


class BmgSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m: torch.Tensor, f: torch.Tensor, coords: torch.Tensor, solver: binding.Solver,
                tol: float = 1e-10, maxit: int = 500):
        kappa = torch.exp(m.detach().to(torch.float64))
        solver.assemble(coords, kappa).setup()
        u, info = solver.solve(f.detach().to(torch.float64), tol=tol, maxit=maxit)
        ctx.save_for_backward(u, kappa)
        ctx.solver, ctx.tol, ctx.maxit = solver, tol, maxit
        ctx.info = info
        return u

    @staticmethod
    def backward(ctx, gu: torch.Tensor):
        u, kappa = ctx.saved_tensors
        lam, dk, _ = ctx.solver.adjoint_grad(u, gu.contiguous().to(torch.float64), tol=ctx.tol, maxit=ctx.maxit)
        return kappa * dk, lam, None, None, None, None


def solve(m, f, coords, solver, tol: float = 1e-10, maxit: int = 500) -> torch.Tensor:
    """u = A(exp(m))^-1 f, differentiable with respect to m and f."""
    return BmgSolve.apply(m, f, coords, solver, tol, maxit)


def solve_batch(ms, fs, coords, solvers, tol: float = 1e-10, maxit: int = 500):
    """Independent problems sharing a grid size: one solver (and hierarchy)
    per member; returns the list of solutions."""
    return [BmgSolve.apply(m, f, coords, s, tol, maxit) for m, f, s in zip(ms, fs, solvers)]
