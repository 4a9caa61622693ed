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


class BmgSolveMany(torch.autograd.Function):
    """A batch of independent members solved concurrently: each member's
    solver runs on its own stream, the forward solves and the adjoint solves
    go through bmg_solve_many (one scheduler keeps all members' refinement
    loops in flight) and the per-cell contraction through bmg_adjoint_cells.
    Inputs: the solvers, the shared coordinates, tol, maxit, then the
    members' m followed by their f."""

    @staticmethod
    def forward(ctx, solvers, coords, tol, maxit, *mf):
        k = len(solvers)
        ms, fs = mf[:k], mf[k:]
        cur = torch.cuda.current_stream()
        kappas = [torch.exp(m.detach().to(torch.float64)).contiguous() for m in ms]
        fs64 = [f.detach().to(torch.float64).contiguous() for f in fs]
        us = [torch.zeros_like(f) for f in fs64]
        ready = cur.record_event()
        for s, kap in zip(solvers, kappas):
            s.stream.wait_event(ready)
            s.assemble(coords, kap).setup()
        # bmg_solve_many returns after every member's stream has drained
        ctx.infos = binding.solve_many(solvers, [[f] for f in fs64], [[u] for u in us], tol=tol, maxit=maxit)
        ctx.save_for_backward(*us, *kappas)
        ctx.solvers, ctx.tol, ctx.maxit = solvers, tol, maxit
        return tuple(us)

    @staticmethod
    def backward(ctx, *gus):
        k = len(ctx.solvers)
        saved = ctx.saved_tensors
        us, kappas = saved[:k], saved[k:]
        gs = [torch.zeros_like(u) if g is None else g.to(torch.float64).contiguous() for g, u in zip(gus, us)]
        lams = [torch.zeros_like(g) for g in gs]
        ready = torch.cuda.current_stream().record_event()
        for s in ctx.solvers:
            s.stream.wait_event(ready)
        binding.solve_many(ctx.solvers, [[g] for g in gs], [[l] for l in lams], tol=ctx.tol, maxit=ctx.maxit)
        dks = []
        for s, u, lam in zip(ctx.solvers, us, lams):
            dks.append(s.adjoint_cells(u, lam))     # synchronises its stream
        return (None, None, None, None) + tuple(kap * dk for kap, dk in zip(kappas, dks)) + tuple(lams)


def _concurrent(solvers) -> bool:
    streams = {s.stream.cuda_stream for s in solvers}
    return (len(solvers) > 1 and len(streams) == len(solvers)
            and all(s.precision == "fp32" and s.outer == "refine" for s in solvers))


def solve_batch(ms, fs, coords, solvers, tol: float = 1e-10, maxit: int = 500):
    """Independent problems sharing a grid size: one solver (and hierarchy)
    per member; returns the list of solutions.  Solvers built with
    precision='fp32', outer='refine', each on a stream of its own, run the
    members concurrently (forward and adjoint); otherwise the members are
    solved one after the other."""
    if _concurrent(solvers):
        coords = coords.to(device=solvers[0].device, dtype=torch.float64).contiguous()
        return list(BmgSolveMany.apply(list(solvers), coords, tol, maxit, *ms, *fs))
    return [BmgSolve.apply(m, f, coords, s, tol, maxit) for m, f, s in zip(ms, fs, solvers)]
