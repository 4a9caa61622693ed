"""Harmonic maps built with the library (Sec. 3, Definition of a harmonic
map and the theorem on convex targets).

Given a boundary map phi from the unit square (cube) onto the boundary of
the physical domain, each physical coordinate of the map is the discrete
harmonic extension of that coordinate of phi: the Q1 Laplace problem on the
identity grid (kappa = 1) with phi as Dirichlet data, solved by bmg_solve
after bmg_boundary_rhs has moved the data to the right-hand side.  For a
convex target and a unimodal phi the result is a valid map (det J > 0 at
every quadrature point), which bmg_assemble then accepts."""
from __future__ import annotations

import torch

from . import binding, inputs


def harmonic_coords(boundary, tol: float = 1e-12, maxit: int = 500, device=None) -> torch.Tensor:
    """Nodal coordinates (d, n, ...) of the harmonic extension of the
    boundary values `boundary` (shape (d, n, ...), interior ignored), as FP64
    on the device."""
    g = torch.as_tensor(boundary, dtype=torch.float64)
    d, n = g.shape[0], g.shape[-1]
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    g = g.to(dev)
    ident = torch.as_tensor(inputs.coords_identity(n, d), device=dev)
    ones = torch.ones((n - 1,) * d, dtype=torch.float64, device=dev)
    s = binding.Solver(d, n, device=dev)
    s.assemble(ident, ones).setup()
    interior = torch.zeros((n,) * d, dtype=torch.bool, device=dev)
    interior[(slice(1, n - 1),) * d] = True
    out = []
    for c in range(d):
        rhs = s.boundary_rhs(ident, ones, g[c])
        x, _ = s.solve(rhs, tol=tol, maxit=maxit)
        out.append(torch.where(interior, x, g[c]))
    return torch.stack(out).contiguous()
