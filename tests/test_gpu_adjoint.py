"""Differentiation: torch.autograd through the library's
forward and adjoint solves, against the oracle's adjoint gradient and
central finite differences of the loss L = 1/2 |u - u_obs|^2."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_08109_gb300 import autograd, binding, inputs
from tests.gpu_util import relerr

pytestmark = pytest.mark.gpu


def _grad(prob, tol=1e-12):
    dev = "cuda"
    coords = torch.as_tensor(prob.coords, device=dev)
    m = torch.as_tensor(prob.extra["m"], device=dev).requires_grad_(True)
    f = torch.as_tensor(prob.rhs, device=dev).requires_grad_(True)
    u_obs = torch.as_tensor(prob.extra["u_obs"], device=dev)
    s = binding.Solver(2, prob.n)
    u = autograd.solve(m, f, coords, s, tol=tol, maxit=500)
    loss = 0.5 * ((u - u_obs) ** 2).sum()
    loss.backward()
    return loss.item(), m.grad.cpu().numpy(), f.grad.cpu().numpy(), u.detach().cpu().numpy()


def test_gradient_matches_oracle_adjoint():
    (prob,) = inputs.annulus_adjoint(65, batch=1)
    _, gm, gf, u = _grad(prob)
    H = oracle.Hierarchy(oracle.assemble(prob.coords, prob.kappa))
    uo = H.pcg(prob.rhs, tol=1e-14, maxit=500)[0]
    lo = H.pcg(uo - prob.extra["u_obs"], tol=1e-14, maxit=500)[0]
    go = prob.kappa * oracle.adjoint_grad(prob.coords, uo, lo)
    assert relerr(gm, go) <= 1e-8
    assert relerr(gf, lo) <= 1e-8


def test_gradient_matches_central_differences():
    """Central differences in m_e with eps = 2e-3, the loss difference formed
    as 1/2 sum (u+ - u-)(u+ + u- - 2 u_obs) to avoid cancellation; relative
    error against max(|g_e|, 1e-2 max|g|).  The two errors of the difference
    quotient: truncation, O(eps^2 |g_e|) (below 1e-6 relative here with exact
    solves), and the solves' stopping error divided by 2 eps, which is the same
    absolute size for every cell and is therefore bounded against max|g|."""
    (prob,) = inputs.annulus_adjoint(129, batch=1)
    _, gm, _, u = _grad(prob, tol=1e-12)
    s = binding.Solver(2, prob.n)
    rng = np.random.default_rng(3)
    cells = [tuple(c) for c in rng.integers(0, prob.n - 1, size=(8, 2))]
    eps = 2e-3
    scale = np.abs(gm).max()
    f = torch.as_tensor(prob.rhs, device="cuda")
    for c in cells:
        sols = []
        for sgn in (+1, -1):
            mm = prob.extra["m"].copy()
            mm[c] += sgn * eps
            s.assemble(torch.as_tensor(prob.coords), torch.as_tensor(np.exp(mm))).setup()
            x, _ = s.solve(f, x0=torch.as_tensor(u, device="cuda"), tol=1e-12, maxit=500)
            sols.append(x.cpu().numpy())
        up, um = sols
        dL = 0.5 * np.sum((up - um) * (up + um - 2 * prob.extra["u_obs"]))
        fd = dL / (2 * eps)
        assert abs(fd - gm[c]) <= 1e-5 * max(abs(gm[c]), 1e-2 * scale), (c, fd, gm[c])


def test_batch_of_independent_members():
    probs = inputs.annulus_adjoint(33, batch=3)
    coords = torch.as_tensor(probs[0].coords, device="cuda")
    ms = [torch.as_tensor(p.extra["m"], device="cuda").requires_grad_(True) for p in probs]
    fs = [torch.as_tensor(p.rhs, device="cuda") for p in probs]
    solvers = [binding.Solver(2, 33) for _ in probs]
    us = autograd.solve_batch(ms, fs, coords, solvers, tol=1e-12)
    loss = sum(0.5 * ((u - torch.as_tensor(p.extra["u_obs"], device="cuda")) ** 2).sum() for u, p in zip(us, probs))
    loss.backward()
    for p, m in zip(probs, ms):
        H = oracle.Hierarchy(oracle.assemble(p.coords, p.kappa))
        uo = H.pcg(p.rhs, tol=1e-14)[0]
        lo = H.pcg(uo - p.extra["u_obs"], tol=1e-14)[0]
        assert relerr(m.grad.cpu().numpy(), p.kappa * oracle.adjoint_grad(p.coords, uo, lo)) <= 1e-8


def test_concurrent_batch_matches_oracle():
    """Members on streams of their own with the refinement solver: forward
    and adjoint solves through bmg_solve_many, the contraction through
    bmg_adjoint_cells.  Same bounds as the one-member-at-a-time path."""
    probs = inputs.annulus_adjoint(129, batch=3)
    coords = torch.as_tensor(probs[0].coords, device="cuda")
    ms = [torch.as_tensor(p.extra["m"], device="cuda").requires_grad_(True) for p in probs]
    fs = [torch.as_tensor(p.rhs, device="cuda").requires_grad_(True) for p in probs]
    solvers = [binding.Solver(2, 129, precision="fp32", outer="refine", stream=torch.cuda.Stream()) for _ in probs]
    assert autograd._concurrent(solvers)
    us = autograd.solve_batch(ms, fs, coords, solvers, tol=1e-12)
    loss = sum(0.5 * ((u - torch.as_tensor(p.extra["u_obs"], device="cuda")) ** 2).sum() for u, p in zip(us, probs))
    loss.backward()
    for p, m, f in zip(probs, ms, fs):
        H = oracle.Hierarchy(oracle.assemble(p.coords, p.kappa))
        uo = H.pcg(p.rhs, tol=1e-14, maxit=500)[0]
        lo = H.pcg(uo - p.extra["u_obs"], tol=1e-14, maxit=500)[0]
        assert relerr(m.grad.cpu().numpy(), p.kappa * oracle.adjoint_grad(p.coords, uo, lo)) <= 1e-8
        assert relerr(f.grad.cpu().numpy(), lo) <= 1e-8


@pytest.mark.parametrize("dim,n", [(2, 65), (3, 9)])
def test_adjoint_cells_matches_oracle_contraction(dim, n):
    """bmg_adjoint_cells on arbitrary u and lambda (zero on the boundary)
    against the oracle's contraction.  Each element term cancels (K_e has
    zero row sums) down to O(h^2) of its summands, so rounding is amplified
    by up to (n-1)^2 relative to the largest term."""
    rng = np.random.default_rng(7 + dim)
    p = inputs.annulus_adjoint(n, batch=1)[0] if dim == 2 else inputs.shell_two_layer(n)
    m = oracle.interior_mask(n, dim)
    u = np.where(m, rng.uniform(-1, 1, size=(n,) * dim), 0.0)
    lam = np.where(m, rng.uniform(-1, 1, size=(n,) * dim), 0.0)
    s = binding.Solver(dim, n).assemble(torch.as_tensor(p.coords), torch.as_tensor(p.kappa)).setup()
    got = s.adjoint_cells(torch.as_tensor(u), torch.as_tensor(lam)).cpu().numpy()
    ref = oracle.adjoint_grad(p.coords, u, lam)
    assert np.abs(got - ref).max() <= np.finfo(float).eps * (n - 1) ** 2 * np.abs(ref).max()


def test_adjoint_cells_refused_before_setup_and_on_a_tensor_operator():
    p = inputs.annulus_anisotropic(17)
    u = torch.zeros((p.n, p.n), dtype=torch.float64, device="cuda")
    s = binding.Solver(2, p.n).assemble(torch.as_tensor(p.coords), torch.as_tensor(p.kappa))
    with pytest.raises(binding.BmgError) as e:
        s.adjoint_cells(u, u)
    assert e.value.code == 10
    s = binding.Solver(2, p.n).assemble_tensor(torch.as_tensor(p.coords), torch.as_tensor(p.extra["D"])).setup()
    with pytest.raises(binding.BmgError) as e:
        s.adjoint_cells(u, u)
    assert e.value.code == 10
