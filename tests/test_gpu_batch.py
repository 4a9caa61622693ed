"""Batching: many independent mapped problems of
uneven sizes and several right-hand sides, solved concurrently through
bmg_solve_many; every solution is checked against the oracle or against
the single-problem path."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_08109_gb300 import binding, inputs
from tests.gpu_util import relerr

pytestmark = pytest.mark.gpu


def _build(probs):
    solvers = []
    for p in probs:
        st = torch.cuda.Stream()
        s = binding.Solver(2, p.n, precision="fp32", outer="refine", stream=st)
        s.assemble(torch.as_tensor(p.coords), torch.as_tensor(p.kappa)).setup()
        solvers.append(s)
    return solvers


def test_batch_matches_oracle_small_sizes():
    probs = inputs.bump_batch(count=12, kmin=3, kmax=6, nrhs=2, seed=11)
    solvers = _build(probs)
    bs = [[torch.as_tensor(p.rhs[r], device="cuda").contiguous() for r in range(2)] for p in probs]
    xs = [[torch.zeros_like(b) for b in row] for row in bs]
    infos = binding.solve_many(solvers, bs, xs, tol=1e-10)
    torch.cuda.synchronize()
    for p, row_x, row_i in zip(probs, xs, infos):
        H = oracle.Hierarchy(oracle.assemble(p.coords, p.kappa))
        for r in range(2):
            assert row_i[r].true_relres <= 1e-10 and row_i[r].status == 0
            xo = H.pcg(p.rhs[r], tol=1e-12, maxit=300)[0]
            assert relerr(row_x[r].cpu().numpy(), xo) <= 1e-7


def test_batch_matches_single_solves_mixed_sizes():
    probs = inputs.bump_batch(count=16, kmin=5, kmax=9, nrhs=2, seed=5)
    solvers = _build(probs)
    bs = [[torch.as_tensor(p.rhs[r], device="cuda").contiguous() for r in range(2)] for p in probs]
    xs = [[torch.zeros_like(b) for b in row] for row in bs]
    infos = binding.solve_many(solvers, bs, xs, tol=1e-10)
    torch.cuda.synchronize()
    for s, p, row_b, row_x, row_i in zip(solvers, probs, bs, xs, infos):
        for r in range(2):
            x1, i1 = s.solve(row_b[r], tol=1e-10)
            torch.cuda.synchronize()
            assert row_i[r].true_relres <= 1e-10
            assert row_i[r].iterations == i1.iterations
            assert float((row_x[r] - x1).norm() / x1.norm()) <= 1e-12


def test_batch_host_buffers_and_zero_rhs():
    probs = inputs.bump_batch(count=3, kmin=4, kmax=5, nrhs=1, seed=2)
    solvers = _build(probs)
    bs = [[torch.as_tensor(p.rhs[0]).contiguous().pin_memory()] for p in probs]
    bs[1][0].zero_()
    xs = [[torch.zeros_like(row[0]).pin_memory()] for row in bs]
    infos = binding.solve_many(solvers, bs, xs, tol=1e-10)
    torch.cuda.synchronize()
    assert infos[1][0].iterations == 0 and float(xs[1][0].abs().max()) == 0.0
    for p in (0, 2):
        assert infos[p][0].true_relres <= 1e-10
