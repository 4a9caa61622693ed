"""The batched solve (bmg_batch_*): many mapped problems of uneven sizes,
up to four right-hand sides each, one stencil read per sweep for all of a
problem's right-hand sides, persistent class kernels over a device
work-list, one graph per batch iteration.  Every system is checked against
the oracle (FP64 residual recomputed with the oracle's operator; solution
against the oracle's FP64 solve) or against the single-problem path."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_08109_gb300 import binding, inputs
from tests.gpu_util import relerr

pytestmark = pytest.mark.gpu


def _solvers(probs):
    out = []
    for p in probs:
        s = binding.Solver(2, p.n, precision="fp32", outer="refine")
        s.assemble(torch.as_tensor(p.coords), torch.as_tensor(p.kappa)).setup()
        out.append(s)
    return out


def _true_relres(A, x, b):
    r = b - oracle.apply(A, x)
    r[0, :] = r[-1, :] = r[:, 0] = r[:, -1] = 0
    bb = b.copy()
    bb[0, :] = bb[-1, :] = bb[:, 0] = bb[:, -1] = 0
    return np.linalg.norm(r) / np.linalg.norm(bb)


@pytest.mark.parametrize("nrhs", [4, 3, 1])
def test_batch_engine_matches_oracle(nrhs):
    """Sizes 65..257 (one to three streamed levels per problem, several
    problems per size class): every system reaches the FP64 tolerance,
    recomputed with the oracle's operator, and matches the oracle's FP64
    solve to what that tolerance allows (as the refinement-mode tests)."""
    probs = inputs.bump_batch(count=7, kmin=6, kmax=8, nrhs=nrhs, seed=13)
    solvers = _solvers(probs)
    B = binding.Batch(solvers)
    bs = [[torch.as_tensor(p.rhs[r], device="cuda").contiguous() for r in range(nrhs)] for p in probs]
    xs = [[torch.zeros_like(b) for b in row] for row in bs]
    infos = B.solve(bs, xs, tol=1e-10)
    torch.cuda.synchronize()
    for p, row_x, row_i in zip(probs, xs, infos):
        A = oracle.assemble(p.coords, p.kappa)
        H = oracle.Hierarchy(A)
        for r in range(nrhs):
            x = row_x[r].cpu().numpy()
            assert row_i[r].status == 0 and row_i[r].true_relres <= 1e-10
            assert _true_relres(A, x, p.rhs[r]) <= 1.01e-10
            xo = H.pcg(p.rhs[r], tol=1e-12, maxit=300)[0]
            assert relerr(x, xo) <= 1e-7
            assert np.all(x[0] == 0) and np.all(x[-1] == 0) and np.all(x[:, 0] == 0) and np.all(x[:, -1] == 0)


def test_batch_engine_matches_single_problem_solves():
    """Each system against the single-problem refinement solve of the same
    right-hand side: both meet the tolerance; the lockstep batch may take a
    few more inner iterations (it refines when the slowest system needs to)."""
    probs = inputs.bump_batch(count=6, kmin=6, kmax=9, nrhs=4, seed=21)
    solvers = _solvers(probs)
    B = binding.Batch(solvers)
    bs = [[torch.as_tensor(p.rhs[r], device="cuda").contiguous() for r in range(4)] for p in probs]
    xs = [[torch.zeros_like(b) for b in row] for row in bs]
    infos = B.solve(bs, xs, tol=1e-10)
    torch.cuda.synchronize()
    for s, row_b, row_x, row_i in zip(solvers, bs, xs, infos):
        for r in range(4):
            x1, i1 = s.solve(row_b[r], tol=1e-10)
            torch.cuda.synchronize()
            assert row_i[r].true_relres <= 1e-10 and i1.true_relres <= 1e-10
            assert float((row_x[r] - x1).norm() / x1.norm()) <= 1e-8


def test_batch_engine_zero_rhs_host_buffers_and_initial_guess():
    probs = inputs.bump_batch(count=3, kmin=6, kmax=7, nrhs=2, seed=2)
    solvers = _solvers(probs)
    B = binding.Batch(solvers)
    bs = [[torch.as_tensor(p.rhs[r]).contiguous().pin_memory() for r in range(2)] for p in probs]
    bs[1][0].zero_()
    xs = [[torch.zeros_like(b).pin_memory() for b in row] for row in bs]
    xs[1][0].fill_(1.0)      # a non-zero guess for the zero right-hand side: the answer is still 0
    xs[2][1].copy_(torch.as_tensor(np.random.default_rng(0).uniform(-1, 1, (probs[2].n, probs[2].n))))
    infos = B.solve(bs, xs, tol=1e-10)
    assert xs[1][0].device.type == "cpu"
    assert float(xs[1][0].abs().max()) == 0.0 and infos[1][0].iterations == 0
    for p in range(3):
        A = oracle.assemble(probs[p].coords, probs[p].kappa)
        for r in range(2):
            if (p, r) == (1, 0):
                continue
            assert infos[p][r].true_relres <= 1e-10
            assert _true_relres(A, xs[p][r].numpy(), probs[p].rhs[r]) <= 1.01e-10


def test_batch_engine_graphs_tiles_and_repeat():
    """Graph replays against direct launches (same kernels, same order: the
    same bits), other tile shapes (the same iterations, solutions within the
    tolerance), and two solves in a row on one batch."""
    probs = inputs.bump_batch(count=5, kmin=6, kmax=8, nrhs=4, seed=8)
    solvers = _solvers(probs)
    Bg = binding.Batch(solvers)
    Bd = binding.Batch(solvers, graphs=False)
    bs = [[torch.as_tensor(p.rhs[r], device="cuda").contiguous() for r in range(4)] for p in probs]

    def run(B):
        xs = [[torch.zeros_like(b) for b in row] for row in bs]
        infos = B.solve(bs, xs, tol=1e-10)
        torch.cuda.synchronize()
        return xs, infos

    xg, ig = run(Bg)
    xd, idd = run(Bd)
    for p in range(len(probs)):
        for r in range(4):
            assert torch.equal(xg[p][r], xd[p][r])
            assert ig[p][r].iterations == idd[p][r].iterations
    xg2, ig2 = run(Bg)
    for p in range(len(probs)):
        for r in range(4):
            assert torch.equal(xg[p][r], xg2[p][r])
    before = Bg.tiles()
    for c, (n, wc, hc, m) in enumerate(before):
        if wc:
            Bg.set_tiles(c, 16 if wc == 32 else 32, 2)
    xt, it = run(Bg)
    for p in range(len(probs)):
        for r in range(4):
            assert it[p][r].true_relres <= 1e-10
            assert float((xt[p][r] - xg[p][r]).norm() / xg[p][r].norm()) <= 1e-8
    Bg.autotune(reps=1)
    xa, ia = run(Bg)
    for p in range(len(probs)):
        for r in range(4):
            assert ia[p][r].true_relres <= 1e-10


def test_batch_engine_rejects_ineligible_contexts():
    p = inputs.bump_batch(count=1, kmin=6, kmax=6, nrhs=1, seed=1)[0]
    s = binding.Solver(2, p.n, precision="fp32", outer="flexible")
    s.assemble(torch.as_tensor(p.coords), torch.as_tensor(p.kappa)).setup()
    with pytest.raises(binding.BmgError) as e:
        binding.Batch([s])
    assert e.value.code == 1
    s2 = binding.Solver(2, 33, precision="fp32", outer="refine")
    q = inputs.bump_batch(count=1, kmin=5, kmax=5, nrhs=1, seed=1)[0]
    s2.assemble(torch.as_tensor(q.coords), torch.as_tensor(q.kappa)).setup()
    with pytest.raises(binding.BmgError):
        binding.Batch([s2])


@pytest.mark.parametrize("n,nrhs,max_rhs", [(129, 4, 4), (257, 3, 4), (129, 6, 4), (65, 2, 1)])
def test_bmg_solve_with_several_right_hand_sides(n, nrhs, max_rhs):
    """bmg_solve with nrhs > 1: solved together (max_rhs >= 2; six right-hand
    sides go as groups of four and two) or in turn (max_rhs 1); every
    solution against the single-right-hand-side solve and the oracle's
    operator."""
    p = inputs.bump_batch(count=1, kmin=7, kmax=7, nrhs=nrhs, seed=n)[0] if n == 129 else None
    if p is None:
        k = {65: 6, 257: 8}[n]
        p = inputs.bump_batch(count=1, kmin=k, kmax=k, nrhs=nrhs, seed=n)[0]
    s = binding.Solver(2, n, precision="fp32", outer="refine", max_rhs=max_rhs)
    s.assemble(torch.as_tensor(p.coords), torch.as_tensor(p.kappa)).setup()
    b = torch.as_tensor(p.rhs, device="cuda").contiguous()
    x, infos = s.solve(b, tol=1e-10)
    torch.cuda.synchronize()
    assert len(infos) == nrhs
    A = oracle.assemble(p.coords, p.kappa)
    for r in range(nrhs):
        assert infos[r].true_relres <= 1e-10
        assert _true_relres(A, x[r].cpu().numpy(), p.rhs[r]) <= 1.01e-10
        x1, _ = s.solve(b[r], tol=1e-10)
        assert float((x[r] - x1).norm() / x1.norm()) <= 1e-8
    # host buffers through the same call
    xh, _ = s.solve(b.cpu(), tol=1e-10)
    assert xh.device.type == "cpu"
    assert float((xh - x.cpu()).norm() / x.norm()) <= 1e-12


def test_adjoint_grad_with_several_right_hand_sides():
    """bmg_adjoint_grad with nrhs = 3 against three single calls and the
    oracle's contraction of the oracle's solves.  The adjoint solves ask for
    1e-12: on this smooth adjoint right-hand side the FP32-preconditioned
    refinement reaches about 3e-13 and no further (an inner FP32 CG run on a
    residual at that floor breaks down, on the single-problem path alike)."""
    n = 129
    p = inputs.bump_batch(count=1, kmin=7, kmax=7, nrhs=3, seed=4)[0]
    s = binding.Solver(2, n, precision="fp32", outer="refine", max_rhs=4)
    s.assemble(torch.as_tensor(p.coords), torch.as_tensor(p.kappa)).setup()
    f = torch.as_tensor(p.rhs, device="cuda").contiguous()
    u, _ = s.solve(f, tol=1e-13, maxit=600)
    g = (u - 0.3 * f).contiguous()
    lam, dk, infos = s.adjoint_grad(u, g, tol=1e-12, maxit=600)
    assert lam.shape == f.shape and dk.shape == (3, n - 1, n - 1) and len(infos) == 3
    H = oracle.Hierarchy(oracle.assemble(p.coords, p.kappa))
    for r in range(3):
        l1, d1, _ = s.adjoint_grad(u[r], g[r], tol=1e-12, maxit=600)
        assert float((dk[r] - d1).norm() / d1.norm()) <= 1e-8
        uo = H.pcg(p.rhs[r], tol=1e-13, maxit=300)[0]
        lo = H.pcg(uo - 0.3 * p.rhs[r], tol=1e-13, maxit=300)[0]
        go = oracle.adjoint_grad(p.coords, uo, lo)
        assert relerr(dk[r].cpu().numpy(), go) <= 1e-8
