"""Auxiliary-space two-grid method (Sec. 2.2 "Setup phase" / "Solution
phase", Sec. 2.3): the library's A_p, M_p and C against the oracle's, its
cycle against the oracle's cycle at a fixed count, its solves against the
oracle's, and its argument and state checks."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle
from oracle import aux
from paper_2509_08109_gb300 import binding, inputs
from tests.gpu_util import relerr

pytestmark = pytest.mark.gpu


def _coarse(n, precision="fp64"):
    coords = inputs.coords_quarter_annulus(n)
    s = binding.Solver(2, n, precision=precision)
    s.assemble(torch.as_tensor(coords), torch.ones((n - 1, n - 1), dtype=torch.float64)).setup()
    return coords, s


def _oracle(m, coords, mass_steps=0):
    n = coords.shape[-1]
    return aux.TwoGrid(m, coords, oracle.assemble(coords, np.ones((n - 1, n - 1))), mass_steps=mass_steps)


def _csr(a, which, shape):
    rp, col, val = a.export(which)
    return sp.csr_matrix((val, col, rp), shape=shape)


@pytest.mark.parametrize("nr,nt,n", [(25, 37, 17), (14, 9, 9)])
def test_operators_match_oracle(nr, nt, n):
    m = inputs.annulus_mesh(nr, nt)
    coords, s = _coarse(n)
    a = binding.AuxSolver(s, m)
    tg = _oracle(m, coords)
    nvi = len(tg.iv)
    A = _csr(a, "A", (nvi, nvi))
    M = _csr(a, "M", (nvi, nvi))
    C = _csr(a, "C", (nvi, n * n))[:, tg.ic]
    for got, ref in ((A, tg.A), (M, tg.M), (C, tg.C)):
        r = ref.toarray()
        assert np.abs(got.toarray() - r).max() <= 1e-13 * np.abs(r).max()


@pytest.mark.parametrize("mass_steps", [0, 3])
def test_fixed_cycles_match_oracle(mass_steps):
    """tol 0 runs exactly maxit cycles on both sides."""
    m = inputs.annulus_mesh(25, 37)
    coords, s = _coarse(17)
    a = binding.AuxSolver(s, m, mass_steps=mass_steps)
    tg = _oracle(m, coords, mass_steps)
    f = m.f[tg.iv]
    u = np.zeros_like(f)
    for _ in range(5):
        u = tg.cycle(f, u)
    got, info = a.solve(torch.as_tensor(m.f, device="cuda"), tol=0.0, maxit=5, raise_on_nonconv=False)
    assert info.iterations == 5
    got = got.cpu().numpy()
    assert np.all(got[m.dirichlet] == 0.0)
    assert relerr(got[tg.iv], u) <= 1e-11


@pytest.mark.parametrize("mass_steps", [0, 3])
def test_solve_matches_oracle(mass_steps):
    m = inputs.annulus_mesh(25, 37)
    coords, s = _coarse(17)
    a = binding.AuxSolver(s, m, mass_steps=mass_steps)
    uo, ito, _ = _oracle(m, coords, mass_steps).solve(m.f, tol=1e-10)
    u, info = a.solve(torch.as_tensor(m.f, device="cuda"), tol=1e-10)
    assert info.status == 0 and info.true_relres <= 1e-10
    assert abs(info.iterations - ito) <= 1
    assert relerr(u.cpu().numpy(), uo) <= 1e-8


def test_fp32_coarse_level_and_residual_recomputed():
    """An FP32 V-cycle as the coarse solve; the returned iterate's residual,
    recomputed on the host from the exported A_p, meets the tolerance."""
    m = inputs.annulus_mesh(97, 145)
    coords, s = _coarse(65, precision="fp32")
    a = binding.AuxSolver(s, m)
    u, info = a.solve(torch.as_tensor(m.f, device="cuda"), tol=1e-10)
    assert info.status == 0
    iv = np.flatnonzero(~m.dirichlet)
    A = _csr(a, "A", (len(iv), len(iv)))
    r = m.f[iv] - A @ u.cpu().numpy()[iv]
    assert np.linalg.norm(r) <= 1.0001e-10 * np.linalg.norm(m.f[iv])


def test_coupled_mass_signs_and_rows():
    """Interior block of C: no entry below -eps max (products of
    non-negative bases and |det J|; barycentric coordinates of points on a
    clipped edge can round to -eps), and every interior vertex couples to
    some interior node."""
    m = inputs.annulus_mesh(41, 61)
    coords, s = _coarse(33)
    a = binding.AuxSolver(s, m)
    rp, col, val = a.export("C")
    assert val.min() >= -1e-15 * val.max() and val.max() > 0.0
    assert np.all(np.diff(rp) > 0)


def test_errors():
    m = inputs.annulus_mesh(9, 13)
    s = binding.Solver(2, 9)
    with pytest.raises(binding.BmgError) as e:          # coarse level not set up
        binding.AuxSolver(s, m)
    assert e.value.code == 10
    coords, s = _coarse(9)
    with pytest.raises(binding.BmgError) as e:          # Jacobi weight out of range
        binding.AuxSolver(s, m, omega=2.5)
    assert e.value.code == 1
    bad = inputs.annulus_mesh(9, 13)
    bad.tri = bad.tri[:, [0, 2, 1]].copy()               # clockwise: negative physical area
    with pytest.raises(binding.BmgError) as e:
        binding.AuxSolver(s, bad)
    assert e.value.code == 5


@pytest.mark.parametrize("mass_steps", [0, 3])
def test_gamma_matches_oracle_lanczos(mass_steps):
    """Coarse-grid scaling (Sec. 2.4): k = 12 steps of generalized Lanczos on
    (P^T A_p P, A_c) from A_c^-1 y0.  The library's recurrence uses the dual
    vectors A_c q_j and the coarse context's PCG; the oracle's uses A_c and
    dense solves.  Same alphas, same gamma."""
    m = inputs.annulus_mesh(25, 37)
    coords, s = _coarse(17)
    a = binding.AuxSolver(s, m, mass_steps=mass_steps)
    tg = _oracle(m, coords, mass_steps)
    y0 = np.random.default_rng(11).uniform(-1.0, 1.0, size=(17, 17))
    g, alpha, beta = a.estimate_gamma(k=12, y0=y0, tol=1e-13)
    Ac = oracle.dense_operator(oracle.assemble(coords, np.ones((16, 16))))
    B = lambda x: tg.restrict(tg.A @ tg.prolong(x))
    x0 = np.linalg.solve(Ac, y0.reshape(-1)[tg.ic])
    go, ritz = aux.gamma_lanczos(B, lambda x: Ac @ x, lambda x: np.linalg.solve(Ac, x), x0, k=12)
    assert len(alpha) == 12
    assert abs(g - go) <= 1e-8 * abs(go)
    assert abs(g - alpha.mean()) <= 1e-14 * abs(g)
    T = np.diag(alpha) + np.diag(beta, 1) + np.diag(beta, -1)
    assert np.allclose(np.sort(np.linalg.eigvalsh(T)), np.sort(ritz), rtol=1e-7, atol=0)


@pytest.mark.parametrize("mass_steps", [0, 2])
def test_flexible_cg_matches_oracle(mass_steps):
    m = inputs.annulus_mesh(25, 37)
    coords, s = _coarse(17)
    a = binding.AuxSolver(s, m, mass_steps=mass_steps, krylov=True)
    uo, ito, trr = _oracle(m, coords, mass_steps).solve_fcg(m.f, tol=1e-10)
    u, info = a.solve(torch.as_tensor(m.f, device="cuda"), tol=1e-10, raise_on_nonconv=False)
    assert abs(info.iterations - ito) <= 1
    assert info.true_relres <= 2e-10
    assert relerr(u.cpu().numpy(), uo) <= 1e-8


def test_flexible_cg_with_fp32_preconditioner():
    """On an FP32 coarse context with the lumped mass, the preconditioning
    cycle runs its physical level in FP32 (difference-form products); the
    FP64 flexible CG still reaches the tolerance, checked on the host from
    the exported A_p, in about the iterations of the all-FP64 cycle."""
    m = inputs.annulus_mesh(97, 145)
    _, s64 = _coarse(65)
    coords, s32 = _coarse(65, precision="fp32")
    f = torch.as_tensor(m.f, device="cuda")
    _, i64 = binding.AuxSolver(s64, m, krylov=True).solve(f, tol=1e-10)
    a = binding.AuxSolver(s32, m, krylov=True)
    u, info = a.solve(f, tol=1e-10)
    assert info.status == 0 and info.iterations <= i64.iterations + 3
    iv = np.flatnonzero(~m.dirichlet)
    A = _csr(a, "A", (len(iv), len(iv)))
    r = m.f[iv] - A @ u.cpu().numpy()[iv]
    assert np.linalg.norm(r) <= 1.0001e-10 * np.linalg.norm(m.f[iv])


def test_identity_map_with_rough_coefficient_matches_oracle():
    """A second geometry: the unit square with T the identity (the coarse
    grid's cells are then the square's own), a log-normal coefficient per
    triangle; operators and the flexible-CG solve against the oracle."""
    m = inputs.square_mesh(27, 23, kappa_sigma=0.5)
    n = 17
    coords = inputs.coords_identity(n, 2)
    s = binding.Solver(2, n)
    s.assemble(torch.as_tensor(coords), torch.ones((n - 1, n - 1), dtype=torch.float64)).setup()
    a = binding.AuxSolver(s, m, krylov=True)
    tg = aux.TwoGrid(m, coords, oracle.assemble(coords, np.ones((n - 1, n - 1))), mass_steps=0)
    nvi = len(tg.iv)
    for which, ref in (("A", tg.A), ("M", tg.M)):
        got = _csr(a, which, (nvi, nvi)).toarray()
        assert np.abs(got - ref.toarray()).max() <= 1e-13 * np.abs(ref.toarray()).max()
    C = _csr(a, "C", (nvi, n * n))[:, tg.ic].toarray()
    assert np.abs(C - tg.C.toarray()).max() <= 1e-13 * np.abs(tg.C.toarray()).max()
    uo, ito, _ = tg.solve_fcg(m.f, tol=1e-10)
    u, info = a.solve(torch.as_tensor(m.f, device="cuda"), tol=1e-10)
    assert info.status == 0 and abs(info.iterations - ito) <= 1
    assert relerr(u.cpu().numpy(), uo) <= 1e-8


@pytest.mark.parametrize("krylov", [True, False])
def test_graph_replay_equals_direct_launches(krylov):
    """Iterations (after the first, for flexible CG) replay a captured graph
    when the coarse context uses graphs; the iterates are bitwise those of
    direct launches, also after gamma changes (the graphs are recaptured)."""
    m = inputs.annulus_mesh(49, 73)
    f = torch.as_tensor(m.f, device="cuda")
    out = []
    for graphs in (True, False):
        coords = inputs.coords_quarter_annulus(33)
        s = binding.Solver(2, 33, precision="fp32", outer="refine", graphs=graphs)
        s.assemble(torch.as_tensor(coords), torch.ones((32, 32), dtype=torch.float64)).setup()
        a = binding.AuxSolver(s, m, krylov=krylov)
        u1, i1 = a.solve(f, tol=1e-10)
        a.set_gamma(0.9)
        u2, i2 = a.solve(f, tol=1e-10)
        out.append((u1.cpu().numpy(), i1.iterations, u2.cpu().numpy(), i2.iterations))
    (a1, n1, b1, k1), (a2, n2, b2, k2) = out
    assert n1 == n2 and k1 == k2
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2)
