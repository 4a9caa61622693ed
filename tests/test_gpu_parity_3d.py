"""3-D parity of the CUDA path (through the C ABI) against the oracle:
27-point trilinear assembly, hierarchical-collapse interpolation, Galerkin
coarse operators, 8-colour V-cycle, PCG, FP32 modes.  Same tolerances as the
2-D tests (FP64 rounding through the hierarchy)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_08109_gb300 import binding, inputs
from tests.gpu_util import U32, check_fp32_vcycle, rel_to_diag, relerr, solver_for

pytestmark = pytest.mark.gpu


def _problem(n, kind="shell"):
    if kind == "shell":
        return inputs.shell_two_layer(n)
    p = inputs.shell_two_layer(n)
    rng = np.random.default_rng(n)
    p.kappa = np.exp(rng.normal(0, 0.7, size=p.kappa.shape))
    return p


@pytest.mark.parametrize("n", [5, 9, 17, 33])
def test_assembly_3d_matches_oracle(n):
    p = _problem(n)
    s = binding.Solver(3, n).assemble(torch.as_tensor(p.coords), torch.as_tensor(p.kappa))
    ref = oracle.assemble(p.coords, p.kappa)
    assert rel_to_diag(s.stencil(0).cpu().numpy(), ref) <= 1e-13


def _identity_random(n, sigma=0.5):
    p = inputs.shell_two_layer(n)
    p.coords = inputs.coords_identity(n, 3)
    p.kappa = np.exp(np.random.default_rng(n).normal(0, sigma, size=p.kappa.shape))
    return p


@pytest.mark.parametrize("n", [9, 17, 33])
def test_hierarchy_3d_matches_oracle_well_conditioned(n):
    """Identity map, log-normal kappa: every level to 1e-12."""
    p = _identity_random(n)
    s = solver_for(p)
    H = oracle.Hierarchy(oracle.assemble(p.coords, p.kappa))
    assert s.levels == H.nlev
    for l in range(H.nlev):
        assert rel_to_diag(s.stencil(l).cpu().numpy(), H.A(l)) <= 1e-12, l
        if l < H.nlev - 1:
            assert np.abs(s.interp(l).cpu().numpy() - H.P(l)).max() <= 1e-12, l


@pytest.mark.parametrize("n,kind", [(9, "shell"), (9, "random"), (17, "shell"), (33, "shell")])
def test_hierarchy_3d_matches_oracle(n, kind):
    """Shell map (polar degeneracy, kappa contrast 1000): the collapse
    amplifies rounding level by level, so the bound per level is the
    oracle's own response to a 2e-16 relative perturbation of its input
    (times 20), and never below 1e-12.  The factor: the library rounds
    differently from the oracle in every operation of the collapse and of
    the Galerkin product, not only once per input entry; a coarse entry
    collects up to 27 x 8 weighted products per level, and independent
    relative errors of one unit roundoff in m operations move the result
    by about sqrt(m) times the response to one such error at the input
    (sqrt(216) ~ 15), so 20 covers one level's worth with margin.  A
    well-conditioned map is held to 1e-12 without scaling (the test above)."""
    p = _problem(n, kind)
    s = solver_for(p)
    A = oracle.assemble(p.coords, p.kappa)
    H = oracle.Hierarchy(A)
    Hp = oracle.Hierarchy(A * (1 + 2e-16 * np.random.default_rng(0).standard_normal(A.shape)))
    assert s.levels == H.nlev
    for l in range(H.nlev):
        Ao = H.A(l)
        sens_a = rel_to_diag(Hp.A(l), Ao)
        assert rel_to_diag(s.stencil(l).cpu().numpy(), Ao) <= max(1e-12, 20 * sens_a), l
        if l < H.nlev - 1:
            Po = H.P(l)
            sens_p = np.abs(Hp.P(l) - Po).max()
            assert np.abs(s.interp(l).cpu().numpy() - Po).max() <= max(1e-12, 20 * sens_p), l


@pytest.mark.parametrize("n,kind", [(3, "random"), (5, "random"), (9, "random"), (17, "shell")])
def test_vcycle_3d_matches_oracle(n, kind):
    p = _problem(n, kind)
    s = solver_for(p)
    H = oracle.Hierarchy(oracle.assemble(p.coords, p.kappa))
    r = inputs.rhs_uniform(np.random.default_rng(3), (n, n, n))
    z = s.vcycle(torch.as_tensor(r, device="cuda")).cpu().numpy()
    assert relerr(z, H.vcycle(r)) <= 1e-12
    z32 = solver_for(p, precision="fp32").vcycle(torch.as_tensor(r, device="cuda")).cpu().numpy()
    check_fp32_vcycle(z32, H, r, 3)


@pytest.mark.parametrize("n,iters", [(9, 4), (17, 6)])
def test_pcg_3d_fixed_iterations(n, iters):
    p = _problem(n)
    s = solver_for(p)
    H = oracle.Hierarchy(oracle.assemble(p.coords, p.kappa))
    x, info = s.solve(torch.as_tensor(p.rhs, device="cuda"), tol=0.0, maxit=iters)
    xo, ito, _, _, _ = H.pcg(p.rhs, tol=0.0, maxit=iters)
    assert info.iterations == iters
    assert relerr(x.cpu().numpy(), xo) <= 1e-9


@pytest.mark.parametrize("precision,outer", [("fp64", "cg"), ("fp32", "flexible"), ("fp32", "refine")])
def test_pcg_3d_free_running(precision, outer):
    n = 17
    p = _problem(n)
    s = solver_for(p, precision=precision, outer=outer)
    x, info = s.solve(torch.as_tensor(p.rhs, device="cuda"), tol=1e-10, maxit=500)
    H = oracle.Hierarchy(oracle.assemble(p.coords, p.kappa))
    xo, ito, _, trr, _ = H.pcg(p.rhs, tol=1e-12, maxit=500)
    assert info.true_relres <= 1e-10
    assert relerr(x.cpu().numpy(), xo) <= 1e-6
    if precision == "fp64":
        xo10, it10, _, _, _ = H.pcg(p.rhs, tol=1e-10, maxit=500)
        assert abs(info.iterations - it10) <= 1
    elif outer == "flexible":
        _, it32, _, _, st32 = H.pcg(p.rhs, tol=1e-10, maxit=500, flexible=True, fp32=True)
        assert st32 == 0 and abs(info.iterations - it32) <= 1


def test_collapse_fallback_matches_oracle():
    """With a rough per-cell coefficient on the shell map some collapsed
    denominators of the 3-D interpolation are not positive (17^3); those
    points use their own uncollapsed couplings in the oracle and in the
    library alike, and the hierarchies agree."""
    n = 17
    p = _problem(n, "random")
    s = solver_for(p)
    A = oracle.assemble(p.coords, p.kappa)
    H = oracle.Hierarchy(A)
    Hp = oracle.Hierarchy(A * (1 + 2e-16 * np.random.default_rng(0).standard_normal(A.shape)))
    for l in range(H.nlev):
        Ao = H.A(l)
        assert rel_to_diag(s.stencil(l).cpu().numpy(), Ao) <= max(1e-12, 20 * rel_to_diag(Hp.A(l), Ao)), l
        if l < H.nlev - 1:
            Po = H.P(l)
            assert np.abs(s.interp(l).cpu().numpy() - Po).max() <= max(1e-12, 20 * np.abs(Hp.P(l) - Po).max()), l
    x, info = s.solve(torch.as_tensor(p.rhs, device="cuda"), tol=1e-10, maxit=1000)
    assert info.true_relres <= 1e-10


def test_adjoint_3d_matches_oracle():
    n = 9
    p = _problem(n, "random")
    s = solver_for(p)
    u, _ = s.solve(torch.as_tensor(p.rhs, device="cuda"), tol=1e-13, maxit=300)
    g = u - torch.as_tensor(p.rhs, device="cuda") * 0.5
    lam, dk, _ = s.adjoint_grad(u, g, tol=1e-13, maxit=300)
    ref = oracle.adjoint_grad(p.coords, u.cpu().numpy(), lam.cpu().numpy())
    assert relerr(dk.cpu().numpy(), ref) <= 1e-12


# ------------------------------------------------------------------ half-sweep 3-D V-cycle
# FP32 levels from 17^3 up smooth with one launch per colour parity of k (the
# half-sweep kernels: 58 x 14 owned points per CTA, with a 3-column, 1-row
# halo).  At 65^3 the 63 interior columns make a full and a ragged tile, the
# 63 rows five tiles with a ragged fifth; at 129^3, three column tiles and
# ten row tiles.  FP64 levels keep the per-colour kernels.  The FP32 coarse
# end (9^3 and below) runs in one CTA from shared memory, so the V-cycle tests
# at 3^3..9^3 exercise it whole and those at 17^3 and up behind half sweeps.
@pytest.mark.parametrize("n", [33, 65])
def test_halfsweep_vcycle_3d_matches_oracle_well_conditioned(n):
    """Identity map, log-normal kappa: the FP64 V-cycle to 1e-12 of the
    oracle's; the FP32 one of both smoother paths element by element against
    the oracle's FP32 arm."""
    p = _identity_random(n)
    H = oracle.Hierarchy(oracle.assemble(p.coords, p.kappa))
    r = inputs.rhs_uniform(np.random.default_rng(n), (n, n, n))
    rt = torch.as_tensor(r, device="cuda")
    z = solver_for(p).vcycle(rt).cpu().numpy()
    assert relerr(z, H.vcycle(r)) <= 1e-12
    for unfused in (False, True):
        z32 = solver_for(p, precision="fp32", unfused=unfused).vcycle(rt).cpu().numpy()
        check_fp32_vcycle(z32, H, r, 3)


@pytest.mark.parametrize("n,kind", [(33, "shell"), (65, "shell"), (65, "random"), (129, "shell")])
def test_halfsweep_vcycle_3d_shell(n, kind):
    """Shell octant (kappa contrast 1000, or a rough per-cell kappa).  The
    half sweeps sum every point's 26 products in the order of the per-colour
    kernels, so the two FP32 paths agree to rounding (they were bitwise
    equal when measured).  The library's FP64 V-cycle differs from the
    oracle's by at most 20 times the oracle's own response to a 2e-16
    relative perturbation of its operator (reading R3: the collapse amplifies
    rounding level by level; at 129^3 this difference is about 3e-5), and
    the FP32 cycles are checked element by element against the FP32 arm with
    that difference in the bound."""
    p = _problem(n, kind)
    A = oracle.assemble(p.coords, p.kappa)
    H = oracle.Hierarchy(A)
    r = inputs.rhs_uniform(np.random.default_rng(n + 1), (n, n, n))
    rt = torch.as_tensor(r, device="cuda")
    z64o = H.vcycle(r)
    scale = np.abs(z64o).max()
    z64 = solver_for(p).vcycle(rt).cpu().numpy()
    d_hier = np.abs(z64 - z64o).max() / scale
    Hp = oracle.Hierarchy(A * (1 + 2e-16 * np.random.default_rng(0).standard_normal(A.shape)))
    sens = np.abs(Hp.vcycle(r) - z64o).max() / scale
    assert d_hier <= max(1e-12, 20 * sens), (d_hier, sens)
    za = solver_for(p, precision="fp32").vcycle(rt).cpu().numpy()
    zb = solver_for(p, precision="fp32", unfused=True).vcycle(rt).cpu().numpy()
    assert np.abs(za - zb).max() / scale <= 4 * U32
    for z32 in (za, zb):
        check_fp32_vcycle(z32, H, r, 3, d_hier)


@pytest.mark.parametrize("precision,outer", [("fp64", "cg"), ("fp32", "flexible"), ("fp32", "refine")])
def test_halfsweep_pcg_3d_free_running(precision, outer):
    """33^3 shell octant through the half-sweep V-cycle: verified 1e-10,
    the oracle's solution, and the oracle's iteration count (FP64 CG, FP32
    flexible CG against the oracle's FP32 arm) within one."""
    n = 33
    p = _problem(n)
    s = solver_for(p, precision=precision, outer=outer)
    x, info = s.solve(torch.as_tensor(p.rhs, device="cuda"), tol=1e-10, maxit=1000)
    H = oracle.Hierarchy(oracle.assemble(p.coords, p.kappa))
    xo, _, _, _, _ = H.pcg(p.rhs, tol=1e-12, maxit=2000)
    assert info.true_relres <= 1e-10
    assert relerr(x.cpu().numpy(), xo) <= 1e-6
    if precision == "fp64":
        _, it10, _, _, _ = H.pcg(p.rhs, tol=1e-10, maxit=2000)
        assert abs(info.iterations - it10) <= 1
    elif outer == "flexible":
        _, it32, _, _, st32 = H.pcg(p.rhs, tol=1e-10, maxit=2000, flexible=True, fp32=True)
        assert st32 == 0 and abs(info.iterations - it32) <= 1


def test_halfsweep_refinement_matches_unfused_iterations_3d():
    """65^3 shell octant, FP32 refinement mode: the two smoother paths take
    the same number of iterations (within one) to a verified 1e-10."""
    p = _problem(65)
    f = torch.as_tensor(p.rhs, device="cuda")
    xa, ia = solver_for(p, precision="fp32", outer="refine").solve(f, tol=1e-10, maxit=2000)
    xb, ib = solver_for(p, precision="fp32", outer="refine", unfused=True).solve(f, tol=1e-10, maxit=2000)
    assert ia.true_relres <= 1e-10 and ib.true_relres <= 1e-10
    assert abs(ia.iterations - ib.iterations) <= 1
