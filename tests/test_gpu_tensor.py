"""SPD diffusion tensor per cell (Sec. 2, Eq. pde): bmg_assemble_tensor
against the oracle's tensor assembly, the hierarchy built from it, and
solves to 1e-10 in both precisions."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_08109_gb300 import binding, inputs
from tests.gpu_util import rel_to_diag, relerr

pytestmark = pytest.mark.gpu

EPS = np.finfo(float).eps


@pytest.mark.parametrize("n", [9, 65, 257])
def test_tensor_assembly_2d_matches_oracle(n):
    p = inputs.annulus_anisotropic(n)
    s = binding.Solver(2, n).assemble_tensor(torch.as_tensor(p.coords), torch.as_tensor(p.extra["D"]))
    ref = oracle.assemble_tensor(p.coords, p.extra["D"])
    assert rel_to_diag(s.stencil(0).cpu().numpy(), ref) <= 4 * n * EPS


@pytest.mark.parametrize("n", [5, 9, 17])
def test_tensor_assembly_3d_matches_oracle(n):
    p = inputs.shell_anisotropic(n)
    s = binding.Solver(3, n).assemble_tensor(torch.as_tensor(p.coords), torch.as_tensor(p.extra["D"]))
    ref = oracle.assemble_tensor(p.coords, p.extra["D"])
    assert rel_to_diag(s.stencil(0).cpu().numpy(), ref) <= 4 * n * EPS


def test_tensor_hierarchy_matches_oracle():
    """The anisotropic operators make the collapse sensitive to rounding (as
    the shell map does), so, as there, each level's bound is 20 times the
    oracle's own response to a 2e-16 relative perturbation of its input,
    and never below 1e-12."""
    p = inputs.annulus_anisotropic(129)
    s = binding.Solver(2, p.n).assemble_tensor(torch.as_tensor(p.coords), torch.as_tensor(p.extra["D"])).setup()
    A = oracle.assemble_tensor(p.coords, p.extra["D"])
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


@pytest.mark.parametrize("precision,outer", [("fp64", "cg"), ("fp32", "refine")])
def test_tensor_solve_matches_oracle(precision, outer):
    p = inputs.annulus_anisotropic(257)
    s = binding.Solver(2, p.n, precision=precision, outer=outer)
    s.assemble_tensor(torch.as_tensor(p.coords), torch.as_tensor(p.extra["D"])).setup()
    x, info = s.solve(torch.as_tensor(p.rhs, device="cuda"), tol=1e-10, maxit=500)
    assert info.status == 0 and info.true_relres <= 1e-10
    H = oracle.Hierarchy(oracle.assemble_tensor(p.coords, p.extra["D"]))
    xo, _, _, trr, st = H.pcg(p.rhs, tol=1e-12, maxit=500)
    assert st == 0
    assert relerr(x.cpu().numpy(), xo) <= 1e-7


def test_adjoint_refused_on_a_tensor_operator():
    p = inputs.annulus_anisotropic(17)
    s = binding.Solver(2, p.n).assemble_tensor(torch.as_tensor(p.coords), torch.as_tensor(p.extra["D"])).setup()
    u = torch.zeros((p.n, p.n), dtype=torch.float64, device="cuda")
    with pytest.raises(binding.BmgError) as e:
        s.adjoint_grad(u, u)
    assert e.value.code == 10
