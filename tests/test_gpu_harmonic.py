"""Non-zero Dirichlet data (bmg_boundary_rhs) and harmonic maps built with
the library (Sec. 3: Definition of a harmonic map, the theorem on convex
targets and the remark on unimodal boundary maps)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_08109_gb300 import binding, inputs, maps
from tests.gpu_util import relerr

pytestmark = pytest.mark.gpu

EPS = np.finfo(float).eps


def _oracle_harmonic(g):
    n = g.shape[-1]
    ident = inputs.coords_identity(n, 2)
    ones = np.ones((n - 1, n - 1))
    H = oracle.Hierarchy(oracle.assemble(ident, ones))
    m = oracle.interior_mask(n, 2)
    out = []
    for c in range(2):
        x, _, _, _, st = H.pcg(oracle.boundary_rhs(ident, ones, g[c]), tol=1e-13, maxit=500)
        assert st == 0
        out.append(np.where(m, x, g[c]))
    return np.stack(out)


@pytest.mark.parametrize("dim,n", [(2, 9), (2, 65), (3, 9), (3, 17)])
def test_boundary_rhs_matches_oracle(dim, n):
    rng = np.random.default_rng(n + dim)
    coords = inputs.coords_bump(n, 0.1, -0.08) if dim == 2 else inputs.coords_shell_octant(n)
    kappa = np.exp(rng.normal(0, 0.5, size=(n - 1,) * dim))
    g = rng.uniform(-1, 1, size=(n,) * dim)
    s = binding.Solver(dim, n)
    got = s.boundary_rhs(torch.as_tensor(coords), torch.as_tensor(kappa), torch.as_tensor(g)).cpu().numpy()
    ref = oracle.boundary_rhs(coords, kappa, g)
    assert np.abs(got - ref).max() <= 4 * n * EPS * np.abs(ref).max()


@pytest.mark.parametrize("n,amp,lobes", [(65, 0.0, 5), (257, 0.0, 5), (129, 0.1, 3)])
def test_harmonic_map_onto_convex_targets(n, amp, lobes):
    """Convex target, unimodal boundary map: the harmonic extension is a
    valid map (bmg_assemble finds det J > 0 everywhere), it matches the
    oracle's extension, and a Poisson problem solves on it."""
    g = inputs.boundary_star(n, amp, lobes)
    X = maps.harmonic_coords(g)
    assert relerr(X.cpu().numpy(), _oracle_harmonic(g)) <= 1e-9
    s = binding.Solver(2, n, precision="fp32", outer="refine")
    s.assemble(X, torch.ones((n - 1, n - 1), dtype=torch.float64, device="cuda")).setup()
    f = torch.as_tensor(inputs.rhs_uniform(np.random.default_rng(0), (n, n)), device="cuda")
    _, info = s.solve(f, tol=1e-10)
    assert info.status == 0 and info.true_relres <= 1e-10


def test_harmonic_map_onto_a_nonconvex_star_folds():
    """Outside the theorem (a strongly non-convex five-lobed star) the
    discrete harmonic extension folds; the library reports it, as the
    oracle does."""
    n = 65
    g = inputs.boundary_star(n, 0.3, 5)
    X = maps.harmonic_coords(g)
    with pytest.raises(oracle.OracleError):
        oracle.assemble(_oracle_harmonic(g), np.ones((n - 1, n - 1)))
    s = binding.Solver(2, n)
    with pytest.raises(binding.BmgError) as e:
        s.assemble(X, torch.ones((n - 1, n - 1), dtype=torch.float64, device="cuda"))
    assert e.value.code == 5
