"""Pins of the auxiliary-space oracle (oracle/aux.py) against what the
mathematics fixes, independently of the oracle's own formulas:

- P1 element matrices of the reference right triangle (closed forms);
- the full stiffness has zero row sums; the full mass sums to the mesh
  polygon's area (shoelace over the boundary ring);
- the full coupled mass sums to the area of the Q1 computational domain
  (shoelace over every computational cell): every Gauss point lies in one
  mapped triangle, the barycentric and bilinear bases are partitions of
  unity, and |det J| of a bilinear cell is affine, so the cut-off rule
  integrates it exactly;
- the oracle's coupled mass (each (triangle, cell) pair integrated over the
  clipped polygon) is the limit of the paper's cut-off Gauss rule (points
  outside the mapped triangle count zero), implemented here independently,
  as its order grows;
- two CG steps satisfy the Galerkin condition on span{r, M r};
- generalized Lanczos run to the full dimension returns the mean of all
  generalized eigenvalues (a trace identity), and its Ritz values interlace
  the dense spectrum from scipy.linalg.eigh;
- the stationary two-grid iteration converges on a small annulus mesh.
"""
import math

import numpy as np
import scipy.linalg as sla
import pytest

import oracle
from oracle import aux
from paper_2509_08109_gb300 import inputs


def test_p1_reference_triangle():
    p = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    K, M, area = aux.p1_element(p, 2.0)
    assert area == 0.5
    Kx = 2.0 * 0.5 * np.array([[2.0, -1.0, -1.0], [-1.0, 1.0, 0.0], [-1.0, 0.0, 1.0]])
    Mx = np.array([[2.0, 1.0, 1.0], [1.0, 2.0, 1.0], [1.0, 1.0, 2.0]]) / 24.0
    assert np.allclose(K, Kx, atol=1e-15)
    assert np.allclose(M, Mx, atol=1e-15)


def _shoelace(P):
    x, y = P[:, 0], P[:, 1]
    return 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))


def test_p1_row_sums_and_area():
    nr, nt = 7, 9
    m = inputs.annulus_mesh(nr, nt)
    A, M = aux.p1_matrices(m)
    assert np.abs(np.asarray(A.sum(axis=1))).max() <= 1e-13
    # boundary ring counter-clockwise: theta = 0 edge (k), outer arc (l), theta = pi/2 edge, inner arc
    ring = [k for k in range(nr)] + [l * nr + nr - 1 for l in range(1, nt)] + \
           [(nt - 1) * nr + k for k in range(nr - 2, -1, -1)] + [l * nr for l in range(nt - 2, 0, -1)]
    assert abs(M.sum() - _shoelace(m.xy[ring])) <= 1e-14


def test_coupled_mass_total_is_the_q1_domain_area():
    m = inputs.annulus_mesh(9, 11)
    n = 9
    coords = inputs.coords_quarter_annulus(n)
    C = aux.coupled_mass(m, coords)
    area = 0.0
    for cj in range(n - 1):
        for ci in range(n - 1):
            quad = np.array([[coords[0, cj, ci], coords[1, cj, ci]], [coords[0, cj, ci + 1], coords[1, cj, ci + 1]],
                             [coords[0, cj + 1, ci + 1], coords[1, cj + 1, ci + 1]],
                             [coords[0, cj + 1, ci], coords[1, cj + 1, ci]]])
            area += _shoelace(quad)
    assert abs(C.sum() - area) <= 1e-13


def _cutoff_C(m, coords, q):
    """The paper's literal rule: a q x q Gauss rule on every candidate cell,
    points outside the mapped triangle counting zero."""
    n = coords.shape[-1]
    h = 1.0 / (n - 1)
    g, w = aux.gauss01(q)
    C = np.zeros((m.xy.shape[0], n * n))
    for tri in m.tri:
        S = m.st[tri]
        d = (S[1, 0] - S[0, 0]) * (S[2, 1] - S[0, 1]) - (S[1, 1] - S[0, 1]) * (S[2, 0] - S[0, 0])
        for cj in range(n - 1):
            for ci in range(n - 1):
                X = coords[0, [cj, cj, cj + 1, cj + 1], [ci, ci + 1, ci, ci + 1]]
                Y = coords[1, [cj, cj, cj + 1, cj + 1], [ci, ci + 1, ci, ci + 1]]
                nodes = [cj * n + ci, cj * n + ci + 1, (cj + 1) * n + ci, (cj + 1) * n + ci + 1]
                for a_ in range(q):
                    for b_ in range(q):
                        s_, t_ = (ci + g[a_]) * h, (cj + g[b_]) * h
                        l1 = ((s_ - S[0, 0]) * (S[2, 1] - S[0, 1]) - (t_ - S[0, 1]) * (S[2, 0] - S[0, 0])) / d
                        l2 = ((S[1, 0] - S[0, 0]) * (t_ - S[0, 1]) - (S[1, 1] - S[0, 1]) * (s_ - S[0, 0])) / d
                        lam = np.array([1 - l1 - l2, l1, l2])
                        if lam.min() < 0:
                            continue
                        dj, phi = aux._q1_point(X, Y, g[a_], g[b_])
                        for a in range(3):
                            for b in range(4):
                                C[tri[a], nodes[b]] += w[a_] * w[b_] * dj * lam[a] * phi[b]
    return C


def test_coupled_mass_is_the_limit_of_the_cutoff_rule():
    """The oracle integrates each (triangle, cell) pair over the clipped
    polygon; the paper's cut-off Gauss rule converges to it as q grows."""
    m = inputs.annulus_mesh(4, 5, seed=3)
    n = 5
    coords = inputs.coords_quarter_annulus(n)
    exact = aux.coupled_mass(m, coords).toarray()
    errs = [np.linalg.norm(_cutoff_C(m, coords, q) - exact) / np.linalg.norm(exact) for q in (2, 8, 32)]
    assert errs[2] <= 2e-2 and errs[2] < errs[1] < errs[0], errs


def test_clipping_a_triangle_inside_a_cell_changes_nothing():
    S = np.array([[0.3, 0.2], [0.6, 0.25], [0.4, 0.7]])
    P = aux.clip_to_cell(S, np.array([0.0, 0.0]), np.array([1.0, 1.0]))
    assert len(P) == 3 and np.allclose(np.array(P)[[1, 2, 0]], S) or np.allclose(np.array(P), S)
    # a triangle covering a whole cell clips to the cell's square
    Q = aux.clip_to_cell(np.array([[-1.0, -1.0], [3.0, -1.0], [-1.0, 3.0]]), np.array([0.0, 0.0]),
                         np.array([1.0, 1.0]))
    assert abs(_shoelace(np.array(Q)) - 1.0) <= 1e-15


def test_two_cg_steps_are_galerkin_on_the_krylov_space():
    rng = np.random.default_rng(0)
    m = inputs.annulus_mesh(6, 8)
    _, M = aux.p1_matrices(m)
    iv = np.flatnonzero(~m.dirichlet)
    M = M[iv][:, iv].toarray()
    r = rng.standard_normal(len(iv))
    x = aux.cg_steps(M, r, 2)
    V = np.stack([r, M @ r], axis=1)
    assert np.abs(V.T @ (M @ x - r)).max() <= 1e-12 * np.abs(V.T @ r).max()


def test_lanczos_to_full_dimension_gives_the_mean_eigenvalue():
    rng = np.random.default_rng(1)
    N = 9
    Q = rng.standard_normal((N, N))
    B = Q @ Q.T + N * np.eye(N)
    R = rng.standard_normal((N, N))
    Ac = R @ R.T + N * np.eye(N)
    lam = sla.eigh(B, Ac, eigvals_only=True)
    g, ritz = aux.gamma_lanczos(lambda x: B @ x, lambda x: Ac @ x, lambda x: np.linalg.solve(Ac, x),
                                rng.standard_normal(N), k=N)
    assert abs(g - lam.mean()) <= 1e-10 * abs(lam.mean())
    g4, ritz4 = aux.gamma_lanczos(lambda x: B @ x, lambda x: Ac @ x, lambda x: np.linalg.solve(Ac, x),
                                  rng.standard_normal(N), k=4)
    assert lam.min() - 1e-12 <= ritz4.min() and ritz4.max() <= lam.max() + 1e-12


@pytest.mark.parametrize("mass_steps", [0, 3])
def test_two_grid_converges_on_a_small_annulus(mass_steps):
    m = inputs.annulus_mesh(25, 37)
    n = 17
    coords = inputs.coords_quarter_annulus(n)
    Ac = oracle.assemble(coords, np.ones((n - 1, n - 1)))
    tg = aux.TwoGrid(m, coords, Ac, mass_steps=mass_steps)
    u, it, hist = tg.solve(m.f, tol=1e-10, maxit=200)
    assert hist[-1] <= 1e-10 and it < 100
    # the converged iterate solves the physical system
    A, _ = aux.p1_matrices(m)
    iv = tg.iv
    res = m.f[iv] - (A @ u)[iv]
    assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(m.f[iv]) * 1.0001


def test_flexible_cg_around_the_cycle():
    """With the lumped mass the cycle is a symmetric preconditioner: flexible
    CG around it needs fewer iterations than the stationary iteration needs
    cycles, and reaches the same solution.  With the paper's CG(2) mass
    solve the stationary iteration diverges on this mesh (cond M_p about
    10), while flexible CG around the same (non-linear) cycle converges."""
    m = inputs.annulus_mesh(25, 37)
    n = 17
    coords = inputs.coords_quarter_annulus(n)
    Ac = oracle.assemble(coords, np.ones((n - 1, n - 1)))
    tg = aux.TwoGrid(m, coords, Ac, mass_steps=0)
    us, its, _ = tg.solve(m.f, tol=1e-10)
    uf, itf, trr = tg.solve_fcg(m.f, tol=1e-10)
    assert itf < its / 2 and trr <= 2e-10
    assert np.linalg.norm(uf - us) <= 1e-8 * np.linalg.norm(us)
    tg2 = aux.TwoGrid(m, coords, Ac, mass_steps=2)
    _, _, hist = tg2.solve(m.f, tol=1e-10, maxit=40)
    assert hist[-1] > 1.0
    u2, it2, trr2 = tg2.solve_fcg(m.f, tol=1e-10)
    assert trr2 <= 2e-10 and np.linalg.norm(u2 - us) <= 1e-8 * np.linalg.norm(us)
