"""Pins of the oracle against facts fixed by the paper and by the mathematics
(closed forms, invariants, dense definitions, brute force).  CPU only.

Each test names the property it pins and the passage it comes from.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2509_08109_gb300 import inputs


def _affine_coords(n, M, c, dim):
    base = inputs.coords_identity(n, dim)
    flat = base.reshape(dim, -1)
    out = (np.asarray(M) @ flat) + np.asarray(c)[:, None]
    return np.ascontiguousarray(out.reshape(base.shape))


# ------------------------------------------------------------------ P1
def test_affine_stencil_closed_form_2d():
    """Q1 stencil of a constant metric G (affine map, Sec. 2.1): integrating
    the bilinear basis products on the unit cell by hand gives
    C = 4/3(g11+g22), W = E = -2/3 g11 + 1/3 g22, S = N = 1/3 g11 - 2/3 g22,
    SW = NE = -(g11+g22)/6 - g12/2, NW = SE = -(g11+g22)/6 + g12/2."""
    rng = np.random.default_rng(11)
    n = 9
    M = np.array([[1.3, 0.4], [-0.2, 0.9]])
    kap = 2.7
    coords = _affine_coords(n, M, [0.3, -1.0], 2)
    A = oracle.assemble(coords, np.full((n - 1, n - 1), kap))
    # G in reference coordinates: J = M h, G = kappa det J J^-1 J^-T (h cancels in 2-D)
    G = kap * np.linalg.det(M) * np.linalg.inv(M) @ np.linalg.inv(M).T
    g11, g12, g22 = G[0, 0], G[0, 1], G[1, 1]
    expect = np.zeros(9)
    expect[4] = 4 / 3 * (g11 + g22)
    expect[3] = expect[5] = -2 / 3 * g11 + 1 / 3 * g22
    expect[1] = expect[7] = 1 / 3 * g11 - 2 / 3 * g22
    expect[0] = expect[8] = -(g11 + g22) / 6 - g12 / 2
    expect[6] = expect[2] = -(g11 + g22) / 6 + g12 / 2
    for j in range(2, n - 2):
        for i in range(2, n - 2):
            np.testing.assert_allclose(A[j, i], expect, rtol=0, atol=1e-13 * expect[4])
    del rng


def test_identity_stencil_3d():
    """Trilinear Q1 Laplacian on a cube of side h: h * (8/3 centre, 0 faces,
    -1/6 edges, -1/12 corners)."""
    n = 9
    h = 1.0 / (n - 1)
    coords = inputs.coords_identity(n, 3)
    A = oracle.assemble(coords, np.ones((n - 1,) * 3))
    row = A[4, 4, 4]
    for o in range(27):
        d = [(o % 3) - 1, (o // 3) % 3 - 1, o // 9 - 1]
        nz = sum(abs(x) for x in d)
        want = {0: 8 / 3, 1: 0.0, 2: -1 / 6, 3: -1 / 12}[nz] * h
        assert abs(row[o] - want) < 1e-14, (o, row[o], want)


# ------------------------------------------------------------------ P2, P3
def test_annulus_metric_closed_form():
    """Quarter annulus x = r cos(pi t/2), y = r sin(pi t/2), r = 1/2 + s/2:
    det(dx/ds) = pi r / 4 and D_c = diag(pi r, 1/(pi r)) (Sec. 2.1's D_c with
    D = I).  The isoparametric (bilinear) map reproduces det J and the
    diagonal to O(h^2) at every Gauss point; its off-diagonal shear varies
    linearly across a cell, so it is O(h) pointwise and cancels in the mean
    over the cell's four Gauss points (the map is a rotation times a
    diagonal scaling)."""
    e2, e1, em = [], [], []
    for n in (17, 33, 65):
        h = 1.0 / (n - 1)
        coords = inputs.coords_quarter_annulus(n)
        xq = oracle.gauss_points(coords)
        w2 = w1 = wm = 0.0
        for e in [0, (n - 1) * (n - 1) // 2 + 3, (n - 1) ** 2 - 1]:
            cj, ci = divmod(e, n - 1)
            xe = np.stack([coords[c][[cj, cj, cj + 1, cj + 1], [ci, ci + 1, ci, ci + 1]] for c in range(2)])
            det, Dc = oracle.metric(xe, 1.0, h)
            for q in range(4):
                r = math.hypot(*xq[e, q])
                w2 = max(w2, abs(det[q] - math.pi * r / 4) / (math.pi * r / 4))
                w2 = max(w2, abs(Dc[q, 0, 0] - math.pi * r) / (math.pi * r))
                w2 = max(w2, abs(Dc[q, 1, 1] - 1 / (math.pi * r)) * math.pi * r)
                w1 = max(w1, abs(Dc[q, 0, 1]), abs(Dc[q, 1, 0]))
            wm = max(wm, abs(Dc[:, 0, 1].mean()))
        e2.append(w2); e1.append(w1); em.append(wm)
    assert e2[-1] < 2e-4 and max(em) < 1e-12
    for i in range(2):
        assert e2[i] / e2[i + 1] > 3.5, e2
        assert 1.8 < e1[i] / e1[i + 1] < 2.2, e1


def test_shell_metric_closed_form():
    """Spherical octant r = 1/2 + s/2, theta = pi t/2, phi = pi w/2:
    det = pi^2 r^2 sin(theta) / 8, D_c = diag(pi^2 r^2 sin th / 2, sin th / 2,
    1 / (2 sin th)).  Diagonal and det to O(h^2) at each Gauss point; the
    off-diagonal shear of the trilinear map is O(h) pointwise."""
    n = 33
    h = 1.0 / (n - 1)
    coords = inputs.coords_shell_octant(n)
    ck, cj, ci = 10, 12, 7
    idx = [(ck + ((a >> 2) & 1), cj + ((a >> 1) & 1), ci + (a & 1)) for a in range(8)]
    xe = np.stack([[coords[c][t] for t in idx] for c in range(3)])
    det, Dc = oracle.metric(xe, 1.0, h)
    g = 0.5 + 0.5 / math.sqrt(3)
    gl = 0.5 - 0.5 / math.sqrt(3)
    for q in range(8):
        s = (ci + (g if q & 1 else gl)) * h
        t = (cj + (g if q & 2 else gl)) * h
        r = 0.5 + 0.5 * s
        th = 0.5 * math.pi * t
        want_det = math.pi ** 2 * r ** 2 * math.sin(th) / 8
        want = np.diag([math.pi ** 2 * r ** 2 * math.sin(th) / 2, math.sin(th) / 2, 1 / (2 * math.sin(th))])
        assert abs(det[q] - want_det) / want_det < 5e-3
        np.testing.assert_allclose(np.diag(Dc[q]), np.diag(want), rtol=5e-3)
        off = Dc[q] - np.diag(np.diag(Dc[q]))
        assert np.abs(off).max() < 0.5 * h * want.max()


@pytest.mark.parametrize("dim", [2, 3])
def test_cond_bound_is_tight_for_scalar_kappa(dim):
    """cond(D_c) <= cond(J_T)^2 cond(D) (Sec. 2.1) holds with equality when D
    is a scalar multiple of I."""
    rng = np.random.default_rng(5 + dim)
    for _ in range(5):
        M = rng.normal(size=(dim, dim)) + 2 * np.eye(dim)
        if np.linalg.det(M) < 0:
            M[:, 0] *= -1
        n = 5
        coords = _affine_coords(n, M, np.zeros(dim), dim)
        xe = np.stack([coords[c].reshape(-1)[[0, 1, n, n + 1, n * n, n * n + 1, n * n + n, n * n + n + 1][: 1 << dim]]
                       for c in range(dim)])
        _, Dc = oracle.metric(xe, 3.5, 1.0 / (n - 1))
        cD = np.linalg.cond(Dc[0])
        cJ = np.linalg.cond(M)
        assert abs(cD - cJ ** 2) / cJ ** 2 < 1e-9   # rounding grows with cond


# ------------------------------------------------------------------ P4
def _full_symmetry_error(A):
    d = A.ndim - 1
    n = A.shape[0]
    err = 0.0
    it = np.ndindex(*A.shape[:-1])
    for pos in it:
        ijk = np.array(pos[::-1])
        if np.any(ijk < 1) or np.any(ijk > n - 2):
            continue
        for o in range(3 ** d):
            off = np.array([(o % 3) - 1, (o // 3) % 3 - 1, o // 9 - 1][:d])
            q = ijk + off
            if np.any(q < 1) or np.any(q > n - 2):
                assert A[pos + (o,)] == 0.0
                continue
            o2 = 3 ** d - 1 - o
            err = max(err, abs(A[pos + (o,)] - A[tuple(q[::-1]) + (o2,)]))
    return err


@pytest.mark.parametrize("dim,n", [(2, 17), (3, 9)])
def test_levels_symmetric_and_zero_row_sums(dim, n):
    """Every level's operator is symmetric (Galerkin P^T A P of a symmetric
    A) and rows at distance >= 2 from the Dirichlet boundary have zero row
    sum (constants are in the kernel of the pure diffusion operator and
    operator-induced interpolation reproduces them)."""
    rng = np.random.default_rng(21)
    if dim == 2:
        coords = inputs.coords_bump(n, 0.12, -0.09)
    else:
        coords = inputs.coords_shell_octant(n)
        coords = coords + 0.0
    kappa = np.exp(rng.normal(0, 0.7, size=(n - 1,) * dim))
    A = oracle.assemble(coords, kappa)
    H = oracle.Hierarchy(A)
    for l in range(H.nlev):
        Al = H.A(l)
        nl = H.level_n(l)
        scale = np.abs(Al[..., (3 ** dim - 1) // 2]).max()
        assert _full_symmetry_error(Al) <= 1e-13 * scale
        if nl >= 7:
            inner = Al[(slice(2, nl - 2),) * dim].sum(axis=-1)
            assert np.abs(inner).max() <= 1e-13 * scale


# ------------------------------------------------------------------ P5
@pytest.mark.parametrize("dim,n", [(2, 17), (3, 9)])
def test_identity_map_galerkin_equals_rediscretisation(dim, n):
    """Identity map, kappa = 1: the collapse gives exactly (bi/tri)linear
    interpolation and, Q1 spaces being nested, P^T A_h P is the Q1 operator of
    the coarse grid (the same stencil in 2-D; twice the fine one in 3-D,
    where the stencil scales with h)."""
    coords = inputs.coords_identity(n, dim)
    A = oracle.assemble(coords, np.ones((n - 1,) * dim))
    P = oracle.interp(A)
    # (bi/tri)linear weights: 2^-(number of odd coordinates), interior coarse only
    for pos in np.ndindex(*P.shape[:-1]):
        ijk = np.array(pos[::-1])
        if np.any(ijk < 1) or np.any(ijk > n - 2):
            assert np.all(P[pos] == 0.0)
            continue
        nodd = int(np.sum(ijk & 1))
        for s in range(1 << dim):
            K = (ijk >> 1) + np.array([(s >> a) & 1 for a in range(dim)])
            bits = np.array([(s >> a) & 1 for a in range(dim)])
            valid = np.all((ijk & 1) | (bits == 0))   # even axes use only slot 0
            interior = np.all(K >= 1) and np.all(K <= (n + 1) // 2 - 2)
            want = 2.0 ** (-nodd) if (valid and interior) else 0.0
            assert abs(P[pos + (s,)] - want) < 1e-14, (pos, s, P[pos + (s,)], want)
    Ac = oracle.rap(A, P)
    nc = (n + 1) // 2
    A2 = oracle.assemble(inputs.coords_identity(nc, dim), np.ones((nc - 1,) * dim))
    np.testing.assert_allclose(Ac, A2, atol=1e-13)
    ctr = (3 ** dim - 1) // 2
    mid = (slice(2, 3),) * dim
    ratio = Ac[(slice(2, 3),) * dim][..., ctr] / A[mid][..., ctr]
    assert abs(float(ratio.ravel()[0]) - (1.0 if dim == 2 else 2.0)) < 1e-13


# ------------------------------------------------------------------ interpolation definition
@pytest.mark.parametrize("dim,n", [(2, 17), (3, 9)])
def test_interpolation_solves_fine_equation_at_all_odd_points(dim, n):
    """Operator-induced interpolation (Sec. 2.2) fills the points with all
    coordinates odd by solving the fine equation there: (A P v)_i = 0 for
    every coarse v.  Edge points satisfy the collapsed (line) equation."""
    rng = np.random.default_rng(3)
    coords = inputs.coords_bump(n, -0.1, 0.13) if dim == 2 else inputs.coords_shell_octant(n)
    A = oracle.assemble(coords, np.exp(rng.normal(0, 1.0, size=(n - 1,) * dim)))
    P = oracle.interp(A)
    Ad = oracle.dense_operator(A)
    Pd = oracle.dense_interp(P)
    AP = Ad @ Pd
    m = oracle.interior_mask(n, dim)
    pos = np.argwhere(m)[:, ::-1]                     # (i, j[, k]) per interior unknown
    allodd = np.all(pos & 1, axis=1)
    assert np.abs(AP[allodd]).max() < 1e-12 * np.abs(Ad).max()
    # line points: collapsed 3-point equation along the odd axis
    S = 3 ** dim
    ones = [(pos[:, a] & 1) for a in range(dim)]
    nodd = sum(ones)
    line = np.nonzero(nodd == 1)[0]
    v = rng.normal(size=Pd.shape[1])
    u = Pd @ v                                       # interpolated fine values
    uf = np.zeros((n,) * dim)
    uf[m] = u
    for r in line[:50]:
        ijk = pos[r]
        a = int(np.argmax(ijk & 1))
        coef = {-1: 0.0, 0: 0.0, 1: 0.0}
        for o in range(S):
            off = [(o % 3) - 1, (o // 3) % 3 - 1, o // 9 - 1][:dim]
            coef[off[a]] += A[tuple(ijk[::-1]) + (o,)]
        lo = ijk.copy(); lo[a] -= 1
        hi = ijk.copy(); hi[a] += 1
        res = coef[-1] * uf[tuple(lo[::-1])] + coef[0] * uf[tuple(ijk[::-1])] + coef[1] * uf[tuple(hi[::-1])]
        assert abs(res) < 1e-12 * (abs(coef[0]) * np.abs(uf).max() + 1e-300)


def test_collapse_fallback_keeps_interpolation_defined():
    """A line point whose collapsed denominator is not positive uses its own
    couplings along the line: with a hand-made row whose perpendicular
    couplings outweigh its diagonal, the weights are -a(-1,0)/a00 and
    -a(+1,0)/a00."""
    n = 5
    A = np.zeros((n, n, 9))
    for j in range(1, n - 1):
        for i in range(1, n - 1):
            A[j, i] = [-0.1, -2.0, -0.1, -1.0, 3.0, -1.0, -0.1, -2.0, -0.1]   # collapse over dy: 3 - 4 < 0
    A = A * oracle.interior_mask(n, 2)[..., None]
    for j in range(1, n - 1):
        for i in range(1, n - 1):
            for o in range(9):
                dx, dy = o % 3 - 1, o // 3 - 1
                if not (1 <= i + dx <= n - 2 and 1 <= j + dy <= n - 2):
                    A[j, i, o] = 0.0
    P = oracle.interp(A)
    # x-edge point (1, 2): weight to coarse (1, 1) is -a(+1,0)/a00 = 1/3
    assert abs(P[2, 1, 1] - 1.0 / 3.0) < 1e-15
    assert P[2, 1, 0] == 0.0          # the coarse node (0, 1) is a boundary node


def _plane_equation(A, uf, ijk, even_axis, fallback):
    """Residual of the collapsed plane equation at fine point ijk (i, j, k):
    sum over in-plane offsets o of coef[o] u(ijk + o), coef[o] the stencil
    summed over the offsets along even_axis (or, for the fallback, the
    in-plane entries alone).  Returns (residual, scale)."""
    dim = 3
    coef = {}
    for o in range(27):
        off = [(o % 3) - 1, (o // 3) % 3 - 1, o // 9 - 1]
        if fallback and off[even_axis] != 0:
            continue
        key = list(off)
        key[even_axis] = 0
        key = tuple(key)
        coef[key] = coef.get(key, 0.0) + A[tuple(ijk[::-1]) + (o,)]
    res, scale = 0.0, 0.0
    for off, c in coef.items():
        q = np.array(ijk) + np.array(off)
        val = uf[tuple(q[::-1])]
        res += c * val
        scale += abs(c) * abs(val)
    del dim
    return res, scale


def _collapsed_plane_diag(A, ijk, even_axis):
    s = 0.0
    for o in range(27):
        off = [(o % 3) - 1, (o // 3) % 3 - 1, o // 9 - 1]
        if all(off[a] == 0 for a in range(3) if a != even_axis):
            s += A[tuple(ijk[::-1]) + (o,)]
    return s


@pytest.mark.parametrize("n,sigma", [(9, 1.0), (17, 0.7)])
def test_interpolation_plane_points_3d(n, sigma):
    """Operator-induced interpolation in 3-D (Sec. 2.2 with the hierarchical
    collapse): at fine points with exactly two odd coordinates the
    interpolated value satisfies the fine equation collapsed onto the point's
    plane, i.e. summed over the one even axis, with the interpolated values
    of its in-plane neighbours.  Where that collapsed diagonal is not positive
    the point uses its own in-plane couplings (the fallback).  Checked on
    every level of a shell-octant hierarchy with a rough coefficient (at
    17^3 the input of the GPU fallback-parity test), where
    the three axes carry very different couplings, so summing over the wrong
    axis (or using the wrong neighbour set) fails; the test also confirms it
    would."""
    coords = inputs.coords_shell_octant(n)
    kappa = np.exp(np.random.default_rng(n).normal(0, sigma, size=(n - 1,) * 3))
    H = oracle.Hierarchy(oracle.assemble(coords, kappa))
    rng = np.random.default_rng(40 + n)
    checked = {False: 0, True: 0}
    wrong_axis_fails = 0
    for l in range(H.nlev - 1):
        A, P, nl = H.A(l), H.P(l), H.level_n(l)
        Pd = oracle.dense_interp(P)
        m = oracle.interior_mask(nl, 3)
        for _ in range(2):
            uf = np.zeros((nl,) * 3)
            uf[m] = Pd @ rng.normal(size=Pd.shape[1])
            for k in range(1, nl - 1):
                for j in range(1, nl - 1):
                    for i in range(1, nl - 1):
                        ijk = (i, j, k)
                        odd = [c & 1 for c in ijk]
                        if sum(odd) != 2:
                            continue
                        e = odd.index(0)
                        fallback = not (_collapsed_plane_diag(A, ijk, e) > 0)
                        res, scale = _plane_equation(A, uf, ijk, e, fallback)
                        assert abs(res) <= 1e-12 * scale + 1e-300, (l, ijk, res, scale)
                        checked[fallback] += 1
                        for wrong in range(3):
                            if wrong == e:
                                continue
                            wres, wscale = _plane_equation(A, uf, ijk, wrong, False)
                            if abs(wres) > 1e-6 * wscale:
                                wrong_axis_fails += 1
    assert checked[False] > 0
    assert wrong_axis_fails > 0.9 * 2 * (checked[False] + checked[True])
    if n == 17:
        assert checked[True] > 0      # the fallback occurs on this hierarchy (R4)


def test_plane_point_fallback_hand_built_3d():
    """A 3-D plane point whose plane-collapsed diagonal is not positive uses
    its own in-plane couplings.  Hand-built operator on 5^3 nodes with the
    same row everywhere: diagonal 3, couplings -2 along z, -1/2 to the four
    in-plane edge neighbours, -1/10 to the in-plane corners and -1/100 to
    the rest (collapsing over z gives 3 - 4 - ... < 0; collapsing a line
    point onto its axis is negative too).  Worked by hand:
      line point (2,1,2) (odd y): fallback weight -a(0,+1,0)/a00 = 1/6 to
        coarse (1,1,1); likewise (1,2,2);
      plane point (1,1,2) (even z): in-plane neighbours (2,1,2), (1,2,2)
        (weight 1/6 each) and the coarse point (2,2,2) (weight 1), so its
        weight to coarse (1,1,1) is (1/2 * 1/6 + 1/2 * 1/6 + 1/10 * 1) / 3
        = 4/45."""
    n = 5
    row = np.zeros(27)
    for o in range(27):
        dx, dy, dz = (o % 3) - 1, (o // 3) % 3 - 1, o // 9 - 1
        if (dx, dy, dz) == (0, 0, 0):
            row[o] = 3.0
        elif dx == 0 and dy == 0:
            row[o] = -2.0
        elif dz == 0 and abs(dx) + abs(dy) == 1:
            row[o] = -0.5
        elif dz == 0:
            row[o] = -0.1
        else:
            row[o] = -0.01
    A = np.zeros((n, n, n, 27))
    for k in range(1, n - 1):
        for j in range(1, n - 1):
            for i in range(1, n - 1):
                for o in range(27):
                    dx, dy, dz = (o % 3) - 1, (o // 3) % 3 - 1, o // 9 - 1
                    if 1 <= i + dx <= n - 2 and 1 <= j + dy <= n - 2 and 1 <= k + dz <= n - 2:
                        A[k, j, i, o] = row[o]
    P = oracle.interp(A)
    # slot s = sx + 2 sy + 4 sz of coarse node (i>>1 + sx, j>>1 + sy, k>>1 + sz)
    assert abs(P[2, 1, 2, 2] - 1.0 / 6.0) < 1e-15     # (2,1,2) -> (1,1,1): sx=0, sy=1, sz=0
    assert abs(P[2, 2, 1, 1] - 1.0 / 6.0) < 1e-15     # (1,2,2) -> (1,1,1): sx=1
    assert abs(P[2, 1, 1, 3] - 4.0 / 45.0) < 1e-15    # (1,1,2) -> (1,1,1): sx=sy=1
    assert np.count_nonzero(P[2, 1, 1]) == 1           # its other coarse nodes are boundary nodes


# ------------------------------------------------------------------ P6
@pytest.mark.parametrize("dim,n", [(2, 9), (2, 17), (3, 9)])
def test_rap_equals_dense_triple_product(dim, n):
    rng = np.random.default_rng(8 + n + dim)
    coords = inputs.coords_bump(n, 0.14, 0.1) if dim == 2 else inputs.coords_shell_octant(n)
    A = oracle.assemble(coords, np.exp(rng.normal(0, 1.0, size=(n - 1,) * dim)))
    P = oracle.interp(A)
    Ac = oracle.rap(A, P)
    dense = oracle.dense_interp(P).T @ oracle.dense_operator(A) @ oracle.dense_interp(P)
    np.testing.assert_allclose(oracle.dense_operator(Ac), dense, atol=1e-13 * np.abs(dense).max())


def test_restrict_and_prolong_are_transposes():
    """R = P^T (Sec. 2.3) and prolongation is x + P xc."""
    rng = np.random.default_rng(4)
    n = 17
    A = oracle.assemble(inputs.coords_quarter_annulus(n), np.exp(rng.normal(size=(n - 1, n - 1))))
    P = oracle.interp(A)
    Pd = oracle.dense_interp(P)
    r = inputs.zero_boundary(rng.normal(size=(n, n)))
    bc = oracle.restrict(P, r)
    np.testing.assert_allclose(bc[1:-1, 1:-1].ravel(), Pd.T @ r[1:-1, 1:-1].ravel(), atol=1e-14)
    xc = inputs.zero_boundary(rng.normal(size=(9, 9)))
    x = inputs.zero_boundary(rng.normal(size=(n, n)))
    y = oracle.prolong(P, xc, x)
    np.testing.assert_allclose(y[1:-1, 1:-1].ravel(), x[1:-1, 1:-1].ravel() + Pd @ xc[1:-1, 1:-1].ravel(),
                               atol=1e-14)


# ------------------------------------------------------------------ smoother
@pytest.mark.parametrize("dim,n,reverse", [(2, 9, False), (2, 9, True), (3, 5, False), (3, 5, True)])
def test_multicolour_gs_is_gauss_seidel_in_colour_order(dim, n, reverse):
    """A multicolour sweep is Gauss-Seidel on the matrix with unknowns ordered
    by colour: x_new = (D + L)^-1 (b - U x_old) in that ordering."""
    rng = np.random.default_rng(9)
    coords = inputs.coords_bump(n, 0.1, 0.1) if dim == 2 else inputs.coords_shell_octant(n)
    A = oracle.assemble(coords, np.exp(rng.normal(size=(n - 1,) * dim)))
    m = oracle.interior_mask(n, dim)
    pos = np.argwhere(m)[:, ::-1]
    colour = sum((pos[:, a] & 1) << a for a in range(dim))
    if reverse:
        colour = (1 << dim) - 1 - colour
    order = np.argsort(colour, kind="stable")
    Ad = oracle.dense_operator(A)[np.ix_(order, order)]
    b = inputs.zero_boundary(rng.normal(size=(n,) * dim))
    x0 = inputs.zero_boundary(rng.normal(size=(n,) * dim))
    x1 = oracle.smooth(A, b, x0, reverse=reverse)
    L = np.tril(Ad)
    U = Ad - L
    want = np.linalg.solve(L, b[m][order] - U @ x0[m][order])
    np.testing.assert_allclose(x1[m][order], want, atol=1e-13 * np.abs(want).max())


# ------------------------------------------------------------------ V-cycle
def _dense_vcycle_matrix(H, l):
    """M_l = (I - E_l) A_l^-1 with E_l = S_post (I - P M_{l+1} P^T A) S_pre,
    S = I - B^-1 A, B the colour-ordered GS matrix (forward / reverse):
    the error-propagation form of the V(1,1)-cycle."""
    Al = H.A(l)
    dim = H.dim
    Ad = oracle.dense_operator(Al)
    N = Ad.shape[0]
    if l == H.nlev - 1:
        return np.linalg.inv(Ad)
    n = H.level_n(l)
    pos = np.argwhere(oracle.interior_mask(n, dim))[:, ::-1]
    colour = sum((pos[:, a] & 1) << a for a in range(dim))

    def gs_matrix(rev):
        key = (1 << dim) - 1 - colour if rev else colour
        rank = np.empty(N, dtype=np.int64)
        rank[np.argsort(key, kind="stable")] = np.arange(N)
        Bm = np.where(rank[:, None] >= rank[None, :], Ad, 0.0)
        return Bm

    I = np.eye(N)
    Spre = I - np.linalg.solve(gs_matrix(False), Ad)
    Spost = I - np.linalg.solve(gs_matrix(True), Ad)
    Pd = oracle.dense_interp(H.P(l))
    Mc = _dense_vcycle_matrix(H, l + 1)
    E = Spost @ (I - Pd @ Mc @ Pd.T @ Ad) @ Spre
    return (I - E) @ np.linalg.inv(Ad)


@pytest.mark.parametrize("dim,n", [(2, 9), (2, 17), (3, 9)])
def test_vcycle_matches_error_propagation_form(dim, n):
    rng = np.random.default_rng(17)
    coords = inputs.coords_quarter_annulus(n) if dim == 2 else inputs.coords_shell_octant(n)
    A = oracle.assemble(coords, np.exp(rng.normal(0, 0.5, size=(n - 1,) * dim)))
    H = oracle.Hierarchy(A)
    M = _dense_vcycle_matrix(H, 0)
    m = oracle.interior_mask(n, dim)
    for _ in range(3):
        r = inputs.zero_boundary(rng.normal(size=(n,) * dim))
        z = H.vcycle(r)
        want = M @ r[m]
        np.testing.assert_allclose(z[m], want, atol=1e-12 * np.abs(want).max())
        assert np.all(z[~m] == 0.0)


@pytest.mark.parametrize("dim,n", [(2, 33), (3, 9)])
def test_vcycle_symmetric_positive(dim, n):
    """The forward/reverse colour order makes M symmetric positive definite,
    so it is a valid CG preconditioner: <Mx,y> = <x,My>, <Mx,x> > 0."""
    rng = np.random.default_rng(23)
    coords = inputs.coords_quarter_annulus(n) if dim == 2 else inputs.coords_shell_octant(n)
    A = oracle.assemble(coords, np.exp(rng.normal(0, 0.5, size=(n - 1,) * dim)))
    H = oracle.Hierarchy(A)
    for _ in range(3):
        x = inputs.zero_boundary(rng.normal(size=(n,) * dim))
        y = inputs.zero_boundary(rng.normal(size=(n,) * dim))
        Mx, My = H.vcycle(x), H.vcycle(y)
        a, b = float(np.sum(Mx * y)), float(np.sum(x * My))
        assert abs(a - b) <= 1e-13 * (abs(a) + abs(b)) + 1e-300
        assert float(np.sum(Mx * x)) > 0


# ------------------------------------------------------------------ P7
@pytest.mark.parametrize("dim,n", [(2, 9), (3, 9)])
@pytest.mark.parametrize("flexible", [False, True])
def test_pcg_matches_brute_force_solve(dim, n, flexible):
    rng = np.random.default_rng(31)
    coords = inputs.coords_quarter_annulus(n) if dim == 2 else inputs.coords_shell_octant(n)
    A = oracle.assemble(coords, np.exp(rng.normal(0, 0.5, size=(n - 1,) * dim)))
    b = inputs.rhs_uniform(rng, (n,) * dim)
    H = oracle.Hierarchy(A)
    x, it, hist, trr, st = H.pcg(b, tol=1e-14, maxit=200, flexible=flexible)
    assert st == 0 and trr <= 1e-14
    m = oracle.interior_mask(n, dim)
    xs = np.linalg.solve(oracle.dense_operator(A), b[m])
    assert np.abs(x[m] - xs).max() / np.abs(xs).max() < 1e-12
    assert np.all(np.diff(hist[:3]) < 0)


# ------------------------------------------------------------------ O7: the FP32 arm
_U32 = 2.0 ** -24      # unit roundoff of float (round to nearest)


def _gamma(m):
    return m * _U32 / (1 - m * _U32)


@pytest.mark.parametrize("dim,n", [(2, 9), (2, 17), (3, 9)])
def test_fp32_vcycle_is_the_vcycle_to_float_rounding(dim, n):
    """The FP32 arm evaluates the V-cycle (pinned above to its dense
    error-propagation form) with float data and float arithmetic.  By the
    standard backward-error argument each of its sums of at most m = 3^d
    terms followed by a division is the exact operation on coefficients
    perturbed by at most gamma_m = m u / (1 - m u) (u = 2^-24), and rounding
    A and P to float perturbs them by u.  A per-level relative
    perturbation of gamma_{m+1} with unit amplification through the L levels
    bounds the deviation by L gamma_{m+1} max|z|; the arm must stay inside
    that bound against the dense form, and above FP64 rounding (it really
    computes in float)."""
    rng = np.random.default_rng(19)
    coords = inputs.coords_quarter_annulus(n) if dim == 2 else inputs.coords_shell_octant(n)
    A = oracle.assemble(coords, np.exp(rng.normal(0, 0.5, size=(n - 1,) * dim)))
    H = oracle.Hierarchy(A)
    M = _dense_vcycle_matrix(H, 0)
    m = oracle.interior_mask(n, dim)
    bound = H.nlev * _gamma(3 ** dim + 1)
    for _ in range(3):
        r = inputs.zero_boundary(rng.normal(size=(n,) * dim))
        z = H.vcycle32(r)
        want = M @ r[m]
        dev = np.abs(z[m] - want).max() / np.abs(want).max()
        assert 1e-9 < dev <= bound, (dev, bound)
        assert np.all(z[~m] == 0.0)


@pytest.mark.parametrize("dim,n", [(2, 65), (2, 257), (3, 17)])
def test_fp32_vcycle_rounding_bound_at_larger_sizes(dim, n):
    """Same bound against the FP64 arm on the configurations' maps with
    their coefficients (log-normal field; two-layer shell)."""
    p = inputs.annulus_lognormal(n) if dim == 2 else inputs.shell_two_layer(n)
    H = oracle.Hierarchy(oracle.assemble(p.coords, p.kappa))
    r = inputs.rhs_uniform(np.random.default_rng(3), (n,) * dim)
    z64, z32 = H.vcycle(r), H.vcycle32(r)
    dev = np.abs(z32 - z64).max() / np.abs(z64).max()
    assert 1e-9 < dev <= H.nlev * _gamma(3 ** dim + 1), dev


@pytest.mark.parametrize("dim,n", [(2, 9), (3, 9)])
def test_fp32_flexible_pcg_matches_brute_force_solve(dim, n):
    """Flexible CG (beta = r_{k+1}.(z_{k+1} - z_k) / r_k.z_k) tolerates a
    preconditioner that is not exactly symmetric or fixed: with the FP32
    V-cycle it still reaches an FP64 residual of 1e-14 and the dense solve's
    solution."""
    rng = np.random.default_rng(31)
    coords = inputs.coords_quarter_annulus(n) if dim == 2 else inputs.coords_shell_octant(n)
    A = oracle.assemble(coords, np.exp(rng.normal(0, 0.5, size=(n - 1,) * dim)))
    b = inputs.rhs_uniform(rng, (n,) * dim)
    H = oracle.Hierarchy(A)
    x, it, hist, trr, st = H.pcg(b, tol=1e-14, maxit=200, flexible=True, fp32=True)
    assert st == 0 and trr <= 1e-14
    m = oracle.interior_mask(n, dim)
    xs = np.linalg.solve(oracle.dense_operator(A), b[m])
    assert np.abs(x[m] - xs).max() / np.abs(xs).max() < 1e-12


@pytest.mark.parametrize("dim,n", [(2, 65), (3, 17)])
def test_fp32_flexible_pcg_iterations_match_fp64(dim, n):
    """A preconditioner perturbed at the level of float rounding leaves the
    flexible-CG iteration count to 1e-10 unchanged (within one)."""
    p = inputs.annulus_lognormal(n) if dim == 2 else inputs.shell_two_layer(n)
    H = oracle.Hierarchy(oracle.assemble(p.coords, p.kappa))
    _, it32, _, trr32, st32 = H.pcg(p.rhs, tol=1e-10, maxit=500, flexible=True, fp32=True)
    _, it64, _, trr64, st64 = H.pcg(p.rhs, tol=1e-10, maxit=500, flexible=True)
    assert st32 == 0 and st64 == 0 and trr32 <= 1e-10
    assert abs(it32 - it64) <= 1


def test_pcg_zero_rhs_and_fixed_iterations():
    n = 17
    A = oracle.assemble(inputs.coords_quarter_annulus(n), np.ones((n - 1, n - 1)))
    H = oracle.Hierarchy(A)
    x, it, hist, trr, st = H.pcg(np.zeros((n, n)), tol=1e-10)
    assert st == 0 and it == 0 and np.all(x == 0)
    b = inputs.rhs_uniform(np.random.default_rng(0), (n, n))
    x, it, hist, trr, st = H.pcg(b, tol=0.0, maxit=3)
    assert st == 0 and it == 3 and len(hist) == 4


# ------------------------------------------------------------------ P8
def test_manufactured_solution_2d_second_order():
    """u = (r-1/2)(1-r) sin(2 theta) on the quarter annulus; -Lap u =
    (9r-4) sin(2 theta) / (2 r^2).  Nodal errors of the Q1 solution fall by
    about 4 per halving of h."""
    errs = []
    for n in (17, 33, 65):
        coords = inputs.coords_quarter_annulus(n)
        xq = oracle.gauss_points(coords)
        r = np.hypot(xq[..., 0], xq[..., 1])
        th = np.arctan2(xq[..., 1], xq[..., 0])
        fq = (9 * r - 4) * np.sin(2 * th) / (2 * r * r)
        b = oracle.load_vector(coords, fq)
        A = oracle.assemble(coords, np.ones((n - 1, n - 1)))
        x, it, _, trr, st = oracle.Hierarchy(A).pcg(b, tol=1e-13, maxit=100)
        assert st == 0
        R = np.hypot(coords[0], coords[1])
        TH = np.arctan2(coords[1], coords[0])
        u = (R - 0.5) * (1 - R) * np.sin(2 * TH)
        errs.append(np.abs(x - u).max())
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert 3.5 < ratios[-1] < 4.5, (errs, ratios)


def test_manufactured_solution_3d_second_order():
    """u = (r-1/2)(1-r) x y z / r^3 on the shell octant (zero on all six
    faces); f = -Lap u derived symbolically."""
    sympy = pytest.importorskip("sympy")
    X, Y, Z = sympy.symbols("x y z", real=True)
    R = sympy.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    U = (R - sympy.Rational(1, 2)) * (1 - R) * X * Y * Z / R ** 3
    F = -(sympy.diff(U, X, 2) + sympy.diff(U, Y, 2) + sympy.diff(U, Z, 2))
    f = sympy.lambdify((X, Y, Z), sympy.simplify(F), "numpy")
    u = sympy.lambdify((X, Y, Z), U, "numpy")
    errs = []
    for n in (9, 17, 33):
        coords = inputs.coords_shell_octant(n)
        xq = oracle.gauss_points(coords)
        fq = f(xq[..., 0], xq[..., 1], xq[..., 2])
        b = oracle.load_vector(coords, fq)
        A = oracle.assemble(coords, np.ones((n - 1,) * 3))
        x, it, _, trr, st = oracle.Hierarchy(A).pcg(b, tol=1e-12, maxit=300)
        assert st == 0
        m = oracle.interior_mask(n, 3)
        ue = u(coords[0], coords[1], coords[2])
        errs.append(np.abs(x[m] - ue[m]).max())
    ratio = errs[1] / errs[2]
    assert 3.0 < ratio < 5.0, errs


# ------------------------------------------------------------------ P10, P11
def test_iterations_roughly_size_independent():
    """D-MG iteration counts stay consistent as the grid is refined (Sec. 4.3)."""
    its = []
    for n in (33, 65, 129):
        p = inputs.annulus_plain(n)
        A = oracle.assemble(p.coords, p.kappa)
        _, it, _, _, st = oracle.Hierarchy(A).pcg(p.rhs, tol=1e-10, maxit=100)
        assert st == 0
        its.append(it)
    assert max(its) - min(its) <= 3, its


def test_grid_and_operator_complexity():
    """GC = sum N_l / N_1 (Sec. 4) is below 4/3 in 2-D and 8/7 in 3-D; with
    symmetric storage (5 values per DoF, Sec. 4.1) OC stays below 5*4/3."""
    for dim, n in [(2, 65), (3, 17)]:
        A = oracle.assemble(inputs.coords_identity(n, dim), np.ones((n - 1,) * dim))
        H = oracle.Hierarchy(A)
        N = [(H.level_n(l) - 2) ** dim for l in range(H.nlev)]
        gc = sum(N) / N[0]
        assert gc < (4 / 3 if dim == 2 else 8 / 7)
        nnz = [int(np.count_nonzero(H.A(l))) for l in range(H.nlev)]
        assert sum(nnz) / nnz[0] < (4 / 3 if dim == 2 else 8 / 7) + 1e-12


# ------------------------------------------------------------------ P12
def test_adjoint_gradient_matches_dense_and_central_differences():
    """dL/dm_e = kappa_e * (-lambda_e^T K_e^0 u_e) with A lambda = u - u_obs,
    L = 1/2 |u - u_obs|^2, kappa = exp(m): against central differences of the
    loss (dense solves) on a 9x9 grid."""
    n = 9
    rng = np.random.default_rng(3)
    coords = inputs.coords_quarter_annulus(n)
    mpar = rng.normal(0, 0.5, size=(n - 1, n - 1))
    u_obs = inputs.rhs_uniform(rng, (n, n))
    f = inputs.rhs_uniform(rng, (n, n))
    msk = oracle.interior_mask(n, 2)

    def solve(mm):
        Ad = oracle.dense_operator(oracle.assemble(coords, np.exp(mm)))
        u = np.zeros((n, n))
        u[msk] = np.linalg.solve(Ad, f[msk])
        return u, Ad

    u, Ad = solve(mpar)
    lam = np.zeros((n, n))
    lam[msk] = np.linalg.solve(Ad, (u - u_obs)[msk])
    g = np.exp(mpar) * oracle.adjoint_grad(coords, u, lam)
    eps = 1e-4
    for e in [(0, 0), (3, 4), (7, 7), (2, 6)]:
        mp = mpar.copy(); mp[e] += eps
        mm = mpar.copy(); mm[e] -= eps
        up, _ = solve(mp)
        um, _ = solve(mm)
        # L(+) - L(-) = 1/2 sum (u+ - u-)(u+ + u- - 2 u_obs)
        dL = 0.5 * np.sum((up - um) * (up + um - 2 * u_obs))
        fd = dL / (2 * eps)
        assert abs(fd - g[e]) <= 1e-6 * max(abs(g[e]), 1e-3 * np.abs(g).max()), (e, fd, g[e])


def test_symmetric_solve_identity():
    """<A^-1 a, b> = <a, A^-1 b> through the oracle's PCG (the adjoint solve
    reuses the forward hierarchy because A is symmetric)."""
    n = 17
    rng = np.random.default_rng(12)
    A = oracle.assemble(inputs.coords_quarter_annulus(n), np.exp(rng.normal(size=(n - 1, n - 1))))
    H = oracle.Hierarchy(A)
    a = inputs.rhs_uniform(rng, (n, n))
    b = inputs.rhs_uniform(rng, (n, n))
    xa = H.pcg(a, tol=1e-14, maxit=200)[0]
    xb = H.pcg(b, tol=1e-14, maxit=200)[0]
    s1, s2 = float(np.sum(xa * b)), float(np.sum(a * xb))
    assert abs(s1 - s2) <= 1e-12 * abs(s1)


# ---------------------------------------------------------------- tensor coefficient
def _spd(dim, rng):
    B = rng.normal(size=(dim, dim))
    return B @ B.T + 0.5 * np.eye(dim)


def _tensor_planes(D, n):
    dim = D.shape[0]
    idx = [(0, 0), (0, 1), (1, 1)] if dim == 2 else [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    return np.stack([np.full((n - 1,) * dim, D[a, b]) for a, b in idx])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tensor_stencil_closed_form_2d(seed):
    """Identity map, constant SPD D: G = D, and the Q1 nine-point row of an
    interior node is C = 4/3 (g11+g22), W = E = -2/3 g11 + 1/3 g22,
    S = N = 1/3 g11 - 2/3 g22, SW = NE = -(g11+g22)/6 - g12/2,
    NW = SE = -(g11+g22)/6 + g12/2 (exact element integrals)."""
    D = _spd(2, np.random.default_rng(seed))
    g11, g12, g22 = D[0, 0], D[0, 1], D[1, 1]
    n = 7
    A = oracle.assemble_tensor(inputs.coords_identity(n, 2), _tensor_planes(D, n))
    row = A[3, 3]
    corner_a, corner_b = -(g11 + g22) / 6 - g12 / 2, -(g11 + g22) / 6 + g12 / 2
    want = np.array([corner_a, g11 / 3 - 2 * g22 / 3, corner_b,
                     -2 * g11 / 3 + g22 / 3, 4 * (g11 + g22) / 3, -2 * g11 / 3 + g22 / 3,
                     corner_b, g11 / 3 - 2 * g22 / 3, corner_a])
    assert np.abs(row - want).max() <= 1e-14 * np.abs(want).max()


def _kron_element(D, h):
    """Exact trilinear element matrix on a cube of side h with constant D,
    K[a][b] = h sum_pq D_pq prod_r f_r, from the 1-D factors int phi' phi'
    (r = p = q), int phi_a' phi_b (r = p only), int phi_a phi_b' (r = q only)
    and int phi_a phi_b (otherwise) on [0, 1]."""
    k = np.array([[1.0, -1.0], [-1.0, 1.0]])
    m = np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])
    c = np.array([[-0.5, -0.5], [0.5, 0.5]])
    K = np.zeros((8, 8))
    for a in range(8):
        for b in range(8):
            s = 0.0
            for p in range(3):
                for q in range(3):
                    t = D[p, q]
                    for r in range(3):
                        ar, br = (a >> r) & 1, (b >> r) & 1
                        if r == p and r == q:
                            t *= k[ar, br]
                        elif r == p:
                            t *= c[ar, br]
                        elif r == q:
                            t *= c[br, ar]
                        else:
                            t *= m[ar, br]
                    s += t
            K[a, b] = h * s
    return K


@pytest.mark.parametrize("seed", [0, 1])
def test_tensor_stencil_kronecker_3d(seed):
    """Identity map, constant SPD D in 3-D: the interior row equals the sum
    of the Kronecker-built element matrices of the node's eight cells."""
    D = _spd(3, np.random.default_rng(seed))
    n = 5
    h = 1.0 / (n - 1)
    A = oracle.assemble_tensor(inputs.coords_identity(n, 3), _tensor_planes(D, n))
    K = _kron_element(D, h)
    row = np.zeros(27)
    for cell in range(8):                        # the node is corner a of the cell
        a = 7 - cell
        for b in range(8):
            d = [((b >> r) & 1) - ((a >> r) & 1) for r in range(3)]
            row[(d[0] + 1) + 3 * (d[1] + 1) + 9 * (d[2] + 1)] += K[a, b]
    got = A[2, 2, 2]
    assert np.abs(got - row).max() <= 1e-14 * np.abs(row).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_tensor_rotation_covariance(dim):
    """A rotated grid x = R xi with the rotated tensor R D0 R^T has the
    metric D0 of the unrotated one, so the stencils agree."""
    rng = np.random.default_rng(5 + dim)
    D0 = _spd(dim, rng)
    Q, _ = np.linalg.qr(rng.normal(size=(dim, dim)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    n = 5
    base = inputs.coords_identity(n, dim)
    rot = np.einsum("rc,c...->r...", Q, base)
    A0 = oracle.assemble_tensor(base, _tensor_planes(D0, n))
    A1 = oracle.assemble_tensor(rot, _tensor_planes(Q @ D0 @ Q.T, n))
    assert np.abs(A1 - A0).max() <= 1e-13 * np.abs(A0).max()


def test_tensor_of_scalar_times_identity_is_the_scalar_assembly():
    p = inputs.annulus_lognormal(17)
    D = np.stack([p.kappa, np.zeros_like(p.kappa), p.kappa])
    A1 = oracle.assemble(p.coords, p.kappa)
    A2 = oracle.assemble_tensor(p.coords, D)
    assert np.abs(A1 - A2).max() <= 1e-14 * np.abs(A1).max()


# ---------------------------------------------------------------- Dirichlet data
def test_boundary_rhs_reproduces_linear_functions():
    """Affine map, constant kappa: Q1 reproduces linear functions, so the
    discrete harmonic extension of a linear function's boundary values is
    that function (A_II x = -A_IB g solved densely)."""
    n = 9
    M = np.array([[1.1, 0.3], [-0.2, 0.8]])
    coords = _affine_coords(n, M, [0.2, -0.1], 2)
    kappa = np.full((n - 1, n - 1), 2.5)
    u = 0.7 + 1.9 * coords[0] - 1.3 * coords[1]
    rhs = oracle.boundary_rhs(coords, kappa, u)
    m = oracle.interior_mask(n, 2)
    x = np.linalg.solve(oracle.dense_operator(oracle.assemble(coords, kappa)), rhs[m])
    assert np.abs(x - u[m]).max() <= 1e-12
    assert np.all(rhs[~m] == 0.0)


@pytest.mark.parametrize("dim", [2, 3])
def test_boundary_rhs_equals_extended_grid_couplings(dim):
    """Brute force: on a grid extended by one layer of nodes, the old
    boundary nodes are interior, and the rows of the old interior nodes hold
    exactly the couplings that the Dirichlet elimination drops."""
    n = 7 if dim == 2 else 5
    rng = np.random.default_rng(30 + dim)
    if dim == 2:
        coords = inputs.coords_bump(n, 0.1, -0.08)
    else:   # an affine map with a small smooth distortion (its odd reflection stays unfolded)
        base = inputs.coords_identity(n, 3)
        bump = 0.05 * np.sin(np.pi * base[0]) * np.sin(np.pi * base[1]) * np.sin(np.pi * base[2])
        coords = _affine_coords(n, [[1.0, 0.2, 0.0], [0.1, 0.9, 0.1], [0.0, -0.1, 1.1]], [0.0, 0.0, 0.0], 3)
        coords = np.ascontiguousarray(coords + bump[None])
    kappa = np.exp(rng.normal(0, 0.5, size=(n - 1,) * dim))
    g = rng.uniform(-1, 1, size=(n,) * dim)
    ext = np.pad(coords, [(0, 0)] + [(1, 1)] * dim, mode="reflect", reflect_type="odd")
    kext = np.pad(kappa, [(1, 1)] * dim, mode="edge")
    A = oracle.assemble(ext, kext)
    inner = oracle.interior_mask(n, dim)
    want = np.zeros((n,) * dim)
    for idx in zip(*np.nonzero(inner)):
        e = tuple(v + 1 for v in idx)
        s = 0.0
        for o in range(3 ** dim):
            off = [(o % 3) - 1, (o // 3) % 3 - 1, o // 9 - 1][:dim][::-1]   # (dz,) dy, dx
            nb = tuple(v + dv for v, dv in zip(idx, off))
            if not inner[nb]:
                s -= A[e + (o,)] * g[nb]
        want[idx] = s
    got = oracle.boundary_rhs(coords, kappa, g)
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


# ------------------------------------------------------------------ the OpenMP build
@pytest.mark.parametrize("dim,n", [(2, 129), (3, 17)])
def test_openmp_build_gives_the_same_bits(dim, n):
    """The OpenMP build shares out only loops whose iterations are
    independent, so its V-cycles and CG iterates are bitwise those of the
    plain build (it exists to time the oracle on all host cores)."""
    oracle.threads(4)
    p = inputs.annulus_lognormal(n) if dim == 2 else inputs.shell_two_layer(n)
    A = oracle.assemble(p.coords, p.kappa)
    H1, H2 = oracle.Hierarchy(A), oracle.Hierarchy(A, omp=True)
    r = inputs.rhs_uniform(np.random.default_rng(2), (n,) * dim)
    assert np.array_equal(H1.vcycle(r), H2.vcycle(r))
    x1, it1, h1, t1, s1 = H1.pcg(p.rhs, tol=1e-10, maxit=400)
    x2, it2, h2, t2, s2 = H2.pcg(p.rhs, tol=1e-10, maxit=400)
    assert it1 == it2 and np.array_equal(x1, x2) and np.array_equal(h1, h2)
