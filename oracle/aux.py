"""The ORACLE for the auxiliary-space two-grid method: test infrastructure only.

A plain, slow FP64 restatement with numpy/scipy of the layer the paper puts
around the structured solve (Sec. 2.2 "Setup phase" and "Solution phase",
Sec. 2.3 Interpolation and its subsection on the coupled mass, Sec. 2.4
coarse-grid scaling):

  * P1 stiffness A_p and mass M_p on the physical triangulation (Sec. 2.1,
    V_p = P1);
  * the coupled mass C_ij = int (phi_p^i o T^-1) phi_c^j |J_T^-1| over the
    computational domain (Sec. 2.3, Eq. coupled_mass_comp), accumulated over
    (triangle, cell) pairs like the paper's cell-wise evaluation, each pair
    integrated exactly over the part of the cell the mapped triangle covers
    (the limit of the paper's cut-off Gauss rule as its order grows);
  * P = M_p^-1 C applied with two unpreconditioned CG iterations on M_p
    (Sec. 2.3), or with the lumped mass; restriction P^T (Sec. 2.3);
  * the two-grid cycle of Sec. 2.2 "Solution phase" with damped Jacobi as
    the relaxation S and one BoxMG V-cycle (``oracle.Hierarchy``) on A_c;
  * gamma, the mean of k Ritz values of the pencil (P^T A_p P, A_c) from a
    generalized Lanczos iteration (Sec. 2.4, Eqs. cgc_scaling_1, gen_eigvalue).

Nothing in the product imports this module.  Readings where the paper is
silent (relaxation, quadrature order, the images of the basis functions)
are the same as the library's and are listed with it.

Conventions: vertex vectors have one entry per mesh vertex (Dirichlet
entries zero); computational grid vectors are (n, n) arrays [j, i] with a
zero boundary, like the rest of the oracle.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from . import Hierarchy


def gauss01(q: int):
    """q-point Gauss-Legendre nodes and weights on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (x + 1.0), 0.5 * w


# ---------------------------------------------------------------- P1 operators
def p1_element(p: np.ndarray, kappa: float):
    """Stiffness and consistent mass of the P1 triangle with vertices p (3 x 2):
    K_ab = kappa |T| grad(l_a) . grad(l_b), M_ab = |T| (1 + delta_ab) / 12."""
    e = np.array([p[2] - p[1], p[0] - p[2], p[1] - p[0]])      # edge opposite vertex a
    area = 0.5 * (e[2, 0] * (-e[1, 1]) - e[2, 1] * (-e[1, 0]))
    g = np.stack([-e[:, 1], e[:, 0]], axis=1) / (2.0 * area)   # grad l_a: edge rotated by -90 deg / 2|T|
    K = kappa * area * (g @ g.T)
    M = area / 12.0 * (np.ones((3, 3)) + np.eye(3))
    return K, M, area


def p1_matrices(mesh):
    """Full (all vertices) A_p and M_p as CSR matrices."""
    nv = mesh.xy.shape[0]
    rows, cols, va, vm = [], [], [], []
    for t, tri in enumerate(mesh.tri):
        K, M, _ = p1_element(mesh.xy[tri], mesh.kappa[t])
        for a in range(3):
            for b in range(3):
                rows.append(tri[a])
                cols.append(tri[b])
                va.append(K[a, b])
                vm.append(M[a, b])
    A = sp.csr_matrix((va, (rows, cols)), shape=(nv, nv))
    M = sp.csr_matrix((vm, (rows, cols)), shape=(nv, nv))
    return A, M


# ---------------------------------------------------------------- coupled mass
def _q1_point(X, Y, xi, eta):
    """Isoparametric Q1 cell (corner order 00, 10, 01, 11): |det J| at the
    reference point (xi, eta) and the four bilinear basis values."""
    phi = np.array([(1 - xi) * (1 - eta), xi * (1 - eta), (1 - xi) * eta, xi * eta])
    dxi = np.array([-(1 - eta), 1 - eta, -eta, eta])
    deta = np.array([-(1 - xi), -xi, 1 - xi, xi])
    J11, J12 = dxi @ X, deta @ X
    J21, J22 = dxi @ Y, deta @ Y
    return abs(J11 * J22 - J12 * J21), phi


def clip_to_cell(poly, lo, hi):
    """Sutherland-Hodgman clipping of a convex polygon (list of 2-vectors)
    against the box [lo, hi], one half-plane at a time (s >= lo_s,
    s <= hi_s, t >= lo_t, t <= hi_t)."""
    P = [np.asarray(v, dtype=float) for v in poly]
    for ax in range(2):
        for bound, keep in ((lo[ax], lambda v, ax=ax, b=lo[ax]: v[ax] >= b),
                            (hi[ax], lambda v, ax=ax, b=hi[ax]: v[ax] <= b)):
            out = []
            for k in range(len(P)):
                a, b = P[k - 1], P[k]
                ka, kb = keep(a), keep(b)
                if ka != kb:
                    s_ = (bound - a[ax]) / (b[ax] - a[ax])
                    x = a + s_ * (b - a)
                    x[ax] = bound
                    out.append(x)
                if kb:
                    out.append(b)
            P = out
            if len(P) < 3:
                return []
    return P


def coupled_mass(mesh, coords: np.ndarray, q: int = 3):
    """Full C (nv x n^2, column j*n + i).  Each (triangle, cell) pair's
    contribution is integrated over their intersection in computational
    space: the mapped triangle is clipped to the cell, the clipped polygon
    is split into a fan of triangles, and each is integrated with a q x q
    Gauss rule in collapsed coordinates (exact for the integrand, which is
    of degree 4: barycentric coordinate x bilinear basis x affine det J)."""
    n = coords.shape[-1]
    h = 1.0 / (n - 1)
    gx, gw = gauss01(q)
    nv = mesh.xy.shape[0]
    rows, cols, vals = [], [], []
    for tri in mesh.tri:
        S = mesh.st[tri]                                   # mapped vertices (3 x 2)
        d = (S[1, 0] - S[0, 0]) * (S[2, 1] - S[0, 1]) - (S[1, 1] - S[0, 1]) * (S[2, 0] - S[0, 0])
        lo = np.clip(np.floor(S.min(axis=0) / h).astype(int), 0, n - 2)
        hi = np.clip(np.floor(S.max(axis=0) / h).astype(int), 0, n - 2)
        for cj in range(lo[1], hi[1] + 1):
            for ci in range(lo[0], hi[0] + 1):
                poly = clip_to_cell(S, np.array([ci * h, cj * h]), np.array([(ci + 1) * h, (cj + 1) * h]))
                if not poly:
                    continue
                X = coords[0, [cj, cj, cj + 1, cj + 1], [ci, ci + 1, ci, ci + 1]]
                Y = coords[1, [cj, cj, cj + 1, cj + 1], [ci, ci + 1, ci, ci + 1]]
                loc = np.zeros((3, 4))
                for k in range(1, len(poly) - 1):
                    v0, v1, v2 = poly[0], poly[k], poly[k + 1]
                    area2 = abs((v1[0] - v0[0]) * (v2[1] - v0[1]) - (v1[1] - v0[1]) * (v2[0] - v0[0]))
                    for a_ in range(q):
                        for b_ in range(q):
                            u, v = gx[a_], gx[b_]
                            p = v0 + u * ((v1 - v0) + v * (v2 - v1))
                            wt = gw[a_] * gw[b_] * u * area2 / (h * h)     # measure on the reference cell
                            l1 = ((p[0] - S[0, 0]) * (S[2, 1] - S[0, 1]) - (p[1] - S[0, 1]) * (S[2, 0] - S[0, 0])) / d
                            l2 = ((S[1, 0] - S[0, 0]) * (p[1] - S[0, 1]) - (S[1, 1] - S[0, 1]) * (p[0] - S[0, 0])) / d
                            lam = np.array([1.0 - l1 - l2, l1, l2])
                            dj, phi = _q1_point(X, Y, p[0] / h - ci, p[1] / h - cj)
                            loc += wt * dj * np.outer(lam, phi)
                nodes = [cj * n + ci, cj * n + ci + 1, (cj + 1) * n + ci, (cj + 1) * n + ci + 1]
                for a in range(3):
                    for b in range(4):
                        rows.append(tri[a])
                        cols.append(nodes[b])
                        vals.append(loc[a, b])
    return sp.csr_matrix((vals, (rows, cols)), shape=(nv, n * n))


# ---------------------------------------------------------------- the two-grid method
def cg_steps(M, r: np.ndarray, k: int = 2) -> np.ndarray:
    """k iterations of unpreconditioned CG on M x = r from x = 0."""
    x = np.zeros_like(r)
    res = r.copy()
    p = res.copy()
    rr = res @ res
    for _ in range(k):
        if rr == 0.0:
            break
        Mp = M @ p
        alpha = rr / (p @ Mp)
        x += alpha * p
        res -= alpha * Mp
        rr_new = res @ res
        p = res + (rr_new / rr) * p
        rr = rr_new
    return x


class TwoGrid:
    """u <- u + S r; r_c = P^T r; V-cycle on A_c; u <- u + gamma P e_c; u <- u + S r.

    S is damped Jacobi (weight omega) on A_p; P = M_p^-1 C with M_p^-1
    applied by `mass_steps` CG iterations (the paper's choice is 2), or by
    the lumped mass when mass_steps == 0."""

    def __init__(self, mesh, coords, A_c_full, q: int = 3, omega: float = 2.0 / 3.0,
                 gamma: float = 1.0, mass_steps: int = 2):
        self.mesh = mesh
        self.n = coords.shape[-1]
        A, M = p1_matrices(mesh)
        C = coupled_mass(mesh, coords, q)
        iv = np.flatnonzero(~mesh.dirichlet)
        gm = np.zeros((self.n, self.n), bool)
        gm[1:-1, 1:-1] = True
        ic = np.flatnonzero(gm.reshape(-1))
        self.iv, self.ic = iv, ic
        self.A = A[iv][:, iv].tocsr()
        self.M = M[iv][:, iv].tocsr()
        self.C = C[iv][:, ic].tocsr()
        self.H = Hierarchy(A_c_full)
        self.omega, self.gamma, self.mass_steps = omega, gamma, mass_steps
        self.dinv = 1.0 / self.A.diagonal()
        # lumped mass: the full row sum, one third of the area around the vertex
        self.mlump = np.asarray(M.sum(axis=1)).ravel()[iv]

    def minv(self, r):
        return cg_steps(self.M, r, self.mass_steps) if self.mass_steps > 0 else r / self.mlump

    def prolong(self, ec):          # ec on interior computational nodes
        return self.minv(self.C @ ec)

    def restrict(self, r):          # r on interior vertices
        return self.C.T @ self.minv(r)

    def coarse(self, rc):
        g = np.zeros(self.n * self.n)
        g[self.ic] = rc
        z = self.H.vcycle(g.reshape(self.n, self.n)).reshape(-1)
        return z[self.ic]

    def cycle(self, f, u):
        u = u + self.omega * self.dinv * (f - self.A @ u)
        ec = self.coarse(self.restrict(f - self.A @ u))
        u = u + self.gamma * self.prolong(ec)
        return u + self.omega * self.dinv * (f - self.A @ u)

    def solve(self, f_all, tol: float = 1e-10, maxit: int = 200):
        """Stationary two-grid iteration from u = 0 until ||f - A u|| <= tol ||f||
        (interior vertices).  Returns (u on all vertices, iterations, history)."""
        f = f_all[self.iv]
        u = np.zeros_like(f)
        nf = np.linalg.norm(f)
        hist = [1.0]
        it = 0
        while it < maxit and hist[-1] > tol:
            u = self.cycle(f, u)
            it += 1
            hist.append(np.linalg.norm(f - self.A @ u) / nf)
        out = np.zeros(self.mesh.xy.shape[0])
        out[self.iv] = u
        return out, it, np.array(hist)


    def solve_fcg(self, f_all, tol: float = 1e-10, maxit: int = 200):
        """Flexible CG with one cycle from a zero guess as the preconditioner
        (beta = r.(z - z_old) / r_old.z_old), until the recursive residual
        meets tol; returns (u on all vertices, iterations, true relative
        residual)."""
        f = f_all[self.iv]
        u = np.zeros_like(f)
        r = f.copy()
        nf = np.linalg.norm(f)
        z = self.cycle(r, np.zeros_like(r))
        p = z.copy()
        rz = r @ z
        it = 0
        while it < maxit:
            q = self.A @ p
            alpha = rz / (p @ q)
            u += alpha * p
            r -= alpha * q
            it += 1
            if np.linalg.norm(r) <= tol * nf:
                break
            z_old = z
            z = self.cycle(r, np.zeros_like(r))
            beta = (r @ (z - z_old)) / rz
            rz = r @ z
            p = z + beta * p
        out = np.zeros(self.mesh.xy.shape[0])
        out[self.iv] = u
        return out, it, np.linalg.norm(f - self.A @ u) / nf


# ---------------------------------------------------------------- coarse-grid scaling
def gamma_lanczos(B_apply, Ac_apply, Ac_solve, x0: np.ndarray, k: int = 12):
    """Generalized Lanczos on B x = lambda A_c x in the A_c inner product
    (the operator A_c^-1 B is A_c-self-adjoint): k steps from x0; returns
    (mean of the k Ritz values, the Ritz values)."""
    q = x0 / math.sqrt(x0 @ Ac_apply(x0))
    q_prev = np.zeros_like(q)
    beta = 0.0
    alphas, betas = [], []
    for j in range(k):
        w = Ac_solve(B_apply(q))                  # A_c^-1 B q
        alpha = w @ Ac_apply(q)
        w = w - alpha * q - beta * q_prev
        alphas.append(alpha)
        beta = math.sqrt(max(w @ Ac_apply(w), 0.0))
        if j + 1 < k:
            betas.append(beta)
            if beta == 0.0:
                break
            q_prev, q = q, w / beta
    T = np.diag(alphas) + np.diag(betas[: len(alphas) - 1], 1) + np.diag(betas[: len(alphas) - 1], -1)
    ritz = np.linalg.eigvalsh(T)
    return float(ritz.mean()), ritz
