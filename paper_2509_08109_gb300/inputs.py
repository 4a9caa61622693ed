"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
checks.  This module holds no arithmetic of the solver itself: it only
samples maps (nodal coordinates), coefficient fields and right-hand sides.

Grid convention: ``n = 2**k + 1`` nodes per side on the computational
square/cube ``[0,1]^d``; numpy arrays are C ordered with the fastest axis
last, i.e. ``coords[c, j, i]`` / ``coords[c, k, j, i]``; ``kappa`` holds one
value per cell, indexed by the cell's lower corner.

Workloads (the paper's Sec. 4 domains that have analytic maps):
  * quarter annulus r in [1/2, 1], theta in [0, pi/2] (Sec. 4.1, quarter
    annulus, rotated to the first quadrant);
  * octant of the spherical shell r in [1/2, 1] (the 3-D analogue);
  * unit square with a smooth bump map x = s + a sin(pi s) sin(pi t),
    y = t + b sin(pi s) sin(pi t) (the batched family);
  * the identity map with the discontinuous coefficients of Sec. 4.1
    (circle, checkerboard, thin layer).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def _axis(n: int) -> np.ndarray:
    return np.linspace(0.0, 1.0, n)


# ------------------------------------------------------------------ maps
def coords_quarter_annulus(n: int) -> np.ndarray:
    """x = (1/2 + s/2) cos(pi t / 2), y = (1/2 + s/2) sin(pi t / 2)."""
    s = _axis(n)[None, :]
    t = _axis(n)[:, None]
    r = 0.5 + 0.5 * s
    th = 0.5 * math.pi * t
    return np.stack([r * np.cos(th), r * np.sin(th)]).astype(np.float64)


def coords_shell_octant(n: int) -> np.ndarray:
    """Spherical coordinates r = 1/2 + s/2, theta = pi t / 2, phi = pi w / 2:
    x = r sin(theta) cos(phi), y = r sin(theta) sin(phi), z = r cos(theta).
    The face t = 0 collapses onto the z axis (a Dirichlet face)."""
    s = _axis(n)[None, None, :]
    t = _axis(n)[None, :, None]
    w = _axis(n)[:, None, None]
    r = 0.5 + 0.5 * s
    th = 0.5 * math.pi * t
    ph = 0.5 * math.pi * w
    x = r * np.sin(th) * np.cos(ph)
    y = r * np.sin(th) * np.sin(ph)
    z = r * np.cos(th) * np.ones_like(ph)
    return np.stack(np.broadcast_arrays(x, y, z)).astype(np.float64)


def coords_bump(n: int, a: float, b: float) -> np.ndarray:
    """x = s + a sin(pi s) sin(pi t), y = t + b sin(pi s) sin(pi t)."""
    s = _axis(n)[None, :]
    t = _axis(n)[:, None]
    bump = np.sin(math.pi * s) * np.sin(math.pi * t)
    return np.stack([s + a * bump, t + b * bump]).astype(np.float64)


def coords_identity(n: int, dim: int = 2) -> np.ndarray:
    """x = s (and y = t, z = w)."""
    return np.stack([_identity_component(n, dim, c) for c in range(dim)])


def _identity_component(n: int, dim: int, c: int) -> np.ndarray:
    shape = [1] * dim
    shape[dim - 1 - c] = n          # component c varies along numpy axis dim-1-c
    v = _axis(n).reshape(shape)
    return np.ascontiguousarray(np.broadcast_to(v, (n,) * dim), dtype=np.float64)


def cell_centroids(coords: np.ndarray) -> np.ndarray:
    """Mean of each cell's 2**d nodal coordinates, shape (d, n-1, ...)."""
    d = coords.shape[0]
    acc = 0.0
    for corner in range(1 << d):
        sl = [slice(None)] * (d + 1)
        for a in range(d):                      # a = 0 is the fastest (last) axis
            bit = (corner >> a) & 1
            sl[d - a] = slice(1, None) if bit else slice(0, -1)
        acc = acc + coords[tuple(sl)]
    return acc / float(1 << d)


# ------------------------------------------------------------------ fields
@dataclass
class GaussianField:
    """Random-Fourier-feature sample of a zero-mean Gaussian field with
    covariance sigma^2 exp(-|dx|^2 / (2 ell^2)):
    g(x) = sigma sqrt(2/M) sum_m cos(omega_m . x + phi_m),
    omega_m ~ N(0, ell^-2 I), phi_m ~ U[0, 2 pi)."""
    omega: np.ndarray      # (M, d)
    phase: np.ndarray      # (M,)
    sigma: float = 1.0

    @classmethod
    def draw(cls, rng: np.random.Generator, dim: int, modes: int = 64, ell: float = 0.05,
             sigma: float = 1.0) -> "GaussianField":
        omega = rng.normal(0.0, 1.0 / ell, size=(modes, dim))
        phase = rng.uniform(0.0, 2.0 * math.pi, size=modes)
        return cls(omega, phase, sigma)

    def __call__(self, pts, chunk: int = 1 << 22):
        """pts shape (d, ...) -> g shape (...).  pts may be a numpy array or a
        torch tensor (evaluated on the tensor's device, FP64)."""
        if not isinstance(pts, np.ndarray):
            return self._torch(pts, chunk)
        d = pts.shape[0]
        flat = pts.reshape(d, -1)
        out = np.empty(flat.shape[1])
        M = self.omega.shape[0]
        scale = self.sigma * math.sqrt(2.0 / M)
        for s0 in range(0, flat.shape[1], chunk):
            blk = flat[:, s0:s0 + chunk]
            arg = self.omega @ blk + self.phase[:, None]
            out[s0:s0 + chunk] = scale * np.cos(arg).sum(axis=0)
        return out.reshape(pts.shape[1:])

    def _torch(self, pts, chunk: int):
        import torch
        d = pts.shape[0]
        flat = pts.reshape(d, -1).to(torch.float64)
        om = torch.as_tensor(self.omega, dtype=torch.float64, device=flat.device)
        ph = torch.as_tensor(self.phase, dtype=torch.float64, device=flat.device)
        scale = self.sigma * math.sqrt(2.0 / om.shape[0])
        out = torch.empty(flat.shape[1], dtype=torch.float64, device=flat.device)
        for s0 in range(0, flat.shape[1], chunk):
            arg = om @ flat[:, s0:s0 + chunk] + ph[:, None]
            out[s0:s0 + chunk] = scale * torch.cos(arg).sum(dim=0)
        return out.reshape(pts.shape[1:])


def rhs_uniform(rng: np.random.Generator, shape) -> np.ndarray:
    """f ~ U[-1, 1] per node, boundary entries zero (they are ignored)."""
    f = rng.uniform(-1.0, 1.0, size=shape)
    zero_boundary(f)
    return f


def zero_boundary(v: np.ndarray) -> np.ndarray:
    for ax in range(v.ndim):
        idx = [slice(None)] * v.ndim
        idx[ax] = 0
        v[tuple(idx)] = 0.0
        idx[ax] = -1
        v[tuple(idx)] = 0.0
    return v


# ------------------------------------------------------------------ workloads
@dataclass
class Problem:
    name: str
    dim: int
    n: int
    coords: np.ndarray
    kappa: np.ndarray
    rhs: np.ndarray                      # (nrhs, n, n[, n]) or (n, n[, n])
    extra: dict = field(default_factory=dict)

    @property
    def unknowns(self) -> int:
        return (self.n - 2) ** self.dim


def annulus_plain(n: int = 65, seed: int = 0) -> Problem:
    """Quarter annulus, kappa = 1, f ~ U[-1,1] per node (seed 0)."""
    rng = np.random.default_rng(seed)
    coords = coords_quarter_annulus(n)
    kappa = np.ones((n - 1, n - 1))
    f = rhs_uniform(rng, (n, n))
    return Problem(f"annulus_plain_n{n}", 2, n, coords, kappa, f)


def annulus_lognormal(n: int = 4097, seed: int = 1) -> Problem:
    """Quarter annulus, kappa = exp(g), g a Gaussian field with 64 random
    Fourier modes (sigma 1, correlation length 0.05) evaluated at the cell
    centroids; f ~ U[-1,1].  Draw order: omega, phase, then f."""
    rng = np.random.default_rng(seed)
    coords = coords_quarter_annulus(n)
    gf = GaussianField.draw(rng, 2)
    kappa = np.exp(gf(cell_centroids(coords)))
    f = rhs_uniform(rng, (n, n))
    return Problem(f"annulus_lognormal_n{n}", 2, n, coords, kappa, f, {"field": gf})


def annulus_lognormal_device(n: int, device, seed: int = 1):
    """The annulus_lognormal workload with the field evaluated by torch on
    `device` (same draws and formula; the cosine sums may differ from the
    numpy evaluation in the last bits).  Returns (coords, kappa, f) as FP64
    tensors on the device."""
    import torch
    rng = np.random.default_rng(seed)
    coords = torch.as_tensor(coords_quarter_annulus(n), device=device)
    gf = GaussianField.draw(rng, 2)
    cen = 0.25 * (coords[:, :-1, :-1] + coords[:, :-1, 1:] + coords[:, 1:, :-1] + coords[:, 1:, 1:])
    kappa = torch.exp(gf(cen)).contiguous()
    f = torch.as_tensor(rhs_uniform(rng, (n, n)), device=device)
    return coords.contiguous(), kappa, f


def shell_two_layer(n: int = 257, seed: int = 2) -> Problem:
    """Spherical-shell octant, kappa = 1 for r < 3/4 and 1000 for r >= 3/4,
    r taken at the cell centre in computational coordinates
    (r = 1/2 + s/2, so r = 3/4 is the grid plane s = 1/2); f ~ U[-1,1]."""
    rng = np.random.default_rng(seed)
    coords = coords_shell_octant(n)
    sc = (np.arange(n - 1) + 0.5) / (n - 1)
    r = 0.5 + 0.5 * sc
    kap_1d = np.where(r < 0.75, 1.0, 1000.0)
    kappa = np.broadcast_to(kap_1d[None, None, :], (n - 1,) * 3).copy()
    f = rhs_uniform(rng, (n, n, n))
    return Problem(f"shell_two_layer_n{n}", 3, n, coords, kappa, f)


def annulus_adjoint(n: int = 1025, batch: int = 8, seed_m: int = 3, seed_obs: int = 4) -> list:
    """Per-cell parameter m ~ N(0, 0.5^2) (seed 3), kappa = exp(m); u_obs and
    f ~ U[-1,1] (seed 4, u_obs first).  One Problem per batch member."""
    rng_m = np.random.default_rng(seed_m)
    rng_o = np.random.default_rng(seed_obs)
    coords = coords_quarter_annulus(n)
    out = []
    ms = [rng_m.normal(0.0, 0.5, size=(n - 1, n - 1)) for _ in range(batch)]
    for b in range(batch):
        u_obs = rhs_uniform(rng_o, (n, n))
        f = rhs_uniform(rng_o, (n, n))
        out.append(Problem(f"annulus_adjoint_n{n}_b{b}", 2, n, coords, np.exp(ms[b]), f,
                           {"m": ms[b], "u_obs": u_obs}))
    return out


def bump_batch(count: int = 512, seed: int = 5, kmin: int = 6, kmax: int = 10, nrhs: int = 4,
               first: int = 0, limit: int | None = None) -> list:
    """Independent unit-square bump-map problems with n = 2**k + 1, k uniform
    in {kmin..kmax}; a, b ~ U[-0.15, 0.15]; log-normal kappa as in the
    annulus workload; nrhs right-hand sides ~ U[-1,1].  Problem p draws, in
    order: k, a, b, omega, phase, then its right-hand sides."""
    rng = np.random.default_rng(seed)
    probs = []
    stop = count if limit is None else min(count, first + limit)
    for p in range(count):
        k = int(rng.integers(kmin, kmax + 1))
        a, b = rng.uniform(-0.15, 0.15, size=2)
        n = (1 << k) + 1
        gf = GaussianField.draw(rng, 2)
        if p < first or p >= stop:
            rng.uniform(-1.0, 1.0, size=(nrhs, n, n))     # keep the stream aligned
            continue
        coords = coords_bump(n, a, b)
        kappa = np.exp(gf(cell_centroids(coords)))
        rhs = rng.uniform(-1.0, 1.0, size=(nrhs, n, n))
        for r in range(nrhs):
            zero_boundary(rhs[r])
        probs.append(Problem(f"bump_{p}_n{n}", 2, n, coords, kappa, rhs, {"a": a, "b": b, "k": k}))
    return probs


def annulus_anisotropic(n: int = 257, eps: float = 0.1, seed: int = 6) -> Problem:
    """Quarter annulus with an SPD diffusion tensor per cell (Sec. 2, Eq. pde):
    D = e_r e_r^T + eps e_t e_t^T, radial diffusion eps^-1 times stronger than
    tangential, e_r the radial unit vector at the cell centroid; planes
    D11, D12, D22 in extra['D'] (kappa holds the trace / 2 for reference);
    f ~ U[-1,1]."""
    rng = np.random.default_rng(seed)
    coords = coords_quarter_annulus(n)
    cen = cell_centroids(coords)
    phi = np.arctan2(cen[1], cen[0])
    c, s = np.cos(phi), np.sin(phi)
    D = np.stack([c * c + eps * s * s, (1.0 - eps) * c * s, s * s + eps * c * c])
    f = rhs_uniform(rng, (n, n))
    return Problem(f"annulus_anisotropic_n{n}", 2, n, coords, 0.5 * (D[0] + D[2]), f, {"D": D, "eps": eps})


def shell_anisotropic(n: int = 33, eps: float = 0.1, seed: int = 7) -> Problem:
    """Spherical-shell octant with D = e_r e_r^T + eps (I - e_r e_r^T) per
    cell; planes D11, D12, D13, D22, D23, D33 in extra['D']; f ~ U[-1,1]."""
    rng = np.random.default_rng(seed)
    coords = coords_shell_octant(n)
    cen = cell_centroids(coords)
    r = np.sqrt((cen ** 2).sum(axis=0))
    e = cen / r
    M = [[eps * (a == b) + (1.0 - eps) * e[a] * e[b] for b in range(3)] for a in range(3)]
    D = np.stack([M[0][0], M[0][1], M[0][2], M[1][1], M[1][2], M[2][2]])
    f = rhs_uniform(rng, (n, n, n))
    return Problem(f"shell_anisotropic_n{n}", 3, n, coords, (D[0] + D[3] + D[5]) / 3.0, f, {"D": D, "eps": eps})


def boundary_star(n: int, amp: float = 0.0, lobes: int = 5) -> np.ndarray:
    """Boundary map phi from the unit square to the star-shaped curve
    r(theta) = 1 + amp cos(lobes theta) around the origin (amp = 0: the unit
    disk), as nodal values on the boundary of an n x n grid (interior zero),
    shape (2, n, n).  The square's boundary is walked counterclockwise from
    the corner (0, 0) at unit speed and the perimeter fraction tau goes to
    theta = 2 pi tau - 3 pi / 4, so corners map to the diagonals; for a convex
    curve this map is unimodal in each coordinate."""
    g = np.zeros((2, n, n))
    h = 1.0 / (n - 1)
    for j in range(n):
        for i in range(n):
            if 0 < i < n - 1 and 0 < j < n - 1:
                continue
            x, y = i * h, j * h
            if j == 0:
                tau = x
            elif i == n - 1:
                tau = 1.0 + y
            elif j == n - 1:
                tau = 3.0 - x
            else:
                tau = 4.0 - y
            th = 2.0 * math.pi * tau / 4.0 - 0.75 * math.pi
            r = 1.0 + amp * math.cos(lobes * th)
            g[0, j, i] = r * math.cos(th)
            g[1, j, i] = r * math.sin(th)
    return g


def identity_coefficient(n: int, kind: str, seed: int = 0) -> Problem:
    """Identity map on [0,1]^2 with a Sec. 4.1 coefficient evaluated at the
    cell centre: 'circle' (100 inside r < 3/5, else 1), 'checkerboard'
    (100 where floor(4x)+floor(4y) is even, else 1), 'thin_layer' (1e-10 for
    0 <= x < 0.06, else 2)."""
    rng = np.random.default_rng(seed)
    coords = coords_identity(n, 2)
    c = cell_centroids(coords)
    x, y = c[0], c[1]
    if kind == "circle":
        kappa = np.where(np.hypot(x, y) < 0.6, 100.0, 1.0)
    elif kind == "checkerboard":
        kappa = np.where((np.floor(4 * x) + np.floor(4 * y)) % 2 == 0, 100.0, 1.0)
    elif kind == "thin_layer":
        kappa = np.where(x < 0.06, 1e-10, 2.0)
    else:
        raise ValueError(kind)
    f = rhs_uniform(rng, (n, n))
    return Problem(f"identity_{kind}_n{n}", 2, n, coords, kappa, f)


# ------------------------------------------------------------------ physical meshes
@dataclass
class Mesh:
    """A P1 triangulation of a physical domain and the images of its
    vertices in the computational square.

    xy:        (nv, 2) physical vertex coordinates
    st:        (nv, 2) computational coordinates T(xy) of the vertices
    tri:       (nt, 3) int32 vertex indices, counter-clockwise in both spaces
    dirichlet: (nv,) bool, boundary vertices (eliminated)
    kappa:     (nt,) diffusion coefficient per triangle
    f:         (nv,) load vector, U[-1, 1] on interior vertices, 0 on the boundary
    """
    name: str
    xy: np.ndarray
    st: np.ndarray
    tri: np.ndarray
    dirichlet: np.ndarray
    kappa: np.ndarray
    f: np.ndarray


def annulus_mesh(nr: int, nt: int, jitter: float = 0.2, seed: int = 8) -> Mesh:
    """Jittered polar triangulation of the quarter annulus r in [1/2, 1],
    theta in [0, pi/2] (the domain of coords_quarter_annulus): nr x nt
    vertices on the lattice r_k = 1/2 + k / (2 (nr-1)), theta_l = pi l /
    (2 (nt-1)); interior vertices moved by up to `jitter` lattice spacings
    in r and theta (uniform, seed); each lattice quad split along the
    diagonal (k+l) % 2 selects.  No triangle folds for jitter < 1/4: every
    vertex starts at least 1/sqrt(2) spacings from the opposite side, and
    moving it and that side's ends by at most sqrt(2) jitter each changes
    the distance by at most 2 sqrt(2) jitter.  T maps (r, theta) to s = 2 r - 1,
    t = 2 theta / pi, so boundary vertices land on the square's sides and
    the mapped triangles tile [0, 1]^2.  kappa = 1 (the paper's default,
    D = I); f ~ U[-1, 1] per interior vertex, drawn after the jitter."""
    rng = np.random.default_rng(seed)
    k = np.arange(nr)[None, :] * np.ones((nt, 1))
    l = np.arange(nt)[:, None] * np.ones((1, nr))
    dr = rng.uniform(-jitter, jitter, size=(nt, nr))
    dt = rng.uniform(-jitter, jitter, size=(nt, nr))
    inner = (k > 0) & (k < nr - 1) & (l > 0) & (l < nt - 1)
    kk = k + np.where(inner, dr, 0.0)
    ll = l + np.where(inner, dt, 0.0)
    r = 0.5 + 0.5 * kk / (nr - 1)
    th = 0.5 * math.pi * ll / (nt - 1)
    xy = np.stack([r * np.cos(th), r * np.sin(th)], axis=-1).reshape(-1, 2)
    st = np.stack([2.0 * r - 1.0, 2.0 * th / math.pi], axis=-1).reshape(-1, 2)
    # exact images on the boundary
    st = st.copy()
    kf, lf = k.reshape(-1), l.reshape(-1)
    st[kf == 0, 0] = 0.0
    st[kf == nr - 1, 0] = 1.0
    st[lf == 0, 1] = 0.0
    st[lf == nt - 1, 1] = 1.0
    dirichlet = ~inner.reshape(-1)
    v = lambda kq, lq: lq * nr + kq
    K, L = np.meshgrid(np.arange(nr - 1), np.arange(nt - 1))
    K, L = K.reshape(-1), L.reshape(-1)
    a, b, c, d = v(K, L), v(K + 1, L), v(K + 1, L + 1), v(K, L + 1)   # quad corners, counter-clockwise
    alt = ((K + L) % 2) == 0
    t1 = np.where(alt[:, None], np.stack([a, b, c], 1), np.stack([a, b, d], 1))
    t2 = np.where(alt[:, None], np.stack([a, c, d], 1), np.stack([b, c, d], 1))
    tri = np.concatenate([t1, t2]).astype(np.int32)
    f = np.where(dirichlet, 0.0, rng.uniform(-1.0, 1.0, size=nr * nt))
    kappa = np.ones(tri.shape[0])
    return Mesh(f"annulus_mesh_{nr}x{nt}", xy, st, tri, dirichlet, kappa, f)


def square_mesh(nx: int, ny: int, jitter: float = 0.2, seed: int = 10, kappa_sigma: float = 0.0) -> Mesh:
    """Jittered triangulation of the unit square with the identity as T
    (st = xy): nx x ny lattice vertices, interior ones moved by up to
    `jitter` spacings, quads split along alternating diagonals; kappa per
    triangle exp(N(0, kappa_sigma^2)) (1 when kappa_sigma is 0); f ~ U[-1, 1]
    on interior vertices.  Drawn in that order from one seeded generator."""
    rng = np.random.default_rng(seed)
    k = np.arange(nx)[None, :] * np.ones((ny, 1))
    l = np.arange(ny)[:, None] * np.ones((1, nx))
    inner = (k > 0) & (k < nx - 1) & (l > 0) & (l < ny - 1)
    dk = rng.uniform(-jitter, jitter, size=(ny, nx))
    dl = rng.uniform(-jitter, jitter, size=(ny, nx))
    x = (k + np.where(inner, dk, 0.0)) / (nx - 1)
    y = (l + np.where(inner, dl, 0.0)) / (ny - 1)
    xy = np.stack([x, y], axis=-1).reshape(-1, 2)
    v = lambda kq, lq: lq * nx + kq
    K, L = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1))
    K, L = K.reshape(-1), L.reshape(-1)
    a, b, c, d = v(K, L), v(K + 1, L), v(K + 1, L + 1), v(K, L + 1)
    alt = ((K + L) % 2) == 0
    t1 = np.where(alt[:, None], np.stack([a, b, c], 1), np.stack([a, b, d], 1))
    t2 = np.where(alt[:, None], np.stack([a, c, d], 1), np.stack([b, c, d], 1))
    tri = np.concatenate([t1, t2]).astype(np.int32)
    kappa = np.exp(rng.normal(0.0, kappa_sigma, size=tri.shape[0])) if kappa_sigma > 0 else np.ones(tri.shape[0])
    dirichlet = ~inner.reshape(-1)
    f = np.where(dirichlet, 0.0, rng.uniform(-1.0, 1.0, size=nx * ny))
    return Mesh(f"square_mesh_{nx}x{ny}", xy, xy.copy(), tri, dirichlet, kappa, f)
