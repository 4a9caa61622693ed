"""The ORACLE: test infrastructure only.

A plain, slow, single-threaded FP64 CPU restatement of the structured
black-box multigrid solve (paper Sec. 2, Sec. 2.1, Sec. 2.2) written in C
(``bmg_oracle.c``) and wrapped here with ctypes and numpy.  It exists to
check the CUDA library; nothing in the product imports it.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may load it.

Array conventions (numpy, C order, so the last axis is the fastest, i):
  grid vectors   shape (n, n) or (n, n, n)          [j, i] / [k, j, i]
  coords         shape (d, n, n[, n])               physical component first
  kappa          shape (n-1, n-1[, n-1])            one value per cell
  tensor         shape (3 | 6, n-1, n-1[, n-1])     upper triangle per cell:
                 D11, D12, D22 (2-D); D11, D12, D13, D22, D23, D33 (3-D)
  full stencil   shape (n, n[, n], 3**d)            slot (dx+1)+3(dy+1)+9(dz+1)
  interpolation  shape (n, n[, n], 2**d)            weight of a fine node to the
                 coarse node (i>>1 + sx, j>>1 + sy, k>>1 + sz), s = sx+2sy+4sz

Parity pins for every function live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bmg_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_SO_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lib = None
_lib_omp = None

_ERRORS = {1: "bad argument", 2: "map folded (det J <= 0)", 3: "setup breakdown",
           4: "operator not SPD", 5: "not converged", 6: "index out of range"}


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle error {code}: {_ERRORS.get(code, '?')}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math), and the same
    source with -fopenmp (liboracle_omp.so, for timing on all cores; its
    shared loops are race-free, so its results are bitwise the same)."""
    for so, extra in ((_SO, []), (_SO_OMP, ["-fopenmp"])):
        if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(_SRC):
            tmp = so + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", *extra, "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, so)
    return _SO


def threads(n: int = 0) -> int:
    """Threads of the OpenMP build (n > 0 sets them); returns the count."""
    return _load(omp=True).or_threads(int(n))


def _load(omp: bool = False):
    global _lib, _lib_omp
    cached = _lib_omp if omp else _lib
    if cached is None:
        build()
        lib = ctypes.CDLL(_SO_OMP if omp else _SO)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        for name, args, res in [
            ("or_element", [I, P, D, P], I),
            ("or_metric", [I, P, D, D, P, P], I),
            ("or_assemble", [I, I, P, P, P], I),
            ("or_gauss_points", [I, I, P, P], I),
            ("or_load", [I, I, P, P, P], I),
            ("or_apply", [I, I, P, P, P], None),
            ("or_smooth", [I, I, P, P, P, I], None),
            ("or_interp", [I, I, P, P], I),
            ("or_rap", [I, I, P, P, P], I),
            ("or_restrict", [I, I, P, P, P], None),
            ("or_prolong", [I, I, P, P, P], None),
            ("or_hier_create", [I, I, P, ctypes.POINTER(P)], I),
            ("or_hier_free", [P], None),
            ("or_hier_levels", [P], I),
            ("or_hier_n", [P, I], I),
            ("or_hier_get_A", [P, I, P], None),
            ("or_hier_get_P", [P, I, P], None),
            ("or_vcycle", [P, P, P], None),
            ("or_vcycle32", [P, P, P], None),
            ("or_pcg", [P, P, P, D, I, I, P, P, P], I),
            ("or_adjoint_grad", [I, I, P, P, P, P], I),
            ("or_element_tensor", [I, P, P, P], I),
            ("or_assemble_tensor", [I, I, P, P, P], I),
            ("or_boundary_rhs", [I, I, P, P, P, P], I),
            ("or_threads", [I], I),
        ]:
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        if omp:
            _lib_omp = lib
        else:
            _lib = lib
    return _lib_omp if omp else _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(code: int):
    if code:
        raise OracleError(code)


def _dim_n(grid_shape):
    d = len(grid_shape)
    n = grid_shape[0]
    assert all(s == n for s in grid_shape), "square/cubic grids only"
    return d, n


# ---------------------------------------------------------------- element
def element(xe, kappa: float) -> np.ndarray:
    """Q1 element stiffness (2**d x 2**d) of one cell; xe shape (d, 2**d)."""
    xe = _f64(xe)
    d = xe.shape[0]
    K = np.zeros((1 << d, 1 << d))
    _check(_load().or_element(d, _ptr(xe), float(kappa), _ptr(K)))
    return K


def element_tensor(xe, D) -> np.ndarray:
    """Q1 element stiffness with a constant SPD tensor D (d x d) on one cell:
    the effective coefficient det J J^-1 D J^-T (Sec. 2.1) at each Gauss
    point."""
    xe = _f64(xe)
    d = xe.shape[0]
    Dm = np.zeros((3, 3))
    Dm[:d, :d] = np.asarray(D, dtype=np.float64)
    K = np.zeros((1 << d, 1 << d))
    _check(_load().or_element_tensor(d, _ptr(xe), _ptr(Dm), _ptr(K)))
    return K


def assemble_tensor(coords, D) -> np.ndarray:
    """Full stencils with an SPD diffusion tensor per cell (Sec. 2, Eq. pde),
    D given as its upper-triangle planes (see the module docstring)."""
    coords = _f64(coords)
    D = _f64(D)
    d, n = _dim_n(coords.shape[1:])
    assert D.shape == ((3 if d == 2 else 6),) + (n - 1,) * d, D.shape
    A = np.zeros(coords.shape[1:] + (3 ** d,))
    _check(_load().or_assemble_tensor(d, n, _ptr(coords), _ptr(D), _ptr(A)))
    return A


def boundary_rhs(coords, kappa, g) -> np.ndarray:
    """-A_{I,B} g: the couplings of interior nodes to the boundary nodes,
    which assembly drops, applied to Dirichlet data g (boundary values of a
    grid vector; interior values ignored).  The lift term of Sec. 2."""
    coords = _f64(coords)
    kappa = _f64(kappa)
    g = _f64(g)
    d, n = _dim_n(coords.shape[1:])
    out = np.zeros(coords.shape[1:])
    _check(_load().or_boundary_rhs(d, n, _ptr(coords), _ptr(kappa), _ptr(g), _ptr(out)))
    return out


def metric(xe, kappa: float, h: float):
    """(det dx/ds, D_c) at the 2**d Gauss points of one cell, computational
    coordinates s with spacing h.  D_c = kappa det J J^-1 J^-T (Sec. 2.1)."""
    xe = _f64(xe)
    d = xe.shape[0]
    det = np.zeros(1 << d)
    Dc = np.zeros((1 << d, 3, 3))
    _check(_load().or_metric(d, _ptr(xe), float(kappa), float(h), _ptr(det), _ptr(Dc)))
    return det, Dc[:, :d, :d]


# ---------------------------------------------------------------- assembly
def assemble(coords, kappa) -> np.ndarray:
    coords = _f64(coords)
    kappa = _f64(kappa)
    d, n = _dim_n(coords.shape[1:])
    A = np.zeros(coords.shape[1:] + (3 ** d,))
    _check(_load().or_assemble(d, n, _ptr(coords), _ptr(kappa), _ptr(A)))
    return A


def gauss_points(coords) -> np.ndarray:
    """Physical Gauss points, shape (ncells, 2**d, d) in cell order."""
    coords = _f64(coords)
    d, n = _dim_n(coords.shape[1:])
    xq = np.zeros(((n - 1) ** d, 1 << d, d))
    _check(_load().or_gauss_points(d, n, _ptr(coords), _ptr(xq)))
    return xq


def load_vector(coords, fq) -> np.ndarray:
    """Consistent Q1 load vector of f sampled at the Gauss points."""
    coords = _f64(coords)
    fq = _f64(fq)
    d, n = _dim_n(coords.shape[1:])
    b = np.zeros(coords.shape[1:])
    _check(_load().or_load(d, n, _ptr(coords), _ptr(fq), _ptr(b)))
    return b


# ---------------------------------------------------------------- operators
def apply(A, x) -> np.ndarray:
    A = _f64(A)
    x = _f64(x)
    d, n = _dim_n(x.shape)
    y = np.zeros_like(x)
    _load().or_apply(d, n, _ptr(A), _ptr(x), _ptr(y))
    return y


def smooth(A, b, x, reverse: bool = False) -> np.ndarray:
    A = _f64(A)
    b = _f64(b)
    x = _f64(x).copy()
    d, n = _dim_n(x.shape)
    _load().or_smooth(d, n, _ptr(A), _ptr(b), _ptr(x), int(reverse))
    return x


def interp(A) -> np.ndarray:
    A = _f64(A)
    grid = A.shape[:-1]
    d, n = _dim_n(grid)
    pw = np.zeros(grid + (1 << d,))
    _check(_load().or_interp(d, n, _ptr(A), _ptr(pw)))
    return pw


def rap(A, pw) -> np.ndarray:
    A = _f64(A)
    pw = _f64(pw)
    grid = A.shape[:-1]
    d, n = _dim_n(grid)
    nc = (n + 1) // 2
    Ac = np.zeros((nc,) * d + (3 ** d,))
    _check(_load().or_rap(d, n, _ptr(A), _ptr(pw), _ptr(Ac)))
    return Ac


def restrict(pw, r) -> np.ndarray:
    pw = _f64(pw)
    r = _f64(r)
    d, n = _dim_n(r.shape)
    bc = np.zeros(((n + 1) // 2,) * d)
    _load().or_restrict(d, n, _ptr(pw), _ptr(r), _ptr(bc))
    return bc


def prolong(pw, xc, x) -> np.ndarray:
    """x + P xc."""
    pw = _f64(pw)
    xc = _f64(xc)
    x = _f64(x).copy()
    d, n = _dim_n(x.shape)
    _load().or_prolong(d, n, _ptr(pw), _ptr(xc), _ptr(x))
    return x


class Hierarchy:
    """BoxMG hierarchy built from a finest full stencil.  omp=True runs it on
    the OpenMP build (the same results, on all cores)."""

    def __init__(self, A, omp: bool = False):
        A = _f64(A)
        grid = A.shape[:-1]
        self.dim, self.n = _dim_n(grid)
        self._lib = _load(omp)
        h = ctypes.c_void_p()
        _check(self._lib.or_hier_create(self.dim, self.n, _ptr(A), ctypes.byref(h)))
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None) and getattr(self, "_lib", None) is not None:
            self._lib.or_hier_free(self._h)
            self._h = None

    @property
    def nlev(self) -> int:
        return self._lib.or_hier_levels(self._h)

    def level_n(self, l: int) -> int:
        return self._lib.or_hier_n(self._h, l)

    def A(self, l: int) -> np.ndarray:
        n = self.level_n(l)
        out = np.zeros((n,) * self.dim + (3 ** self.dim,))
        self._lib.or_hier_get_A(self._h, l, _ptr(out))
        return out

    def P(self, l: int) -> np.ndarray:
        n = self.level_n(l)
        out = np.zeros((n,) * self.dim + (1 << self.dim,))
        self._lib.or_hier_get_P(self._h, l, _ptr(out))
        return out

    def vcycle(self, r) -> np.ndarray:
        r = _f64(r)
        z = np.zeros_like(r)
        self._lib.or_vcycle(self._h, _ptr(r), _ptr(z))
        return z

    def vcycle32(self, r) -> np.ndarray:
        """One V-cycle of the FP32 arm: float copies of every level's A and P,
        float arithmetic, FP64 solve on the 3-node grid; r rounded to float
        on entry, the result widened to FP64."""
        r = _f64(r)
        z = np.zeros_like(r)
        self._lib.or_vcycle32(self._h, _ptr(r), _ptr(z))
        return z

    def pcg(self, b, x0=None, tol: float = 1e-10, maxit: int = 200, flexible: bool = False,
            fp32: bool = False):
        """Returns (x, iterations, residual history, true relative residual, status).
        fp32: precondition with the FP32 V-cycle (use with flexible=True, the
        mixed-precision form); the CG vectors and dots stay FP64."""
        b = _f64(b)
        x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
        hist = np.zeros(maxit + 1)
        it = ctypes.c_int()
        trr = ctypes.c_double()
        mode = int(bool(flexible)) | (2 if fp32 else 0)
        st = self._lib.or_pcg(self._h, _ptr(b), _ptr(x), float(tol), int(maxit), mode,
                            ctypes.byref(it), _ptr(hist), ctypes.byref(trr))
        return x, it.value, hist[: it.value + 1].copy(), trr.value, st


def adjoint_grad(coords, u, lam) -> np.ndarray:
    """dL/dkappa per cell = -lambda_e^T K_e^0 u_e."""
    coords = _f64(coords)
    u = _f64(u)
    lam = _f64(lam)
    d, n = _dim_n(u.shape)
    g = np.zeros((n - 1,) * d)
    _check(_load().or_adjoint_grad(d, n, _ptr(coords), _ptr(u), _ptr(lam), _ptr(g)))
    return g


# ---------------------------------------------------------------- dense views
def interior_mask(n: int, d: int) -> np.ndarray:
    m = np.zeros((n,) * d, dtype=bool)
    m[(slice(1, n - 1),) * d] = True
    return m


def dense_operator(A) -> np.ndarray:
    """Dense matrix of the full stencil over the interior unknowns."""
    A = _f64(A)
    grid = A.shape[:-1]
    d, n = _dim_n(grid)
    idx = -np.ones(grid, dtype=np.int64)
    m = interior_mask(n, d)
    idx[m] = np.arange(m.sum())
    N = int(m.sum())
    M = np.zeros((N, N))
    offs = [np.array([(o % 3) - 1, (o // 3) % 3 - 1, o // 9 - 1][:d]) for o in range(3 ** d)]
    for pos in zip(*np.nonzero(m)):
        pos_xyz = np.array(pos[::-1])          # (i, j[, k])
        row = idx[pos]
        for o, off in enumerate(offs):
            a = A[pos + (o,)]
            if a == 0.0:
                continue
            q = tuple((pos_xyz + off)[::-1])
            col = idx[q]
            assert col >= 0, "coupling to an eliminated node"
            M[row, col] += a
    return M


def dense_interp(pw) -> np.ndarray:
    """Dense P (fine interior x coarse interior) from the slot storage."""
    pw = _f64(pw)
    grid = pw.shape[:-1]
    d, n = _dim_n(grid)
    nc = (n + 1) // 2
    mf = interior_mask(n, d)
    mc = interior_mask(nc, d)
    fidx = -np.ones(grid, dtype=np.int64)
    fidx[mf] = np.arange(mf.sum())
    cidx = -np.ones((nc,) * d, dtype=np.int64)
    cidx[mc] = np.arange(mc.sum())
    Pm = np.zeros((int(mf.sum()), int(mc.sum())))
    for pos in zip(*np.nonzero(mf)):
        ijk = np.array(pos[::-1])
        for s in range(1 << d):
            w = pw[pos + (s,)]
            if w == 0.0:
                continue
            K = (ijk >> 1) + np.array([(s >> a) & 1 for a in range(d)])
            col = cidx[tuple(K[::-1])]
            assert col >= 0, "weight to a boundary coarse node"
            Pm[fidx[pos], col] = w
    return Pm
