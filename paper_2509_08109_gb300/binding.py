"""Thin ctypes binding of libbmg.so (C ABI in include/bmg.h).

Argument marshalling only: torch tensors supply device memory (the
workspace and the arrays) and the CUDA stream; every step of the solve
runs in the library's kernels.  The library must have been built
(``paper_2509_08109_gb300.build.build()``); loading fails loudly otherwise,
and there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbmg.so")
_lib = None

PREC = {"fp64": 0, "fp32": 1}
OUTER = {"cg": 0, "flexible": 1, "refine": 2}

STATUS = {0: "ok", 1: "invalid argument", 2: "unsupported shape", 3: "CUDA runtime error",
          4: "workspace missing or too small", 5: "map folded", 6: "setup breakdown",
          7: "CG breakdown (not SPD)", 8: "not converged", 9: "bounded wait expired", 10: "call out of order"}


class BmgError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: bmg status {code} ({STATUS.get(code, '?')})")
        self.code = code


class _Opts(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int), ("precision", ctypes.c_int),
                ("outer", ctypes.c_int), ("flags", ctypes.c_int), ("max_rhs", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("levels", ctypes.c_int), ("relres", ctypes.c_double),
                ("true_relres", ctypes.c_double), ("rho", ctypes.c_double),
                ("grid_complexity", ctypes.c_double), ("operator_complexity", ctypes.c_double),
                ("status", ctypes.c_int), ("refinements", ctypes.c_int)]


class _AuxOpts(ctypes.Structure):
    _fields_ = [("omega", ctypes.c_double), ("mass_steps", ctypes.c_int), ("gamma", ctypes.c_double),
                ("krylov", ctypes.c_int)]


@dataclass
class SolveInfo:
    iterations: int
    levels: int
    relres: float
    true_relres: float
    rho: float
    grid_complexity: float
    operator_complexity: float
    status: int
    refinements: int = 0


def load() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2509_08109_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    sigs = {
        "bmg_default_opts": ([ctypes.POINTER(_Opts)], None),
        "bmg_create": ([ctypes.POINTER(_Opts), ctypes.POINTER(P)], I),
        "bmg_workspace_bytes": ([P, ctypes.POINTER(ctypes.c_size_t)], I),
        "bmg_attach": ([P, P, ctypes.c_size_t, P], I),
        "bmg_assemble": ([P, P, P], I),
        "bmg_set_stencil": ([P, P], I),
        "bmg_setup": ([P], I),
        "bmg_vcycle": ([P, P, P], I),
        "bmg_solve": ([P, I, P, P, D, I, P], I),
        "bmg_adjoint_grad": ([P, I, P, P, P, P, P, D, I, P], I),
        "bmg_adjoint_cells": ([P, P, P, P, P], I),
        "bmg_solve_many": ([P, I, I, P, P, D, I, P], I),
        "bmg_levels": ([P], I),
        "bmg_level_n": ([P, I], I),
        "bmg_get_stencil": ([P, I, P], I),
        "bmg_get_interp": ([P, I, P], I),
        "bmg_launch_count": ([P], ctypes.c_longlong),
        "bmg_get_tiles": ([P, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "bmg_set_tiles": ([P, I, I, I, I], I),
        "bmg_autotune": ([P, I, ctypes.POINTER(D)], I),
        "bmg_profile": ([P, I], I),
        "bmg_profile_read": ([P, I, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(D)], I),
        "bmg_destroy": ([P], None),
        "bmg_status_str": ([I], ctypes.c_char_p),
        "bmg_assemble_noalloc": ([I, I, P, P, P, P], I),
        "bmg_assemble_tensor": ([P, P, P], I),
        "bmg_boundary_rhs": ([P, P, P, P, P], I),
        "bmg_aux_default_opts": ([ctypes.POINTER(_AuxOpts)], None),
        "bmg_aux_create": ([P, I, P, P, P, I, P, ctypes.POINTER(_AuxOpts), ctypes.POINTER(P)], I),
        "bmg_aux_workspace_bytes": ([P, ctypes.POINTER(ctypes.c_size_t)], I),
        "bmg_aux_setup": ([P, P, ctypes.c_size_t, P, P], I),
        "bmg_aux_solve": ([P, P, P, D, I, ctypes.POINTER(_Info)], I),
        "bmg_aux_set_gamma": ([P, D], I),
        "bmg_aux_estimate_gamma": ([P, I, P, D, ctypes.POINTER(D), P, P, ctypes.POINTER(I)], I),
        "bmg_aux_export": ([P, I, ctypes.POINTER(I), ctypes.POINTER(ctypes.c_longlong), P, P, P], I),
        "bmg_aux_destroy": ([P], None),
        "bmg_batch_create": ([I, P, I, ctypes.POINTER(P)], I),
        "bmg_batch_workspace_bytes": ([P, ctypes.POINTER(ctypes.c_size_t)], I),
        "bmg_batch_attach": ([P, P, ctypes.c_size_t, P], I),
        "bmg_batch_solve": ([P, I, P, P, D, I, P], I),
        "bmg_batch_classes": ([P], I),
        "bmg_batch_get_tiles": ([P, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I),
                                 ctypes.POINTER(I)], I),
        "bmg_batch_set_tiles": ([P, I, I, I], I),
        "bmg_batch_autotune": ([P, I, ctypes.POINTER(D)], I),
        "bmg_batch_launch_count": ([P], ctypes.c_longlong),
        "bmg_batch_destroy": ([P], None),
    }
    for name, (args, res) in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def exported_symbols() -> list:
    return ["bmg_default_opts", "bmg_create", "bmg_workspace_bytes", "bmg_attach", "bmg_assemble",
            "bmg_set_stencil", "bmg_setup", "bmg_vcycle", "bmg_solve", "bmg_solve_many", "bmg_adjoint_grad",
            "bmg_adjoint_cells", "bmg_levels",
            "bmg_level_n", "bmg_get_stencil", "bmg_get_interp", "bmg_launch_count", "bmg_get_tiles",
            "bmg_set_tiles", "bmg_autotune", "bmg_profile",
            "bmg_profile_read", "bmg_destroy", "bmg_status_str", "bmg_assemble_noalloc", "bmg_assemble_tensor",
            "bmg_boundary_rhs", "bmg_aux_default_opts", "bmg_aux_create", "bmg_aux_workspace_bytes",
            "bmg_aux_setup", "bmg_aux_solve", "bmg_aux_set_gamma", "bmg_aux_estimate_gamma", "bmg_aux_export",
            "bmg_aux_destroy", "bmg_batch_create", "bmg_batch_workspace_bytes", "bmg_batch_attach",
            "bmg_batch_solve", "bmg_batch_classes", "bmg_batch_get_tiles", "bmg_batch_set_tiles",
            "bmg_batch_autotune", "bmg_batch_launch_count", "bmg_batch_destroy"]


def _check(code: int, where: str):
    if code != 0:
        raise BmgError(code, where)


def _ptr(t: torch.Tensor):
    assert t.is_contiguous() and t.dtype == torch.float64, (t.dtype, t.is_contiguous())
    return ctypes.c_void_p(t.data_ptr())


def assemble_noalloc(dim: int, n: int, coords: torch.Tensor, kappa: torch.Tensor, out: torch.Tensor,
                     stream=None) -> torch.Tensor:
    """bmg_assemble_noalloc: the finest operator as full 3^dim-entry rows,
    written into `out` (device, n^dim x 3^dim doubles), without a context or
    any allocation in the library.  All tensors must already be on the
    current CUDA device; nothing is copied or allocated here either.
    The C entry point takes no lengths, so the sizes are checked here:
    coords dim * n^dim, kappa (n-1)^dim and out n^dim * 3^dim doubles
    (ValueError otherwise, before any device work)."""
    dim, n = int(dim), int(n)
    if dim in (2, 3) and n >= 3:
        for name, t, want in (("coords", coords, dim * n ** dim), ("kappa", kappa, (n - 1) ** dim),
                              ("out", out, n ** dim * 3 ** dim)):
            if t.numel() != want:
                raise ValueError(f"bmg_assemble_noalloc: {name} has {t.numel()} elements, "
                                 f"dim {dim}, n {n} needs {want}")
    for t in (coords, kappa, out):
        if not (t.dtype == torch.float64 and t.is_contiguous()):
            raise ValueError("bmg_assemble_noalloc: tensors must be contiguous float64")
        if not (t.is_cuda and t.device.index == torch.cuda.current_device()):
            raise ValueError("bmg_assemble_noalloc: tensors must be on the current CUDA device")
    s = stream if stream is not None else torch.cuda.current_stream()
    code = load().bmg_assemble_noalloc(int(dim), int(n), _ptr(coords), _ptr(kappa), _ptr(out),
                                       ctypes.c_void_p(s.cuda_stream))
    if code == 2:
        raise BmgError(code, f"bmg_assemble_noalloc: dim {dim}, n {n} is beyond the static scratch "
                             f"(n <= 640 in 2-D, n <= 48 in 3-D)")
    _check(code, "bmg_assemble_noalloc")
    return out


def _info_of(i: "_Info") -> SolveInfo:
    return SolveInfo(i.iterations, i.levels, i.relres, i.true_relres, i.rho, i.grid_complexity,
                     i.operator_complexity, i.status, i.refinements)


def solve_many(solvers, bs, xs, tol: float = 1e-10, maxit: int = 500):
    """Concurrent independent solves (library scheduler).  solvers: Solver
    objects built with precision='fp32', outer='refine', each attached to its
    own stream; bs[p] / xs[p]: lists of nrhs tensors (host or device) for
    problem p; xs hold the initial guesses and receive the solutions.
    Returns a list (per problem) of lists of SolveInfo."""
    lib = load()
    count = len(solvers)
    nrhs = len(bs[0]) if count else 1
    hs = (ctypes.c_void_p * count)(*[s._h.value for s in solvers])
    bp = (ctypes.c_void_p * (count * nrhs))()
    xp = (ctypes.c_void_p * (count * nrhs))()
    keep = []
    for p in range(count):
        assert len(bs[p]) == nrhs and len(xs[p]) == nrhs
        for r in range(nrhs):
            b = bs[p][r]
            x = xs[p][r]
            assert b.dtype == torch.float64 and x.dtype == torch.float64 and b.is_contiguous() and x.is_contiguous()
            keep += [b, x]
            bp[p * nrhs + r] = b.data_ptr()
            xp[p * nrhs + r] = x.data_ptr()
    infos = (_Info * (count * nrhs))()
    code = lib.bmg_solve_many(hs, count, nrhs, bp, xp, float(tol), int(maxit), infos)
    _check(code, "bmg_solve_many")
    return [[_info_of(infos[p * nrhs + r]) for r in range(nrhs)] for p in range(count)]


class Batch:
    """bmg_batch_*: many set-up problems (Solver objects with
    precision='fp32', outer='refine', 2-D, n >= 65, one device) solved
    together, up to four right-hand sides each.  The solvers must stay alive
    and unchanged while the batch is used."""

    def __init__(self, solvers, graphs: bool = True, stream: torch.cuda.Stream | None = None):
        lib = load()
        self.solvers = list(solvers)
        count = len(self.solvers)
        hs = (ctypes.c_void_p * count)(*[s._h.value for s in self.solvers])
        h = ctypes.c_void_p()
        _check(lib.bmg_batch_create(count, hs, 0 if graphs else 2, ctypes.byref(h)), "bmg_batch_create")
        self._h = h
        nbytes = ctypes.c_size_t()
        _check(lib.bmg_batch_workspace_bytes(h, ctypes.byref(nbytes)), "bmg_batch_workspace_bytes")
        self.workspace_bytes = nbytes.value
        self.device = self.solvers[0].device
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self._ws = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=self.device)
            _check(lib.bmg_batch_attach(h, ctypes.c_void_p(self._ws.data_ptr()),
                                        ctypes.c_size_t(self.workspace_bytes),
                                        ctypes.c_void_p(self.stream.cuda_stream)), "bmg_batch_attach")

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.bmg_batch_destroy(self._h)
            self._h = None

    @property
    def launches(self) -> int:
        return load().bmg_batch_launch_count(self._h)

    def tiles(self):
        """[(n, wc, hc, members)] per size class."""
        lib = load()
        out = []
        for c in range(lib.bmg_batch_classes(self._h)):
            n, wc, hc, m = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
            _check(lib.bmg_batch_get_tiles(self._h, c, ctypes.byref(n), ctypes.byref(wc), ctypes.byref(hc),
                                           ctypes.byref(m)), "bmg_batch_get_tiles")
            out.append((n.value, wc.value, hc.value, m.value))
        return out

    def set_tiles(self, cls: int, wc: int, hc: int):
        with torch.cuda.device(self.device):
            _check(load().bmg_batch_set_tiles(self._h, int(cls), int(wc), int(hc)), "bmg_batch_set_tiles")

    def autotune(self, reps: int = 3) -> float:
        ms = ctypes.c_double()
        with torch.cuda.device(self.device):
            _check(load().bmg_batch_autotune(self._h, int(reps), ctypes.byref(ms)), "bmg_batch_autotune")
        return ms.value

    def solve(self, bs, xs, tol: float = 1e-10, maxit: int = 500, raise_on_nonconv: bool = True):
        """bs[p] / xs[p]: lists of nrhs tensors (n_p x n_p float64, host or
        device) of problem p; xs hold the initial guesses and receive the
        solutions.  Returns (per problem) lists of SolveInfo."""
        lib = load()
        count = len(self.solvers)
        assert len(bs) == count and len(xs) == count
        nrhs = len(bs[0])
        bp = (ctypes.c_void_p * (count * nrhs))()
        xp = (ctypes.c_void_p * (count * nrhs))()
        keep = []
        for p in range(count):
            assert len(bs[p]) == nrhs and len(xs[p]) == nrhs
            n = self.solvers[p].n
            for r in range(nrhs):
                b, x = bs[p][r], xs[p][r]
                for t in (b, x):
                    if not (t.dtype == torch.float64 and t.is_contiguous() and t.numel() == n * n):
                        raise ValueError(f"problem {p}: right-hand sides and solutions must be contiguous "
                                         f"float64 {n}x{n} tensors")
                keep += [b, x]
                bp[p * nrhs + r] = b.data_ptr()
                xp[p * nrhs + r] = x.data_ptr()
        infos = (_Info * (count * nrhs))()
        with torch.cuda.device(self.device):
            code = lib.bmg_batch_solve(self._h, nrhs, bp, xp, float(tol), int(maxit), infos)
        res = [[_info_of(infos[p * nrhs + r]) for r in range(nrhs)] for p in range(count)]
        if code == 8 and not raise_on_nonconv:
            return res
        _check(code, "bmg_batch_solve")
        return res


class Solver:
    """One structured problem: n nodes per side in dim dimensions.

    precision: 'fp64' (plain) or 'fp32' (FP32 V-cycle).
    outer: 'cg', 'flexible' (FP64 flexible CG around the FP32 V-cycle) or
    'refine' (FP64 iterative refinement around an FP32 CG; fp32 only).
    Default: 'cg' for fp64, 'flexible' for fp32.
    """

    def __init__(self, dim: int, n: int, precision: str = "fp64", outer: str | None = None,
                 device=None, stream: torch.cuda.Stream | None = None, unfused: bool = False,
                 graphs: bool = True, max_rhs: int = 1):
        lib = load()
        self.dim, self.n, self.precision = dim, n, precision
        if outer is None:
            outer = "flexible" if precision == "fp32" else "cg"
        self.outer = outer
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        opts = _Opts(dim, n, PREC[precision], OUTER[outer], (1 if unfused else 0) | (0 if graphs else 2),
                     int(max_rhs))
        h = ctypes.c_void_p()
        _check(lib.bmg_create(ctypes.byref(opts), ctypes.byref(h)), "bmg_create")
        self._h = h
        nbytes = ctypes.c_size_t()
        _check(lib.bmg_workspace_bytes(h, ctypes.byref(nbytes)), "bmg_workspace_bytes")
        self.workspace_bytes = nbytes.value
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self._ws = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=self.device)
            _check(lib.bmg_attach(h, ctypes.c_void_p(self._ws.data_ptr()), ctypes.c_size_t(self.workspace_bytes),
                                  ctypes.c_void_p(self.stream.cuda_stream)), "bmg_attach")

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.bmg_destroy(self._h)
            self._h = None

    # ------------------------------------------------------------ queries
    @property
    def levels(self) -> int:
        return load().bmg_levels(self._h)

    def level_n(self, l: int) -> int:
        return load().bmg_level_n(self._h, l)

    @property
    def launches(self) -> int:
        return load().bmg_launch_count(self._h)

    @property
    def grid_shape(self):
        return (self.n,) * self.dim

    def _dev(self, t: torch.Tensor) -> torch.Tensor:
        return t.to(device=self.device, dtype=torch.float64).contiguous()

    # ------------------------------------------------------------ setup
    def assemble(self, coords, kappa):
        coords = self._dev(torch.as_tensor(coords))
        kappa = self._dev(torch.as_tensor(kappa))
        assert coords.shape == (self.dim,) + self.grid_shape, coords.shape
        assert kappa.shape == (self.n - 1,) * self.dim, kappa.shape
        with torch.cuda.device(self.device):
            _check(load().bmg_assemble(self._h, _ptr(coords), _ptr(kappa)), "bmg_assemble")
        self._coords = coords
        return self

    def assemble_tensor(self, coords, D):
        """bmg_assemble_tensor: D of shape (3, n-1, n-1) in 2-D (D11, D12,
        D22) or (6, n-1, n-1, n-1) in 3-D (D11, D12, D13, D22, D23, D33)."""
        coords = self._dev(torch.as_tensor(coords))
        D = self._dev(torch.as_tensor(D))
        assert coords.shape == (self.dim,) + self.grid_shape, coords.shape
        assert D.shape == ((3 if self.dim == 2 else 6),) + (self.n - 1,) * self.dim, D.shape
        with torch.cuda.device(self.device):
            _check(load().bmg_assemble_tensor(self._h, _ptr(coords), _ptr(D)), "bmg_assemble_tensor")
        self._coords = coords
        return self

    def boundary_rhs(self, coords, kappa, g) -> torch.Tensor:
        """bmg_boundary_rhs: -A_{I,B} g for Dirichlet data g (grid shape)."""
        coords = self._dev(torch.as_tensor(coords))
        kappa = self._dev(torch.as_tensor(kappa))
        g = self._dev(torch.as_tensor(g))
        assert g.shape == self.grid_shape, g.shape
        out = torch.empty_like(g)
        with torch.cuda.device(self.device):
            _check(load().bmg_boundary_rhs(self._h, _ptr(coords), _ptr(kappa), _ptr(g), _ptr(out)),
                   "bmg_boundary_rhs")
        return out

    def set_stencil(self, full):
        full = self._dev(torch.as_tensor(full))
        assert full.shape == self.grid_shape + (3 ** self.dim,)
        with torch.cuda.device(self.device):
            _check(load().bmg_set_stencil(self._h, _ptr(full)), "bmg_set_stencil")
        return self

    def setup(self):
        with torch.cuda.device(self.device):
            _check(load().bmg_setup(self._h), "bmg_setup")
        return self

    # ------------------------------------------------------------ solve
    def vcycle(self, r: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        r = torch.as_tensor(r, dtype=torch.float64)
        r = r.contiguous() if r.device.type == "cpu" else self._dev(r)
        if out is None:
            out = torch.empty_like(r)
        with torch.cuda.device(self.device):
            _check(load().bmg_vcycle(self._h, _ptr(r), _ptr(out)), "bmg_vcycle")
        return out

    def _nrhs_of(self, t: torch.Tensor) -> int:
        if t.dim() == self.dim:
            return 0
        if t.dim() == self.dim + 1 and tuple(t.shape[1:]) == self.grid_shape:
            return t.shape[0]
        raise ValueError(f"expected shape {self.grid_shape} or (nrhs,) + {self.grid_shape}, got {tuple(t.shape)}")

    def solve(self, b, x0=None, tol: float = 1e-10, maxit: int = 500, out=None, raise_on_nonconv=True):
        """x such that ||b - A x|| <= tol ||b||.  b (and out) may live on the
        host or the device; the result has b's device.  b of shape
        (nrhs, n, ...) solves nrhs right-hand sides in one bmg_solve call
        (together on a context created with max_rhs >= 2) and returns a
        list of SolveInfo."""
        b = torch.as_tensor(b, dtype=torch.float64)
        b = b.contiguous() if b.device.type == "cpu" else self._dev(b)
        nrhs = self._nrhs_of(b)
        if out is None:
            out = torch.zeros_like(b) if x0 is None else torch.as_tensor(x0, dtype=torch.float64).to(b.device).clone()
        elif x0 is not None:
            out.copy_(torch.as_tensor(x0))
        elif x0 is None:
            out.zero_()
        infos = (_Info * max(nrhs, 1))()
        with torch.cuda.device(self.device):
            code = load().bmg_solve(self._h, max(nrhs, 1), _ptr(b), _ptr(out), float(tol), int(maxit), infos)
        if code not in (0, 8) or (code == 8 and raise_on_nonconv):
            _check(code, "bmg_solve")
        res = [_info_of(i) for i in infos]
        return out, (res if nrhs else res[0])

    def adjoint_grad(self, u, dLdu, tol: float = 1e-10, maxit: int = 500):
        """(lambda, dL/dkappa per cell, info) for A lambda = dL/du; u and
        dLdu of shape (nrhs, n, ...) give nrhs independent gradients (one
        bmg_adjoint_grad call; info is then a list)."""
        u = self._dev(torch.as_tensor(u))
        g = self._dev(torch.as_tensor(dLdu))
        nrhs = self._nrhs_of(g)
        assert u.shape == g.shape, (u.shape, g.shape)
        lam = torch.zeros_like(g)
        cells = (self.n - 1,) * self.dim
        dk = torch.empty(((nrhs,) if nrhs else ()) + cells, dtype=torch.float64, device=self.device)
        infos = (_Info * max(nrhs, 1))()
        with torch.cuda.device(self.device):
            _check(load().bmg_adjoint_grad(self._h, max(nrhs, 1), _ptr(self._coords), _ptr(u), _ptr(g), _ptr(lam),
                                           _ptr(dk), float(tol), int(maxit), infos), "bmg_adjoint_grad")
        res = [_info_of(i) for i in infos]
        return lam, dk, (res if nrhs else res[0])

    def adjoint_cells(self, u, lam) -> torch.Tensor:
        """bmg_adjoint_cells: dL/dkappa per cell, -lambda_e^T K_e^0 u_e, for
        an adjoint lambda solved elsewhere (e.g. by solve_many)."""
        u = self._dev(torch.as_tensor(u))
        lam = self._dev(torch.as_tensor(lam))
        dk = torch.empty((self.n - 1,) * self.dim, dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            _check(load().bmg_adjoint_cells(self._h, _ptr(self._coords), _ptr(u), _ptr(lam), _ptr(dk)),
                   "bmg_adjoint_cells")
        return dk

    # ------------------------------------------------------------ tile shapes
    def tiles(self) -> list:
        """[(wc, hc, hc_up)] per level pair of the streaming kernels ([] if
        unused): strip width, rows per CTA of the down and the up kernel."""
        out = []
        for l in range(self.levels - 1):
            wc, hc, hu = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
            if load().bmg_get_tiles(self._h, l, ctypes.byref(wc), ctypes.byref(hc), ctypes.byref(hu)) != 0:
                return []
            out.append((wc.value, hc.value, hu.value))
        return out

    def set_tiles(self, tiles):
        """tiles: per level (wc, hc) or (wc, hc, hc_up); hc_up defaults to hc."""
        for l, t in enumerate(tiles):
            wc, hc = t[0], t[1]
            hu = t[2] if len(t) > 2 else hc
            _check(load().bmg_set_tiles(self._h, l, int(wc), int(hc), int(hu)), "bmg_set_tiles")

    def autotune(self, reps: int = 3, cache: str | None = None) -> list:
        """Device-timed choice of the tile shapes (bmg_autotune).  With a
        cache file (JSON), reuse the choice stored for this GPU, grid and
        precision, or store the new one."""
        import json
        key = f"{torch.cuda.get_device_name(self.device)}|d{self.dim}|n{self.n}|{self.precision}|{self.outer}"
        table = {}
        if cache and os.path.exists(cache):
            try:
                table = json.load(open(cache))
            except ValueError:
                table = {}
            if key in table:
                self.set_tiles(table[key])
                return self.tiles()
        ms = ctypes.c_double()
        with torch.cuda.device(self.device):
            _check(load().bmg_autotune(self._h, int(reps), ctypes.byref(ms)), "bmg_autotune")
        t = self.tiles()
        if cache:
            table[key] = t
            tmp = cache + f".tmp{os.getpid()}"
            json.dump(table, open(tmp, "w"), indent=1)
            os.replace(tmp, cache)
        return t

    # ------------------------------------------------------------ profiling
    PROF_KINDS = {"smooth": 0, "residual": 1, "restrict": 2, "prolong": 3, "spmv": 4, "update": 5,
                  "vdown": 6, "vup": 7}

    def profile(self, enable: bool):
        _check(load().bmg_profile(self._h, int(enable)), "bmg_profile")

    def profile_read(self) -> dict:
        """{kind: (device ms, launches, algorithmic bytes)} of the finest level."""
        out = {}
        for name, k in self.PROF_KINDS.items():
            ms = ctypes.c_double()
            nl = ctypes.c_longlong()
            by = ctypes.c_double()
            _check(load().bmg_profile_read(self._h, k, ctypes.byref(ms), ctypes.byref(nl), ctypes.byref(by)),
                   "bmg_profile_read")
            if nl.value:
                out[name] = (ms.value, nl.value, by.value)
        return out

    # ------------------------------------------------------------ exports
    def stencil(self, level: int) -> torch.Tensor:
        n = self.level_n(level)
        out = torch.empty((n,) * self.dim + (3 ** self.dim,), dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            _check(load().bmg_get_stencil(self._h, level, _ptr(out)), "bmg_get_stencil")
        return out

    def interp(self, level: int) -> torch.Tensor:
        n = self.level_n(level)
        out = torch.empty((n,) * self.dim + (2 ** self.dim,), dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            _check(load().bmg_get_interp(self._h, level, _ptr(out)), "bmg_get_interp")
        return out


class AuxSolver:
    """The auxiliary-space two-grid method (bmg_aux_*): a P1 triangulation of
    the physical domain solved with `coarse` (a set-up 2-D Solver, assembled
    with bmg_assemble) as its structured coarse level.

    mesh: an object with xy (nv x 2), st (nv x 2, computational images),
    tri (ntri x 3), dirichlet (nv bools) and kappa (ntri) arrays, e.g.
    inputs.annulus_mesh.  mass_steps: CG iterations for M_p^-1 in P, or 0
    for the lumped mass.  krylov: flexible CG with one cycle as the
    preconditioner instead of the paper's stationary iteration."""

    def __init__(self, coarse: "Solver", mesh, omega: float = 2.0 / 3.0, mass_steps: int = 0, gamma: float = 1.0,
                 krylov: bool = False):
        import numpy as np
        lib = load()
        self.coarse = coarse
        self.nv = int(mesh.xy.shape[0])
        self.ntri = int(mesh.tri.shape[0])
        xy = np.ascontiguousarray(mesh.xy, dtype=np.float64)
        st = np.ascontiguousarray(mesh.st, dtype=np.float64)
        tri = np.ascontiguousarray(mesh.tri, dtype=np.int32)
        dirichlet = np.ascontiguousarray(mesh.dirichlet, dtype=np.uint8)
        opts = _AuxOpts(float(omega), int(mass_steps), float(gamma), 1 if krylov else 0)
        h = ctypes.c_void_p()
        _check(lib.bmg_aux_create(coarse._h, self.nv, xy.ctypes.data_as(ctypes.c_void_p),
                                  st.ctypes.data_as(ctypes.c_void_p), dirichlet.ctypes.data_as(ctypes.c_void_p),
                                  self.ntri, tri.ctypes.data_as(ctypes.c_void_p), ctypes.byref(opts),
                                  ctypes.byref(h)), "bmg_aux_create")
        self._h = h
        nbytes = ctypes.c_size_t()
        _check(lib.bmg_aux_workspace_bytes(h, ctypes.byref(nbytes)), "bmg_aux_workspace_bytes")
        self.workspace_bytes = nbytes.value
        dev = coarse.device
        with torch.cuda.device(dev):
            self._ws = torch.empty(max(self.workspace_bytes, 1), dtype=torch.uint8, device=dev)
            kappa = torch.as_tensor(mesh.kappa, dtype=torch.float64).to(dev).contiguous()
            _check(lib.bmg_aux_setup(h, ctypes.c_void_p(self._ws.data_ptr()), ctypes.c_size_t(self.workspace_bytes),
                                     _ptr(kappa), _ptr(coarse._coords)), "bmg_aux_setup")

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.bmg_aux_destroy(self._h)
            self._h = None

    def set_gamma(self, gamma: float):
        _check(load().bmg_aux_set_gamma(self._h, float(gamma)), "bmg_aux_set_gamma")

    def estimate_gamma(self, k: int = 12, y0=None, seed: int = 9, tol: float = 1e-10, apply: bool = False):
        """gamma = mean of the k Ritz values of generalized Lanczos on
        (P^T A_p P, A_c) (bmg_aux_estimate_gamma); y0 defaults to U[-1, 1]
        on the coarse grid (seeded).  Returns (gamma, alpha, beta)."""
        import numpy as np
        n = self.coarse.n
        if y0 is None:
            y0 = np.random.default_rng(seed).uniform(-1.0, 1.0, size=(n, n))
        y0 = torch.as_tensor(y0, dtype=torch.float64).to(self.coarse.device).contiguous()
        g = ctypes.c_double()
        alpha = np.zeros(k)
        beta = np.zeros(max(k - 1, 1))
        steps = ctypes.c_int()
        with torch.cuda.device(self.coarse.device):
            _check(load().bmg_aux_estimate_gamma(self._h, int(k), _ptr(y0), float(tol), ctypes.byref(g),
                                                 alpha.ctypes.data_as(ctypes.c_void_p),
                                                 beta.ctypes.data_as(ctypes.c_void_p), ctypes.byref(steps)),
                   "bmg_aux_estimate_gamma")
        if apply:
            self.set_gamma(g.value)
        m = steps.value
        return g.value, alpha[:m], beta[:max(m - 1, 0)]

    def solve(self, f, u0=None, tol: float = 1e-10, maxit: int = 500, raise_on_nonconv=True):
        dev = self.coarse.device
        f = torch.as_tensor(f, dtype=torch.float64).to(dev).contiguous()
        u = torch.zeros_like(f) if u0 is None else torch.as_tensor(u0, dtype=torch.float64).to(dev).clone()
        info = _Info()
        with torch.cuda.device(dev):
            code = load().bmg_aux_solve(self._h, _ptr(f), _ptr(u), float(tol), int(maxit), ctypes.byref(info))
        if code not in (0, 8) or (code == 8 and raise_on_nonconv):
            _check(code, "bmg_aux_solve")
        return u, _info_of(info)

    def export(self, which: str):
        """(rowptr, col, val) numpy arrays of 'A', 'M' or 'C' (see bmg_aux_export)."""
        import numpy as np
        w = {"A": 0, "M": 1, "C": 2}[which]
        lib = load()
        nr = ctypes.c_int()
        nnz = ctypes.c_longlong()
        _check(lib.bmg_aux_export(self._h, w, ctypes.byref(nr), ctypes.byref(nnz), None, None, None), "bmg_aux_export")
        rp = np.zeros(nr.value + 1, dtype=np.int64)
        col = np.zeros(nnz.value, dtype=np.int32)
        val = np.zeros(nnz.value, dtype=np.float64)
        _check(lib.bmg_aux_export(self._h, w, ctypes.byref(nr), ctypes.byref(nnz), rp.ctypes.data_as(ctypes.c_void_p),
                                  col.ctypes.data_as(ctypes.c_void_p), val.ctypes.data_as(ctypes.c_void_p)),
               "bmg_aux_export")
        return rp, col, val
