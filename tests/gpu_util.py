"""Helpers shared by the GPU parity tests (no solver arithmetic here)."""
import numpy as np
import torch

import oracle
from paper_2509_08109_gb300 import binding


def solver_for(problem, precision="fp64", outer=None, unfused=False):
    s = binding.Solver(problem.dim, problem.n, precision=precision, outer=outer, unfused=unfused)
    s.assemble(torch.as_tensor(problem.coords), torch.as_tensor(problem.kappa))
    s.setup()
    return s


def rel_to_diag(gpu: np.ndarray, ref: np.ndarray) -> float:
    """max |gpu - ref| per row scaled by that row's diagonal (the centre slot)."""
    ctr = (ref.shape[-1] - 1) // 2
    d = np.abs(ref[..., ctr])[..., None]
    d = np.where(d > 0, d, 1.0)
    return float(np.max(np.abs(gpu - ref) / d))


def relerr(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    den = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (den if den > 0 else 1.0))
