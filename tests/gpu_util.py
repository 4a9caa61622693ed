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


U32 = 2.0 ** -24     # unit roundoff of float


def fp32_vcycle_bound(H, r, dim):
    """Bounds for an FP32 V-cycle of the library against the oracle.

    The oracle's FP32 arm evaluates the same V-cycle with float data and
    float arithmetic; its deviation from the FP64 arm, dev_arm (max-abs
    over max|z64|), is the size of single-precision rounding on this input.
    The library rounds the same operations in the same precision in another
    order (and forms the residual from the couplings to later colours, the
    same sum in exact arithmetic), so its deviation from either arm is of
    that size: the bound against the FP32 arm is 4 dev_arm (two deviations
    that may point opposite ways, their maxima at different nodes), and at
    least 4 u.  The a-priori bound against the FP64 arm is L gamma_{3^d+1}
    (a relative backward error of one sum plus a division per level, unit
    amplification over L levels).  Returns (z64, z32, bound_arm, bound_64),
    bounds relative to max|z64|."""
    z64 = H.vcycle(r)
    z32 = H.vcycle32(r)
    scale = np.abs(z64).max()
    dev_arm = np.abs(z32 - z64).max() / scale
    m = 3 ** dim + 1
    gamma = m * U32 / (1 - m * U32)
    return z64, z32, 4 * max(dev_arm, U32), H.nlev * gamma


def check_fp32_vcycle(z, H, r, dim, d_hier=0.0):
    """Element-wise check of a library FP32 V-cycle z (numpy) against both
    oracle arms; returns the two deviations for reporting.

    d_hier: where the library's FP64 hierarchy itself differs from the
    oracle's by more than FP64 rounding (the shell map's collapse amplifies
    rounding level by level), the max-abs deviation (over max|z64|) of the
    library's FP64 V-cycle from the oracle's.  The FP32 copies inherit that
    difference, and to first order the FP32 cycle responds to it as the FP64
    cycle does, so it enters both bounds twice (a factor two for the
    first-order approximation)."""
    z64, z32, b_arm, b_64 = fp32_vcycle_bound(H, r, dim)
    scale = np.abs(z64).max()
    d_arm = np.abs(z - z32).max() / scale
    d_64 = np.abs(z - z64).max() / scale
    assert d_arm <= b_arm + 2 * d_hier, (d_arm, b_arm, d_hier)
    assert d_64 <= b_64 + 2 * d_hier, (d_64, b_64, d_hier)
    return d_arm, d_64
