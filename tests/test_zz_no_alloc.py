"""bmg_assemble_noalloc: the allocation-free assembly entry point, called
through the C ABI twice in a row and compared with bmg_assemble +
bmg_get_stencil(0) (2-D, 3-D), with the oracle at the largest accepted size,
and on its errors.  The file name makes pytest collect it last, so it runs
both after every other test and, alone, in a fresh process."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_08109_gb300 import binding, inputs
from tests.gpu_util import rel_to_diag

pytestmark = pytest.mark.gpu

TOL = 1e-13   # relative to the row's diagonal, as the assembly parity tests


def _noalloc(p, out):
    coords = torch.as_tensor(p.coords, device="cuda").contiguous()
    kappa = torch.as_tensor(p.kappa, device="cuda").contiguous()
    binding.assemble_noalloc(p.dim, p.n, coords, kappa, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("dim,n", [(2, 129), (3, 33)])
def test_twice_in_a_row_matches_existing_entry_point(dim, n):
    p = inputs.annulus_lognormal(n) if dim == 2 else inputs.shell_two_layer(n)
    s = binding.Solver(dim, n).assemble(torch.as_tensor(p.coords), torch.as_tensor(p.kappa))
    ref = s.stencil(0).cpu().numpy()
    shape = (n,) * dim + (3 ** dim,)
    out1 = torch.full(shape, np.nan, dtype=torch.float64, device="cuda")
    out2 = torch.full(shape, np.nan, dtype=torch.float64, device="cuda")
    a1 = _noalloc(p, out1)
    a2 = _noalloc(p, out2)
    assert np.isfinite(a1).all() and np.isfinite(a2).all()
    assert rel_to_diag(a1, ref) <= TOL
    assert rel_to_diag(a2, ref) <= TOL


def test_largest_accepted_size_matches_oracle():
    """Against the oracle the bound grows with n: the Jacobian is formed from
    coordinate differences of size 1/(n-1), whose relative rounding is about
    (n-1) eps, so the entries agree to a few n eps of the diagonal."""
    n = 640    # not 2^k+1: the entry point needs no hierarchy
    p = inputs.annulus_plain(n)
    out = torch.empty((n, n, 9), dtype=torch.float64, device="cuda")
    got = _noalloc(p, out)
    assert rel_to_diag(got, oracle.assemble(p.coords, p.kappa)) <= 4 * n * np.finfo(float).eps


@pytest.mark.parametrize("dim,n", [(2, 641), (3, 49)])
def test_beyond_the_static_array_is_rejected(dim, n):
    """Correctly sized buffers, one node per side beyond what the static
    array holds: the library refuses the size itself."""
    coords = torch.zeros(dim * n ** dim, dtype=torch.float64, device="cuda")
    kappa = torch.ones((n - 1) ** dim, dtype=torch.float64, device="cuda")
    out = torch.zeros(n ** dim * 3 ** dim, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.BmgError) as e:
        binding.assemble_noalloc(dim, n, coords, kappa, out)
    assert e.value.code == 2
    assert "static scratch" in str(e.value)


def test_warm_call_allocates_no_device_memory():
    """After a first call (which may load the library's module and with it
    the static array), further calls change neither the device's free
    memory nor torch's allocator state."""
    n = 257
    p = inputs.annulus_lognormal(n)
    coords = torch.as_tensor(p.coords, device="cuda").contiguous()
    kappa = torch.as_tensor(p.kappa, device="cuda").contiguous()
    out = torch.empty((n, n, 9), dtype=torch.float64, device="cuda")
    binding.assemble_noalloc(2, n, coords, kappa, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(3):
        binding.assemble_noalloc(2, n, coords, kappa, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0 and torch.cuda.memory_reserved() == reserved0


def test_folded_map_then_valid_map():
    """The error word is cleared at the start of every call."""
    n = 9
    p = inputs.annulus_plain(n)
    bad = p.coords.copy()
    bad[0, 4, 4] += 0.6
    out = torch.empty((n, n, 9), dtype=torch.float64, device="cuda")
    kappa = torch.as_tensor(p.kappa, device="cuda")
    with pytest.raises(binding.BmgError) as e:
        binding.assemble_noalloc(2, n, torch.as_tensor(bad, device="cuda"), kappa, out)
    assert e.value.code == 5
    got = _noalloc(p, out)
    assert rel_to_diag(got, oracle.assemble(p.coords, p.kappa)) <= TOL
