"""Host-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every function include/bmg.h declares; the host-only calls validate
their arguments.  No GPU needed (no call here touches the device)."""
import ctypes
import os
import re

import pytest
import torch

from paper_2509_08109_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(bmg_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "bmg_solve" in names and "bmg_adjoint_grad" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(binding.exported_symbols()) <= set(names)


def test_build_targets_sm103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


@pytest.mark.parametrize("n,dim,code", [(65, 2, 0), (4097, 2, 0), (64, 2, 2), (2, 2, 2), (3, 2, 0), (65, 4, 2), (17, 3, 0), (257, 3, 0), (16, 3, 2)])
def test_create_validates_shape(lib, n, dim, code):
    opts = binding._Opts(dim, n, 0, 0, 0)
    h = ctypes.c_void_p()
    rc = lib.bmg_create(ctypes.byref(opts), ctypes.byref(h))
    assert rc == code
    if rc == 0:
        nb = ctypes.c_size_t()
        assert lib.bmg_workspace_bytes(h, ctypes.byref(nb)) == 0
        assert nb.value > 0
        levels = lib.bmg_levels(h)
        sizes = [lib.bmg_level_n(h, l) for l in range(levels)]
        assert sizes[0] == n and sizes[-1] == 3
        assert all(2 * sizes[l + 1] - 1 == sizes[l] for l in range(levels - 1))
        lib.bmg_destroy(h)
    else:
        assert not h.value


def test_workspace_fp32_larger_than_fp64(lib):
    sizes = {}
    for prec in (0, 1):
        opts = binding._Opts(2, 1025, prec, 0, 0)
        h = ctypes.c_void_p()
        assert lib.bmg_create(ctypes.byref(opts), ctypes.byref(h)) == 0
        nb = ctypes.c_size_t()
        lib.bmg_workspace_bytes(h, ctypes.byref(nb))
        sizes[prec] = nb.value
        lib.bmg_destroy(h)
    assert sizes[1] > sizes[0]


def test_calls_before_attach_are_rejected(lib):
    opts = binding._Opts(2, 17, 0, 0, 0, 1)
    h = ctypes.c_void_p()
    assert lib.bmg_create(ctypes.byref(opts), ctypes.byref(h)) == 0
    assert lib.bmg_setup(h) == 4            # no workspace
    assert lib.bmg_solve(h, 1, None, None, ctypes.c_double(1e-10), 10, None) == 4
    assert lib.bmg_create(None, ctypes.byref(h)) == 1
    assert lib.bmg_status_str(6).decode().startswith("setup breakdown")
    lib.bmg_destroy(h)


@pytest.mark.parametrize("dim,n,code", [(2, 641, 2), (3, 49, 2), (4, 9, 2), (2, 2, 2), (2, 640, 1), (3, 48, 1),
                                        (3, 1 << 22, 2), (2, 1 << 22, 2), (2, 2 ** 31 - 1, 2),
                                        (3, 2 ** 31 - 1, 2), (2, -5, 2)])
def test_noalloc_validates_before_device_work(lib, dim, n, code):
    """Shape and null-pointer checks of bmg_assemble_noalloc come before any
    CUDA call, so they answer without a device; n is bounded before any size
    arithmetic, so huge n cannot wrap into an accepted size."""
    assert lib.bmg_assemble_noalloc(dim, n, None, None, None, None) == code


@pytest.mark.parametrize("which", ["coords", "kappa", "out"])
def test_noalloc_binding_rejects_wrong_sizes_on_the_host(which):
    """The C entry point takes no lengths, so the binding checks every
    buffer's size before the call (an undersized output would otherwise be
    written past its end on the device)."""
    n = 17
    sizes = {"coords": 2 * n * n, "kappa": (n - 1) ** 2, "out": n * n * 9}
    sizes[which] -= 1
    t = {k: torch.zeros(v, dtype=torch.float64) for k, v in sizes.items()}
    with pytest.raises(ValueError, match=which):
        binding.assemble_noalloc(2, n, t["coords"], t["kappa"], t["out"])


def test_noalloc_binding_rejects_host_tensors():
    n = 17
    t = [torch.zeros(k, dtype=torch.float64) for k in (2 * n * n, (n - 1) ** 2, n * n * 9)]
    with pytest.raises(ValueError, match="current CUDA device"):
        binding.assemble_noalloc(2, n, *t)


def test_aux_defaults_and_null_arguments(lib):
    """The auxiliary-space calls validate their arguments before any device
    work: defaults of the options, null pointers, no coarse context."""
    o = binding._AuxOpts()
    lib.bmg_aux_default_opts(ctypes.byref(o))
    assert abs(o.omega - 2.0 / 3.0) < 1e-15 and o.mass_steps == 0 and o.gamma == 1.0 and o.krylov == 0
    h = ctypes.c_void_p()
    assert lib.bmg_aux_create(None, 3, None, None, None, 1, None, None, ctypes.byref(h)) == 1
    assert h.value is None
    nb = ctypes.c_size_t()
    assert lib.bmg_aux_workspace_bytes(None, ctypes.byref(nb)) == 1
    assert lib.bmg_aux_solve(None, None, None, 1e-10, 10, None) == 1
    g = ctypes.c_double()
    assert lib.bmg_aux_estimate_gamma(None, 12, None, 1e-10, ctypes.byref(g), None, None, None) == 1


def test_max_rhs_reserves_workspace_only_where_eligible(lib):
    """max_rhs > 1 adds room for solving right-hand sides together on a 2-D
    FP32 refinement-mode context with n >= 65, and nothing elsewhere; values
    outside 0..4 are refused."""
    def ws(dim, n, prec, outer, max_rhs):
        opts = binding._Opts(dim, n, prec, outer, 0, max_rhs)
        h = ctypes.c_void_p()
        assert lib.bmg_create(ctypes.byref(opts), ctypes.byref(h)) == 0
        nb = ctypes.c_size_t()
        assert lib.bmg_workspace_bytes(h, ctypes.byref(nb)) == 0
        lib.bmg_destroy(h)
        return nb.value
    assert ws(2, 129, 1, 2, 4) > ws(2, 129, 1, 2, 1)
    assert ws(2, 129, 1, 2, 1) == ws(2, 129, 1, 2, 0)
    assert ws(2, 129, 0, 0, 4) == ws(2, 129, 0, 0, 1)       # FP64: right-hand sides in turn
    assert ws(3, 33, 1, 2, 4) == ws(3, 33, 1, 2, 1)         # 3-D
    assert ws(2, 33, 1, 2, 4) == ws(2, 33, 1, 2, 1)         # below the streamed sizes
    for bad in (-1, 5):
        opts = binding._Opts(2, 129, 1, 2, 0, bad)
        h = ctypes.c_void_p()
        assert lib.bmg_create(ctypes.byref(opts), ctypes.byref(h)) == 1


def _ws_bytes(lib, dim, n, prec, outer, flags):
    opts = binding._Opts(dim, n, binding.PREC[prec], binding.OUTER[outer], flags, 1)
    h = ctypes.c_void_p()
    assert lib.bmg_create(ctypes.byref(opts), ctypes.byref(h)) == 0
    nb = ctypes.c_size_t()
    assert lib.bmg_workspace_bytes(h, ctypes.byref(nb)) == 0
    sizes = [lib.bmg_level_n(h, l) for l in range(lib.bmg_levels(h))]
    lib.bmg_destroy(h)
    return nb.value, sizes


@pytest.mark.parametrize("n", [17, 33, 65, 257])
def test_colour_blocked_rows_only_for_the_per_colour_3d_path(lib, n):
    """The FP32 3-D half sweeps read the symmetric planes; the full 27-entry
    rows grouped by colour (27 (n_l - 2)^3 floats per level but the coarsest,
    each block 256-byte aligned in the workspace) exist only for the
    per-colour smoother that BMG_FLAG_UNFUSED selects.  FP64 and 2-D
    workspaces do not depend on the flag."""
    fused, sizes = _ws_bytes(lib, 3, n, "fp32", "refine", 0)
    unfused, _ = _ws_bytes(lib, 3, n, "fp32", "refine", 1)
    blocks = sum(-(-27 * (m - 2) ** 3 * 4 // 256) * 256 for m in sizes[:-1])
    assert unfused - fused == blocks
    assert _ws_bytes(lib, 3, n, "fp64", "cg", 0)[0] == _ws_bytes(lib, 3, n, "fp64", "cg", 1)[0]
    assert _ws_bytes(lib, 2, 4 * n - 3, "fp32", "refine", 0)[0] == _ws_bytes(lib, 2, 4 * n - 3, "fp32", "refine", 1)[0]
