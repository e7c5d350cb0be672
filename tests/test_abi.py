"""The C ABI library builds for sm_103a, loads, and exports every symbol that
include/rg.h declares (no GPU needed: nothing here calls into the device)."""
import ctypes
import os
import re
import subprocess

from paper_2106_11594_gb300 import build, rg


def test_header_declares_the_boundary():
    names = rg.declared_functions()
    for fn in ["rg_init", "rg_add_rows", "rg_solution", "rg_free", "rg_batch_init",
               "rg_batch_add_rows", "rg_batch_solution", "rg_batch_free", "rg_last_error"]:
        assert fn in names


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    L = ctypes.CDLL(path)
    for name in rg.declared_functions():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (rg_\w+)$", out, re.M))
    assert set(rg.declared_functions()) <= exported


def test_library_is_built_for_sm_103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_version_string_without_gpu():
    L = rg.lib()
    assert b"sm_103a" in L.rg_version()
    assert L.rg_last_error() == b""


def test_noalloc_binding_rejects_bad_arguments_before_any_launch():
    """rg_solve_noalloc takes raw pointers, so the binding checks dtype, shape and
    contiguity first: a float32 or short X would otherwise be written past its end."""
    import pytest
    import torch
    G = torch.zeros((4, 8), dtype=torch.float64)
    y = torch.zeros(4, dtype=torch.float64)
    X = torch.zeros(8, dtype=torch.float64)
    bad_cases = [
        (G.float(), y, X),                              # Gamma float32
        (G, y, X.float()),                              # X float32
        (G, y, torch.zeros(7, dtype=torch.float64)),    # X shorter than m
        (G, torch.zeros(3, dtype=torch.float64), X),    # y length != n
        (G.reshape(-1), y, X),                          # Gamma not 2-D
        (torch.zeros((8, 4), dtype=torch.float64).t(), y, X),  # Gamma not contiguous
    ]
    for g_, y_, x_ in bad_cases:
        with pytest.raises(rg.RGError) as ei:
            rg.solve_noalloc(g_, y_, x_)
        assert ei.value.code == rg.RG_EINVAL


def test_flag_validation_without_gpu():
    """rg_init checks its flags before touching the device: the orthogonal variant is
    FP64-only and excludes the orthonormal one."""
    import ctypes as ct
    L = rg.lib()
    h = ct.c_void_p()
    for flags in (rg.RG_ORTHOGONAL | rg.RG_MIXED, rg.RG_ORTHOGONAL | rg.RG_ORTHONORMAL, 64):
        assert L.rg_init(ct.byref(h), 16, 1e-10, flags, 0, None) == rg.RG_EINVAL
        assert not h.value


def test_batch_knobs_reject_a_null_handle_without_gpu():
    import ctypes as ct
    L = rg.lib()
    out = ct.c_int64(-1)
    assert L.rg_batch_set_tc_group(None, 4, ct.byref(out)) == rg.RG_EINVAL
    assert L.rg_batch_set_block_rows(None, 64, ct.byref(out)) == rg.RG_EINVAL
    assert out.value == -1
