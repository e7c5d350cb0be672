"""Thin Python binding of librg.so (include/rg.h): argument marshalling only.

Every function here calls the C ABI of the same name; all arithmetic runs in the CUDA
kernels of librg.so. PyTorch provides device memory and the current CUDA stream. There
is no CPU fallback: if the library cannot be built or loaded, or no GPU is present, the
calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re

from . import build as _build

RG_OK, RG_EINVAL, RG_ENOMEM, RG_ECUDA, RG_ECAPACITY, RG_ENONFINITE, RG_ETIMEOUT = range(7)
RG_FP64, RG_MIXED = 0, 1
RG_TEST_REL, RG_TEST_PAPER = 0, 2
RG_ORTHONORMAL = 4  # the orthonormal variant (Section 2.2); implied by RG_MIXED
RG_ORTHOGONAL = 8  # the orthogonal variant (Section 2.2, alpha = 1); FP64 only

STATUS_NAMES = {0: "RG_OK", 1: "RG_EINVAL", 2: "RG_ENOMEM", 3: "RG_ECUDA", 4: "RG_ECAPACITY",
                5: "RG_ENONFINITE", 6: "RG_ETIMEOUT"}

HEADER = os.path.join(_build.ROOT, "include", "rg.h")

_lib = None


class RGError(RuntimeError):
    def __init__(self, code: int, func: str, msg: str):
        super().__init__(f"{func} -> {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def declared_functions():
    """Names of the functions include/rg.h declares."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:rg_status|const char\*)\s+(rg_\w+)\s*\(", txt, re.M)))


def lib(build: bool = True):
    """Load librg.so (building it first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    L = ctypes.CDLL(path)
    vp, i64, i32, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sig = {
        "rg_init": [vp, i64, f64, i32, i64, vp],
        "rg_add_rows": [vp, vp, vp, i64, vp],
        "rg_add_rows_host": [vp, vp, vp, i64, vp],
        "rg_solution": [vp, vp, vp],
        "rg_solution_host": [vp, vp, vp],
        "rg_rank": [vp, vp],
        "rg_rows_seen": [vp, vp],
        "rg_sync": [vp],
        "rg_reset": [vp],
        "rg_export": [vp, vp, vp, vp, vp, vp, i64, vp],
        "rg_set_stream": [vp, vp],
        "rg_free": [vp],
        "rg_batch_init": [vp, i64, vp, f64, i32, vp, vp],
        "rg_batch_add_rows": [vp, vp, vp, vp, vp, vp],
        "rg_batch_solution": [vp, vp, vp, vp],
        "rg_batch_sync": [vp],
        "rg_batch_reset": [vp],
        "rg_batch_free": [vp],
        "rg_solve_noalloc": [vp, vp, i64, i64, f64, i32, i64, vp, vp, vp],
        "rg_adjoint": [vp, vp, vp, i64, vp, vp, vp, vp],
        "rg_pinv": [vp, vp, i64, vp, i64],
        "rg_batch_adjoint": [vp, vp, vp, vp, vp, i64, vp, vp, vp, vp],
        "rg_batch_set_stream": [vp, vp],
        "rg_set_screen": [vp, f64],
        "rg_batch_set_screen": [vp, f64],
        "rg_batch_set_block_rows": [vp, i64, vp],
        "rg_batch_set_tc_group": [vp, i64, vp],
        "rg_snapshot_size": [vp, vp],
        "rg_snapshot": [vp, vp, i64],
        "rg_restore": [vp, vp, i64],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.rg_last_error.restype = ctypes.c_char_p
    L.rg_version.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(code: int, func: str):
    if code != RG_OK:
        raise RGError(code, func, lib().rg_last_error().decode())


def _ptr(t):
    """Device or host pointer of a tensor / numpy array (None -> NULL)."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return ctypes.c_void_p(t.data_ptr())
    return t.ctypes.data_as(ctypes.c_void_p)


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _need_cuda():
    import torch
    if not torch.cuda.is_available():
        raise RGError(RG_ECUDA, "rg", "no CUDA device: librg has no CPU fallback")


def solve_noalloc(Gamma, y, X, tol: float = 1e-10, mode: int = RG_FP64,
                  test: int = RG_TEST_REL, r_max: int = 0, stream=None, with_rank: bool = True):
    """rg_solve_noalloc: one stream from scratch with no allocation inside the library.
    Gamma (n, m), y (n,), X (m,) are contiguous float64 CUDA tensors on the current device.
    Returns the rank (synchronising) or None when with_rank is False (asynchronous; device
    errors of the call are then not reported). Arguments that do not match that contract
    raise RGError(RG_EINVAL) before anything is launched."""
    import torch

    def bad(msg):
        raise RGError(RG_EINVAL, "rg_solve_noalloc", msg)

    for name, t in (("Gamma", Gamma), ("y", y), ("X", X)):
        if not isinstance(t, torch.Tensor):
            bad(f"{name} is not a tensor")
        if t.dtype != torch.float64:
            bad(f"{name} has dtype {t.dtype}, float64 required")
        if not t.is_contiguous():
            bad(f"{name} is not contiguous")
    if Gamma.dim() != 2:
        bad(f"Gamma has {Gamma.dim()} dimensions, 2 required")
    n, m = int(Gamma.shape[0]), int(Gamma.shape[1])
    if y.numel() != n:
        bad(f"y has {y.numel()} elements, Gamma has {n} rows")
    if X.numel() < m:
        bad(f"X has {X.numel()} elements, fewer than m = {m}")
    _need_cuda()
    cur = torch.cuda.current_device()
    for name, t in (("Gamma", Gamma), ("y", y), ("X", X)):
        if t.device.type != "cuda" or t.device.index != cur:
            bad(f"{name} is on {t.device}, not on the current CUDA device {cur}")
    r = ctypes.c_int64(0)
    _check(lib().rg_solve_noalloc(_ptr(Gamma), _ptr(y), n, m, float(tol), int(mode) | int(test),
                                  int(r_max), _ptr(X), ctypes.byref(r) if with_rank else None,
                                  _stream(stream)), "rg_solve_noalloc")
    return int(r.value) if with_rank else None


class RankGreville:
    """One recursive least-squares stream (rg_init / rg_add_rows / rg_solution / rg_free)."""

    def __init__(self, m: int, tol: float = 1e-10, mode: int = RG_FP64,
                 test: int = RG_TEST_REL, r_max: int = 0, stream=None):
        _need_cuda()
        self.m = int(m)
        self.flags = int(mode) | int(test)
        self._h = ctypes.c_void_p()
        self._stream = stream
        _check(lib().rg_init(ctypes.byref(self._h), self.m, float(tol), self.flags, int(r_max),
                             _stream(stream)), "rg_init")

    def add_rows(self, Gamma, y, indep=None):
        """Gamma: (k, m) float64 CUDA tensor (contiguous); y: (k,); indep: (k,) uint8 or None."""
        k = 0 if Gamma.numel() == 0 else Gamma.shape[0]
        _check(lib().rg_add_rows(self._h, _ptr(Gamma), _ptr(y), k, _ptr(indep)), "rg_add_rows")

    def add_rows_host(self, Gamma, y, indep=None):
        """Same with host (numpy) buffers; copies happen inside the call."""
        k = Gamma.shape[0]
        _check(lib().rg_add_rows_host(self._h, _ptr(Gamma), _ptr(y), k, _ptr(indep)),
               "rg_add_rows_host")

    def solution(self, X, with_rank: bool = True):
        r = ctypes.c_int64(0)
        _check(lib().rg_solution(self._h, _ptr(X), ctypes.byref(r) if with_rank else None),
               "rg_solution")
        return int(r.value) if with_rank else None

    def adjoint(self, A, y, g, gA, gy, X=None):
        """rg_adjoint: dL/dA into gA and dL/dy into gy for dL/dX = g, given the rows A and
        targets y fed since init/reset (float64 CUDA tensors)."""
        _check(lib().rg_adjoint(self._h, _ptr(A), _ptr(y), int(A.shape[0]), _ptr(g), _ptr(gA),
                                _ptr(gy), _ptr(X)), "rg_adjoint")

    def pinv(self, A, Apinv):
        """rg_pinv: A^+ (m x n) of the rows A (n x m) fed since init/reset into Apinv, a
        float64 CUDA tensor of shape (m, ld >= n) (row stride ld)."""
        assert Apinv.dim() == 2 and Apinv.shape[0] == self.m and Apinv.stride(1) == 1
        _check(lib().rg_pinv(self._h, _ptr(A), int(A.shape[0]), _ptr(Apinv), int(Apinv.stride(0))),
               "rg_pinv")

    def set_screen(self, tau_lo: float):
        """rg_set_screen: floor of mixed mode's FP32 screen."""
        _check(lib().rg_set_screen(self._h, float(tau_lo)), "rg_set_screen")

    def solution_host(self, X):
        r = ctypes.c_int64(0)
        _check(lib().rg_solution_host(self._h, _ptr(X), ctypes.byref(r)), "rg_solution_host")
        return int(r.value)

    def rank(self) -> int:
        r = ctypes.c_int64(0)
        _check(lib().rg_rank(self._h, ctypes.byref(r)), "rg_rank")
        return int(r.value)

    def rows_seen(self) -> int:
        r = ctypes.c_int64(0)
        _check(lib().rg_rows_seen(self._h, ctypes.byref(r)), "rg_rows_seen")
        return int(r.value)

    def sync(self):
        _check(lib().rg_sync(self._h), "rg_sync")

    def reset(self):
        _check(lib().rg_reset(self._h), "rg_reset")

    def export(self, C=None, Ct=None, Pinv=None, w=None, basis_rows=None, capacity=None):
        cap = self.m if capacity is None else capacity
        r = ctypes.c_int64(0)
        _check(lib().rg_export(self._h, _ptr(C), _ptr(Ct), _ptr(Pinv), _ptr(w), _ptr(basis_rows),
                               int(cap), ctypes.byref(r)), "rg_export")
        return int(r.value)

    def snapshot_size(self) -> int:
        """rg_snapshot_size: bytes of one snapshot of this state."""
        out = ctypes.c_int64(0)
        _check(lib().rg_snapshot_size(self._h, ctypes.byref(out)), "rg_snapshot_size")
        return int(out.value)

    def new_snapshot_buffer(self, device=None):
        """A device buffer (uint8 CUDA tensor) that holds one snapshot."""
        import torch
        return torch.empty(self.snapshot_size(), dtype=torch.uint8,
                           device=device if device is not None else torch.cuda.current_device())

    def snapshot(self, buf):
        """rg_snapshot into buf (uint8 CUDA tensor of at least snapshot_size() bytes)."""
        _check(lib().rg_snapshot(self._h, _ptr(buf), int(buf.numel())), "rg_snapshot")

    def restore(self, buf):
        """rg_restore from a snapshot buffer."""
        _check(lib().rg_restore(self._h, _ptr(buf), int(buf.numel())), "rg_restore")

    def close(self):
        if self._h:
            lib().rg_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class RankGrevilleBatch:
    """B independent streams of uneven shape (rg_batch_*)."""

    def __init__(self, m_list, tol: float = 1e-10, mode: int = RG_FP64, test: int = RG_TEST_REL,
                 r_max_list=None, stream=None):
        import numpy as np
        _need_cuda()
        self.m = np.ascontiguousarray(m_list, dtype=np.int64)
        self.B = int(self.m.shape[0])
        rm = None if r_max_list is None else np.ascontiguousarray(r_max_list, dtype=np.int64)
        self._h = ctypes.c_void_p()
        _check(lib().rg_batch_init(ctypes.byref(self._h), self.B, _ptr(self.m), float(tol),
                                   int(mode) | int(test), _ptr(rm), _stream(stream)),
               "rg_batch_init")

    def add_rows(self, Gamma_packed, row_offsets, elem_offsets, y_packed, indep=None):
        _check(lib().rg_batch_add_rows(self._h, _ptr(Gamma_packed), _ptr(row_offsets),
                                       _ptr(elem_offsets), _ptr(y_packed), _ptr(indep)),
               "rg_batch_add_rows")

    def solution(self, X_packed, x_offsets=None, ranks=None):
        _check(lib().rg_batch_solution(self._h, _ptr(X_packed), _ptr(x_offsets), _ptr(ranks)),
               "rg_batch_solution")

    def adjoint(self, Gamma_packed, row_offsets, elem_offsets, y_packed, total_rows, g_packed,
                gA_packed, gy_packed, x_offsets=None):
        """rg_batch_adjoint: gradients of every instance (same packing as add_rows)."""
        _check(lib().rg_batch_adjoint(self._h, _ptr(Gamma_packed), _ptr(row_offsets),
                                      _ptr(elem_offsets), _ptr(y_packed), int(total_rows),
                                      _ptr(g_packed), _ptr(x_offsets), _ptr(gA_packed),
                                      _ptr(gy_packed)), "rg_batch_adjoint")

    def set_stream(self, stream=None):
        """Issue later calls on `stream` (default: torch's current stream), e.g. inside
        torch.cuda.graph capture."""
        _check(lib().rg_batch_set_stream(self._h, _stream(stream)), "rg_batch_set_stream")

    def set_screen(self, tau_lo: float):
        """rg_batch_set_screen: floor of mixed mode's FP32 screen."""
        _check(lib().rg_batch_set_screen(self._h, float(tau_lo)), "rg_batch_set_screen")

    def block_rows(self, rows: int = 0) -> int:
        """Set (rows > 0) and/or return the per-block row cap (rg_batch_set_block_rows)."""
        out = ctypes.c_int64(0)
        _check(lib().rg_batch_set_block_rows(self._h, int(rows), ctypes.byref(out)),
               "rg_batch_set_block_rows")
        return int(out.value)

    def tc_group(self, group: int = 0) -> int:
        """Set (group > 0) and/or return the second-product slices per tensor-core commit
        (rg_batch_set_tc_group)."""
        out = ctypes.c_int64(0)
        _check(lib().rg_batch_set_tc_group(self._h, int(group), ctypes.byref(out)),
               "rg_batch_set_tc_group")
        return int(out.value)

    def sync(self):
        _check(lib().rg_batch_sync(self._h), "rg_batch_sync")

    def reset(self):
        _check(lib().rg_batch_reset(self._h), "rg_batch_reset")

    def close(self):
        if self._h:
            lib().rg_batch_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
