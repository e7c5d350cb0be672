"""ctypes wrapper of the plain-C FP64 oracle ``rg_oracle.c`` (TEST INFRASTRUCTURE).

``build()`` compiles the C file with gcc into ``oracle/_build/librgo.so``; nothing here
touches a GPU. Only tests, the smoke check and the benchmark's CPU-baseline leg use it.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rg_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "librgo.so")

TEST_REL = 0
TEST_PAPER = 2

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile rg_oracle.c (plain -O2, OpenMP only across batched instances). Floating-point
    contraction is off: every product and sum rounds on its own, as the paper's NumPy
    implementation does, so the oracle gives bit-identical results on x86 and Arm hosts
    (GCC fuses a * b + c into one FMA by default on aarch64, not on x86-64 at -O2)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(SRC),
                                                                       os.path.getmtime(__file__)):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=c99", SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB)
            i64, f64p, i64p, u8p = ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p
            L.rgo_solve_mut.argtypes = [i64, i64, f64p, f64p, ctypes.c_double, ctypes.c_int, i64,
                                        ctypes.c_int, f64p, i64p, i64p, u8p, f64p, f64p, f64p,
                                        i64p]
            L.rgo_solve_mut.restype = ctypes.c_int
            L.rgo_solve_var.argtypes = [i64, i64, f64p, f64p, ctypes.c_double, ctypes.c_int, i64,
                                        ctypes.c_int, ctypes.c_int, f64p, i64p, i64p, u8p, f64p,
                                        f64p, f64p, i64p]
            L.rgo_solve_var.restype = ctypes.c_int
            L.rgo_solve_batch.argtypes = [i64, i64p, i64p, i64p, f64p, f64p, ctypes.c_double,
                                          ctypes.c_int, ctypes.c_int, f64p, i64p, ctypes.c_void_p]
            L.rgo_solve_batch.restype = ctypes.c_int
            L.rgo_solve_batch_var.argtypes = [i64, i64p, i64p, i64p, f64p, f64p, ctypes.c_double,
                                              ctypes.c_int, ctypes.c_int, ctypes.c_int, f64p,
                                              i64p, ctypes.c_void_p, u8p]
            L.rgo_solve_batch_var.restype = ctypes.c_int
            L.rgo_pinv_mut.argtypes = [i64, i64, f64p, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                       f64p, i64p, u8p]
            L.rgo_pinv_mut.restype = ctypes.c_int
            L.rgo_max_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclasses.dataclass
class Result:
    X: np.ndarray  # m
    rank: int
    basis_rows: np.ndarray  # rank, int64: input-row index of each basis row (C's rows)
    indep: np.ndarray  # n, uint8: 1 where the row grew the rank
    Ct: np.ndarray  # rank x m dual basis
    Pinv: np.ndarray  # rank x rank
    C: np.ndarray  # rank x m basis (the selected rows)
    rows_done: int
    status: int


GENERAL, ORTHONORMAL, ORTHOGONAL = 0, 1, 2


def solve(A, Y, tol: float = 1e-10, test_mode: int = TEST_REL, r_max: int = 0,
          mutation: int = 0, variant: int = GENERAL) -> Result:
    """Run Algorithm 1 over all rows of A (n x m) with targets Y, from an empty state.
    variant=ORTHONORMAL takes Section 2.2's orthonormal rank factorization (C = Ct = Q);
    variant=ORTHOGONAL its orthogonal one (alpha = 1: C holds the raw rejections, Ct the
    same rows divided by their squared norms)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64).reshape(-1)
    n, m = A.shape
    assert Y.shape[0] == n
    rm = m if r_max <= 0 else min(r_max, m)
    X = np.zeros(m)
    rank = np.zeros(1, dtype=np.int64)
    basis = np.zeros(rm, dtype=np.int64)
    indep = np.zeros(max(n, 1), dtype=np.uint8)
    Ct = np.zeros(rm * m)
    C = np.zeros(rm * m)
    Pinv = np.zeros(rm * rm)
    done = np.zeros(1, dtype=np.int64)
    st = lib().rgo_solve_var(n, m, _ptr(A), _ptr(Y), float(tol), int(test_mode), int(r_max),
                             int(variant), int(mutation), _ptr(X), _ptr(rank), _ptr(basis),
                             _ptr(indep), _ptr(Ct), _ptr(Pinv), _ptr(C), _ptr(done))
    if st not in (0, 4):
        raise RuntimeError(f"rgo_solve failed with status {st}")
    r = int(rank[0])
    return Result(X=X, rank=r, basis_rows=basis[:r].copy(), indep=indep[:n].copy(),
                  Ct=Ct[:r * m].reshape(r, m).copy(), Pinv=Pinv[:r * r].reshape(r, r).copy(),
                  C=C[:r * m].reshape(r, m).copy(), rows_done=int(done[0]), status=st)


def pinv(A, tol: float = 1e-10, test_mode: int = TEST_REL, mutation: int = 0):
    """Pseudoinverse update of Theorems label_th_pinv_indep / label_th_pinv_lindep over the
    rows of A (n x m): returns (A^+ as an m x n array, rank, per-row independence flags)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    n, m = A.shape
    Ap = np.zeros(m * max(n, 1))
    rank = np.zeros(1, dtype=np.int64)
    indep = np.zeros(max(n, 1), dtype=np.uint8)
    st = lib().rgo_pinv_mut(n, m, _ptr(A), float(tol), int(test_mode), int(mutation), _ptr(Ap),
                            _ptr(rank), _ptr(indep))
    if st != 0:
        raise RuntimeError(f"rgo_pinv failed with status {st}")
    return Ap[:m * n].reshape(m, n).copy(), int(rank[0]), indep[:n].copy()


def solve_batch(A_packed, Y_packed, row_off, elem_off, x_off, tol: float = 1e-10,
                test_mode: int = TEST_REL, threads: int = 0, variant: int = GENERAL,
                with_indep: bool = False):
    """Batched oracle (OpenMP over instances). Returns (X_packed, ranks), or
    (X_packed, ranks, indep_packed) with with_indep (per-row flags packed by row_off; rows
    after a capacity stop hold 0xFF). A capacity stop (status 4) is allowed; other failures
    raise."""
    A = np.ascontiguousarray(A_packed, dtype=np.float64)
    Y = np.ascontiguousarray(Y_packed, dtype=np.float64)
    ro = np.ascontiguousarray(row_off, dtype=np.int64)
    eo = np.ascontiguousarray(elem_off, dtype=np.int64)
    xo = np.ascontiguousarray(x_off, dtype=np.int64)
    B = ro.shape[0] - 1
    X = np.zeros(max(int(xo[-1]), 1))
    ranks = np.zeros(max(B, 1), dtype=np.int64)
    status = np.zeros(max(B, 1), dtype=np.int32)
    indep = np.zeros(max(int(ro[-1]), 1), dtype=np.uint8) if with_indep else None
    lib().rgo_solve_batch_var(B, _ptr(ro), _ptr(eo), _ptr(xo), _ptr(A), _ptr(Y), float(tol),
                              int(test_mode), int(variant), int(threads), _ptr(X), _ptr(ranks),
                              _ptr(status), _ptr(indep))
    if B and not np.isin(status[:B], (0, 4)).all():
        raise RuntimeError(f"rgo_solve_batch failed: statuses {np.unique(status[:B])}")
    X, ranks = X[:int(xo[-1])], ranks[:B]
    if with_indep:
        return X, ranks, indep[:int(ro[-1])]
    return X, ranks


def max_threads() -> int:
    return int(lib().rgo_max_threads())
