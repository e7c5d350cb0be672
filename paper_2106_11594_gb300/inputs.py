"""Seeded synthetic workloads for the rank-Greville recursive least-squares update.

This module only draws random numbers and forms the observation matrices; it holds
none of the method's arithmetic (no projection, rejection, rank test or update).
Both the CPU oracle tests and the CUDA path take their inputs from here, so the two
implementations see bit-identical rows.

Workloads follow the paper's synthetic construction R_N(n, m, r): a product of
N(0, 1) matrices, which has rank r (Section 4.1, Eq. label_eq_tests_speed), with a
measured target Y = A x_true + noise (Eq. label_eq_linear_relation).

Seeding: every matrix is drawn from numpy's PCG64 seeded by
``SeedSequence(2106_11594, spawn_key=(workload_id, instance))`` so that instance b of
a batched workload is reproducible on its own, independently of the others.

Readings (the paper leaves these open):
  * noise "N(0, 1e-3)" means standard deviation 1e-3;
  * workload 5 (ill-conditioned rank growth) is built as U diag(s) V with the active
    row-space dimension growing in 8 phases, and 5% of rows replaced by random
    combinations of 2-3 earlier rows (see ``ill_conditioned_stream``).
"""
from __future__ import annotations

import dataclasses

from typing import Optional

import numpy as np

BASE_SEED = 2106_11594


def rng_for(workload_id: int, instance: int = 0) -> np.random.Generator:
    """PCG64 generator for (workload, instance)."""
    ss = np.random.SeedSequence(BASE_SEED, spawn_key=(int(workload_id), int(instance)))
    return np.random.Generator(np.random.PCG64(ss))


@dataclasses.dataclass
class Stream:
    """One least-squares stream: rows of A arrive in order with targets Y."""

    A: np.ndarray  # n x m, float64, C-contiguous
    Y: np.ndarray  # n, float64
    rank: int  # rank of the generator (the exact rank of the factor product)
    name: str = ""
    growth: Optional[np.ndarray] = None  # n, uint8: 1 where the generator's prefix rank grows

    @property
    def n(self) -> int:
        return self.A.shape[0]

    @property
    def m(self) -> int:
        return self.A.shape[1]


def factor_stream(n: int, m: int, r: int, noise: float, rng: np.random.Generator,
                  name: str = "") -> Stream:
    """A = G1 G2 with G1 (n x r), G2 (r x m) i.i.d. N(0, 1); Y = A x_true + noise."""
    G1 = rng.standard_normal((n, r))
    G2 = rng.standard_normal((r, m))
    x_true = rng.standard_normal(m)
    eps = rng.standard_normal(n) * noise
    A = np.ascontiguousarray(G1 @ G2)
    Y = A @ x_true + eps
    return Stream(A=A, Y=np.ascontiguousarray(Y), rank=min(r, n, m), name=name)


def factor_stream_factors(n: int, m: int, r: int, noise: float, rng: np.random.Generator):
    """The raw draws behind ``factor_stream`` (G1, G2, x_true, noise vector), in the same
    order, for callers that need the factors themselves (for example an exact-rational
    product)."""
    G1 = rng.standard_normal((n, r))
    G2 = rng.standard_normal((r, m))
    x_true = rng.standard_normal(m)
    eps = rng.standard_normal(n) * noise
    return G1, G2, x_true, eps


# ---------------------------------------------------------------------------
# The five workloads
# ---------------------------------------------------------------------------

def small_stream(n: int = 256, m: int = 64, r: int = 8) -> Stream:
    """Workload 1: single plain FP64 stream, n=256, m=64, r=8, noise 1e-3."""
    return factor_stream(n, m, r, 1e-3, rng_for(1), name=f"stream n={n} m={m} r={r}")


def large_stream(n: int = 65536, m: int = 1024, r: int = 64) -> Stream:
    """Workload 2: single large stream, n=65536, m=1024, r=64, noise 1e-3.

    With G1 Gaussian its leading r x r block is nonsingular with probability one, so
    the first r rows each grow the rank by one and every later row is dependent.
    Smaller (n, m, r) keep the construction for parity tests.
    """
    return factor_stream(n, m, r, 1e-3, rng_for(2), name=f"stream n={n} m={m} r={r}")


@dataclasses.dataclass
class Batch:
    """Ragged batch of independent streams, packed back to back."""

    streams: list
    name: str = ""

    @property
    def B(self) -> int:
        return len(self.streams)

    def shapes(self):
        return [(s.n, s.m) for s in self.streams]

    def packed(self):
        """(A_packed, Y_packed, row_offsets, elem_offsets, x_offsets).

        Instance b's rows are A_packed[elem_offsets[b]:elem_offsets[b+1]] viewed as
        (n_b, m_b) row-major; its targets are Y_packed[row_offsets[b]:row_offsets[b+1]];
        its solution occupies X[x_offsets[b]:x_offsets[b+1]] (length m_b).
        """
        n = np.array([s.n for s in self.streams], dtype=np.int64)
        m = np.array([s.m for s in self.streams], dtype=np.int64)
        row_off = np.zeros(self.B + 1, dtype=np.int64)
        row_off[1:] = np.cumsum(n)
        elem_off = np.zeros(self.B + 1, dtype=np.int64)
        elem_off[1:] = np.cumsum(n * m)
        x_off = np.zeros(self.B + 1, dtype=np.int64)
        x_off[1:] = np.cumsum(m)
        A = np.empty(int(elem_off[-1]), dtype=np.float64)
        Y = np.empty(int(row_off[-1]), dtype=np.float64)
        for b, s in enumerate(self.streams):
            A[elem_off[b]:elem_off[b + 1]] = s.A.reshape(-1)
            Y[row_off[b]:row_off[b + 1]] = s.Y
        return A, Y, row_off, elem_off, x_off


def uneven_batch_shapes(B: int = 4096, m_lo: int = 32, m_hi: int = 512):
    """Workload 3 shapes: m ~ U{m_lo..m_hi}, r ~ U{2..floor(m/4)}, n ~ U{m..8m}."""
    rng = rng_for(3, 1 << 30)
    m = rng.integers(m_lo, m_hi + 1, size=B)
    r = np.array([rng.integers(2, max(2, mi // 4) + 1) for mi in m])
    n = np.array([rng.integers(mi, 8 * mi + 1) for mi in m])
    return n.astype(np.int64), m.astype(np.int64), r.astype(np.int64)


def uneven_batch(B: int = 4096, m_lo: int = 32, m_hi: int = 512, instances=None) -> Batch:
    """Workload 3: B independent streams of uneven (n, m, r), Gaussian factors, noise 1e-4.

    ``instances`` selects a subset of instance ids (shapes and draws are those of the
    full batch, so a subset is a faithful sample of it)."""
    n, m, r = uneven_batch_shapes(B, m_lo, m_hi)
    ids = range(B) if instances is None else instances
    streams = [factor_stream(int(n[b]), int(m[b]), int(r[b]), 1e-4, rng_for(3, b),
                             name=f"inst {b}") for b in ids]
    return Batch(streams=streams, name=f"uneven batch B={B}")


def uniform_batch(B: int = 1024, n: int = 2048, m: int = 256, r: int = 32,
                  instances=None) -> Batch:
    """Workload 4: B streams with n=2048, m=256, r=32, Gaussian factors, noise 1e-3."""
    ids = range(B) if instances is None else instances
    streams = [factor_stream(n, m, r, 1e-3, rng_for(4, b), name=f"inst {b}") for b in ids]
    return Batch(streams=streams, name=f"uniform batch B={B} n={n} m={m} r={r}")


def loss_targets(batch: Batch) -> list:
    """x_target ~ N(0, 1)^m per instance, for the loss L = ||X - x_target||^2."""
    return [rng_for(4, 1 << 20 | b).standard_normal(s.m) for b, s in enumerate(batch.streams)]


def ill_conditioned_stream(n: int = 32768, m: int = 2048, r: int = 256, phases: int = 8,
                           combo_frac: float = 0.05, s_lo: float = 1e-6) -> Stream:
    """Workload 5: rank-growth stress with a wide singular-value spread.

    V: r x m with orthonormal rows; U: n x r with orthonormal columns; s: r scales
    log-uniform on [s_lo, 1] in random order. Phase p (of ``phases``) covers rows
    [p n/phases, (p+1) n/phases) and activates the first (p+1) r/phases directions:
    row i = (u_i masked to the active directions) diag(s) V. A further ``combo_frac``
    of the rows (never the first row of a phase) are replaced by c_1 Gamma_a + c_2
    Gamma_b (+ c_3 Gamma_c) of 2-3 earlier rows with c ~ N(0, 1).
    """
    rng = rng_for(5)
    V = np.linalg.qr(rng.standard_normal((m, r)))[0].T.copy()  # r x m, orthonormal rows
    U = np.linalg.qr(rng.standard_normal((n, r)))[0]  # n x r, orthonormal columns
    s = np.exp(rng.uniform(np.log(s_lo), 0.0, size=r))
    s = s[rng.permutation(r)]
    per = n // phases
    step = r // phases
    active = np.minimum((np.arange(n) // per + 1) * step, r)
    mask = np.arange(r)[None, :] < active[:, None]
    A = ((U * mask) * s[None, :]) @ V
    n_combo = int(round(combo_frac * n))
    phase_starts = set(range(0, n, per))
    cand = np.array([i for i in range(3, n) if i not in phase_starts])
    pos = np.sort(rng.choice(cand, size=n_combo, replace=False))
    for i in pos:
        k = int(rng.integers(2, 4))
        src = rng.choice(i, size=k, replace=False)
        c = rng.standard_normal(k)
        A[i] = c @ A[src]
    x_true = rng.standard_normal(m)
    Y = A @ x_true + rng.standard_normal(n) * 1e-3
    # The prefix rank grows on the first `step` rows of each phase that are not
    # combinations (generically: those rows' new coordinates form a nonsingular block).
    growth = np.zeros(n, dtype=np.uint8)
    combo = np.zeros(n, dtype=bool)
    combo[pos] = True
    for p0 in range(0, n, per):
        fresh = [i for i in range(p0, min(n, p0 + per)) if not combo[i]]
        growth[fresh[:step]] = 1
    return Stream(A=np.ascontiguousarray(A), Y=Y, rank=r,
                  name=f"ill-conditioned stream n={n} m={m} r={r}", growth=growth)


# ---------------------------------------------------------------------------
# Small exactly-representable inputs (for the exact-rational pins)
# ---------------------------------------------------------------------------

def integer_lowrank(n: int, m: int, r: int, seed: int, lo: int = -3, hi: int = 3):
    """A = G1 G2 with small-integer factors, so A is exact in FP64 and has exact rank
    <= r; Y small integers. Returns (A, Y) as float64 arrays."""
    rng = rng_for(100, seed)
    G1 = rng.integers(lo, hi + 1, size=(n, r)).astype(np.float64)
    G2 = rng.integers(lo, hi + 1, size=(r, m)).astype(np.float64)
    Y = rng.integers(-5, 6, size=n).astype(np.float64)
    return np.ascontiguousarray(G1 @ G2), Y


def pascal(n: int) -> np.ndarray:
    """Symmetric Pascal matrix P_ij = C(i+j, i), i, j = 0..n-1 (Section 4.2 test family)."""
    from math import comb
    return np.array([[comb(i + j, i) for j in range(n)] for i in range(n)], dtype=np.float64)


def usv(n: int, seed: int = 0):
    """U S V^T with U (5n x n) and V (n x n) random orthonormal columns and
    S = diag(2^{(i-1)/2}), i = 1..n (Section 4.2 test family). Returns (A, U, S, V)."""
    rng = rng_for(101, seed)
    U = np.linalg.qr(rng.standard_normal((5 * n, n)))[0]
    V = np.linalg.qr(rng.standard_normal((n, n)))[0]
    S = np.diag(2.0 ** (np.arange(n) / 2.0))
    return U @ S @ V.T, U, S, V


def kahan(n: int, c: float) -> np.ndarray:
    """Kahan matrix K(c, s) = diag(1, s, ..., s^{n-1}) T with T upper triangular,
    T_ii = 1 and T_ij = -c for j > i, c^2 + s^2 = 1 (Section 4.2 test family)."""
    s = np.sqrt(1.0 - c * c)
    T = np.triu(-c * np.ones((n, n)), 1) + np.eye(n)
    return np.diag(s ** np.arange(n)) @ T
