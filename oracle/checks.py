"""Properties the exact result must satisfy (TEST INFRASTRUCTURE).

  * Penrose equations (Section 1, Eqs. label_eq_penrose:1-4) on A^+ built from the
    maintained factors, A^+ = Ct^T P^-1 B^T (Section 2.1) with B = A Ct^T
    (A Ct^T = B C Ct^T = B because C Ct^T = I).
  * Invariants: X in rowspace(A); normal equations A^T (A X - Y) = 0; dual basis
    Ct C^T = I_r; P^-1 (B^T B) = I_r.
  * The Section 4.2 accuracy metrics e_algo (Eq. label_eq_stability_factor) and
    res_algo (Eq. label_eq_residual_error).
"""
from __future__ import annotations

import numpy as np

EPS_M = np.finfo(np.float64).eps


def pinv_from_factors(A, Ct, Pinv):
    """A^+ = Ct^T P^-1 B^T with B = A Ct^T."""
    B = A @ Ct.T
    return Ct.T @ Pinv @ B.T


def penrose_residuals(A, Ap):
    """Relative residuals of the four Penrose equations."""
    nA = np.linalg.norm(A, 2)
    nP = np.linalg.norm(Ap, 2)
    AAp = A @ Ap
    ApA = Ap @ A
    r1 = np.linalg.norm(AAp @ A - A, 2) / nA
    r2 = np.linalg.norm(ApA @ Ap - Ap, 2) / nP
    r3 = np.linalg.norm(AAp - AAp.T, 2) / max(np.linalg.norm(AAp, 2), 1e-300)
    r4 = np.linalg.norm(ApA - ApA.T, 2) / max(np.linalg.norm(ApA, 2), 1e-300)
    return r1, r2, r3, r4


def rowspace_residual(X, Ct, C):
    """||X - Ct^T (C X)|| / ||X||: zero iff X lies in span of C's rows."""
    nx = np.linalg.norm(X)
    if nx == 0:
        return 0.0
    return np.linalg.norm(X - Ct.T @ (C @ X)) / nx


def normal_eq_residual(A, X, Y):
    """||A^T (A X - Y)|| / (||A||^2 ||X|| + ||A|| ||Y||)."""
    nA = np.linalg.norm(A, 2)
    den = nA * nA * np.linalg.norm(X) + nA * np.linalg.norm(Y)
    return np.linalg.norm(A.T @ (A @ X - Y)) / max(den, 1e-300)


def dual_basis_residual(Ct, C):
    r = C.shape[0]
    return np.linalg.norm(Ct @ C.T - np.eye(r), 2)


def pinv_gram_residual(A, Ct, Pinv):
    B = A @ Ct.T
    r = Ct.shape[0]
    return np.linalg.norm(Pinv @ (B.T @ B) - np.eye(r), 2)


def stability_factor(Ap_algo, Ap_exact, A):
    """e_algo = ||A^+_algo - A^+|| / (eps_M ||A^+|| kappa_2(A))."""
    sv = np.linalg.svd(A, compute_uv=False)
    sv = sv[sv > sv[0] * 1e-300]
    kappa = sv[0] / sv[-1]
    return np.linalg.norm(Ap_algo - Ap_exact, 2) / (EPS_M * np.linalg.norm(Ap_exact, 2) * kappa)


def residual_error(Ap_algo, A):
    """res_algo = ||A^+_algo A - I|| / (||A|| ||A^+_algo||)."""
    m = A.shape[1]
    return np.linalg.norm(Ap_algo @ A - np.eye(m), 2) / (
        np.linalg.norm(A, 2) * np.linalg.norm(Ap_algo, 2))


def kappa2(A):
    sv = np.linalg.svd(A, compute_uv=False)
    return sv[0] / sv[-1]


def rel_err(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    d = np.linalg.norm(ref)
    return np.linalg.norm(x - ref) / (d if d > 0 else 1.0)
