"""Adjoint of the minimum-norm least-squares solution X = A^+ y (TEST INFRASTRUCTURE).

Only tests/, the smoke check and the bench's CPU legs use this module; the CUDA path
shares nothing with it.

For a loss L(X) with g = dL/dX, differentiating A^+ on the manifold of matrices of fixed
rank (the classical derivative of the pseudoinverse, obtained from the four Penrose
equations of Section 1, Eqs. label_eq_penrose:1-4) gives, with
    h = A^+T g,  rho = y - A X,  z = A^+T X,  g_perp = (I - A^+ A) g,
    dL/dy = h,
    dL/dA = -h X^T + rho (A^+ h)^T + z g_perp^T.
The paper does not state this derivative; it follows from A^+ = Ct^T P^-1 B^T
(Section 2.1), which is what the GPU adjoint evaluates. Here A^+ is formed by a library
pseudoinverse (np.linalg.pinv with a rank cut-off) or from the FP64 oracle's factors,
and the formula is evaluated term by term with dense products, nothing fused.
"""
from __future__ import annotations

import numpy as np


def pinv_rank(A, rank: int) -> np.ndarray:
    """Pseudoinverse of A truncated to its `rank` largest singular values (SVD)."""
    U, s, Vt = np.linalg.svd(np.asarray(A, dtype=np.float64), full_matrices=False)
    k = int(rank)
    if k == 0:
        return np.zeros((A.shape[1], A.shape[0]))
    return (Vt[:k].T / s[:k]) @ U[:, :k].T


def adjoint(A, y, g, Ap=None, rank=None, mutation: int = 0):
    """Returns (X, dL/dA, dL/dy) for X = A^+ y and dL/dX = g.

    Ap: the pseudoinverse to use (default: SVD pseudoinverse at `rank`, or at the
    numerical rank when rank is None). mutation != 0 plants a known mistake (tests only):
    1 drops the rho term, 2 drops the z term, 3 flips the sign of the h X^T term,
    4 uses g in place of g_perp."""
    A = np.asarray(A, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64).reshape(-1)
    g = np.asarray(g, dtype=np.float64).reshape(-1)
    if Ap is None:
        if rank is None:
            rank = np.linalg.matrix_rank(A)
        Ap = pinv_rank(A, rank)
    X = Ap @ y
    h = Ap.T @ g
    rho = y - A @ X
    z = Ap.T @ X
    Aph = Ap @ h
    gperp = g - Ap @ (A @ g)
    if mutation == 4:
        gperp = g
    t1 = -np.outer(h, X)
    if mutation == 3:
        t1 = -t1
    t2 = np.outer(rho, Aph) if mutation != 1 else 0.0
    t3 = np.outer(z, gperp) if mutation != 2 else 0.0
    gA = t1 + t2 + t3
    return X, gA, h.copy()


def adjoint_from_factors(A, y, g, Ct, Pinv):
    """Same, with A^+ = Ct^T P^-1 B^T, B = A Ct^T, from the FP64 oracle's factors."""
    A = np.asarray(A, dtype=np.float64)
    B = A @ Ct.T
    Ap = Ct.T @ Pinv @ B.T
    return adjoint(A, y, g, Ap=Ap)
