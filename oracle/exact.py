"""Exact-rational rank-Greville and an independent exact pseudoinverse (TEST INFRASTRUCTURE).

Two routes to the same exact minimum-norm least-squares solution X = A^+ Y
(Section 1, Eq. label_eq_least_squares_pseudoinverse):

  * ``alg1``: Algorithm 1 (Section 3) in ``fractions.Fraction`` arithmetic, with the
    exact test Gamma_r != 0. The method uses only field operations, so this run is
    exact (Section 3, last paragraph).
  * ``pinv_theorem1``: a rank factorization A = B C from the reduced row echelon form
    (C = the nonzero RREF rows, B = the pivot columns of A), then Theorem 1,
    A^+ = C^T (C C^T)^-1 (B^T B)^-1 B^T (Eq. eq_explicit_pseudo), all in Fractions.

The two share nothing but Fraction arithmetic; uniqueness of the Moore-Penrose inverse
(Section 1, Penrose equations) means they must agree exactly.
"""
from __future__ import annotations

from fractions import Fraction

F0 = Fraction(0)
F1 = Fraction(1)


def to_fractions(M):
    """Exact Fraction copy of a float (or int) array / nested list."""
    try:
        import numpy as np
        arr = np.asarray(M)
        if arr.ndim == 1:
            return [Fraction(float(x)) if arr.dtype.kind == "f" else Fraction(int(x)) for x in arr]
        return [to_fractions(row) for row in arr]
    except ImportError:  # pragma: no cover
        return [[Fraction(x) for x in row] for row in M]


def matmul(A, B):
    n, k, m = len(A), len(B), len(B[0]) if B else 0
    return [[sum((A[i][t] * B[t][j] for t in range(k)), F0) for j in range(m)] for i in range(n)]


def transpose(A):
    return [list(col) for col in zip(*A)] if A else []


def dot(u, v):
    return sum((a * b for a, b in zip(u, v)), F0)


def alg1(A, Y):
    """Algorithm 1 over the rows of A (list of lists of Fraction) with targets Y.

    Returns dict(X, indep, basis_rows, C, Ct, Pinv)."""
    n = len(A)
    m = len(A[0])
    C, Ct, Pinv = [], [], []
    X = [F0] * m
    indep, basis = [], []
    for idx in range(n):
        G, y = A[idx], Y[idx]
        r = len(C)
        gamma = [dot(Ct[i], G) for i in range(r)]
        Gr = [G[c] - sum((C[i][c] * gamma[i] for i in range(r)), F0) for c in range(m)]
        if any(g != 0 for g in Gr):
            s = dot(Gr, Gr)
            K = [g / s for g in Gr]
            Ct = [[Ct[i][c] - gamma[i] * K[c] for c in range(m)] for i in range(r)] + [K]
            C = C + [list(G)]
            Pinv = [row + [F0] for row in Pinv] + [[F0] * r + [F1]]
            indep.append(1)
            basis.append(idx)
        else:
            zeta = [dot(Pinv[i], gamma) for i in range(r)]
            d = F1 + dot(gamma, zeta)
            K = [sum((Ct[i][c] * zeta[i] for i in range(r)), F0) / d for c in range(m)]
            Pinv = [[Pinv[i][j] - zeta[i] * zeta[j] / d for j in range(r)] for i in range(r)]
            indep.append(0)
        dy = y - dot(G, X)
        X = [X[c] + K[c] * dy for c in range(m)]
    return dict(X=X, indep=indep, basis_rows=basis, C=C, Ct=Ct, Pinv=Pinv)


def rref(A):
    """Reduced row echelon form of A (Fractions). Returns (R, pivots)."""
    R = [list(row) for row in A]
    n = len(R)
    m = len(R[0]) if n else 0
    pivots = []
    row = 0
    for col in range(m):
        if row >= n:
            break
        p = next((i for i in range(row, n) if R[i][col] != 0), None)
        if p is None:
            continue
        R[row], R[p] = R[p], R[row]
        pv = R[row][col]
        R[row] = [x / pv for x in R[row]]
        for i in range(n):
            if i != row and R[i][col] != 0:
                f = R[i][col]
                R[i] = [a - f * b for a, b in zip(R[i], R[row])]
        pivots.append(col)
        row += 1
    return R[:len(pivots)], pivots


def solve(M, Bmat):
    """Solve M Z = Bmat exactly for square nonsingular M (Gauss-Jordan)."""
    n = len(M)
    aug = [list(M[i]) + list(Bmat[i]) for i in range(n)]
    R, piv = rref(aug)
    if piv[:n] != list(range(n)):
        raise ZeroDivisionError("singular system")
    return [row[n:] for row in R[:n]]


def inverse(M):
    n = len(M)
    return solve(M, [[F1 if i == j else F0 for j in range(n)] for i in range(n)])


def pinv_theorem1(A):
    """A^+ from the RREF rank factorization and Theorem 1 (exact). Returns (A^+, B, C)."""
    C, piv = rref(A)
    if not piv:
        n, m = len(A), len(A[0])
        return [[F0] * n for _ in range(m)], [[] for _ in range(n)], []
    B = [[row[j] for j in piv] for row in A]
    Ct = transpose(C)
    Bt = transpose(B)
    sig_inv = inverse(matmul(C, Ct))
    P_inv = inverse(matmul(Bt, B))
    Ap = matmul(matmul(matmul(Ct, sig_inv), P_inv), Bt)
    return Ap, B, C


def lstsq_theorem1(A, Y):
    Ap, _, _ = pinv_theorem1(A)
    return [dot(row, Y) for row in Ap]


def rank(A):
    return len(rref(A)[1])
