"""Pins of the oracle's adjoint (dL/dA, dL/dy of X = A^+ y) against central finite
differences of a library pseudoinverse, a closed form, and planted mistakes. CPU only."""
import numpy as np
import pytest

from oracle import adjoint as adj
from oracle import fp64

H = 1e-6


def loss(X, xt):
    return float(np.sum((X - xt) ** 2))


def fd_grad_A(A, y, xt, rank):
    G = np.zeros_like(A)
    for i in range(A.shape[0]):
        for j in range(A.shape[1]):
            E = np.zeros_like(A)
            E[i, j] = H
            lp = loss(adj.pinv_rank(A + E, rank) @ y, xt)
            lm = loss(adj.pinv_rank(A - E, rank) @ y, xt)
            G[i, j] = (lp - lm) / (2 * H)
    return G


def fd_grad_y(A, y, xt, rank):
    Ap = adj.pinv_rank(A, rank)
    G = np.zeros_like(y)
    for i in range(len(y)):
        e = np.zeros_like(y)
        e[i] = H
        G[i] = (loss(Ap @ (y + e), xt) - loss(Ap @ (y - e), xt)) / (2 * H)
    return G


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("n,m", [(7, 4), (4, 7), (5, 5)])
def test_full_rank_matches_finite_differences(n, m):
    rng = np.random.default_rng(n * 10 + m)
    A = rng.standard_normal((n, m))
    y = rng.standard_normal(n)
    xt = rng.standard_normal(m)
    r = min(n, m)
    X, gA, gy = adj.adjoint(A, y, 2 * (adj.pinv_rank(A, r) @ y - xt), rank=r)
    assert rel(gA, fd_grad_A(A, y, xt, r)) < 1e-7
    assert rel(gy, fd_grad_y(A, y, xt, r)) < 1e-7


def test_rank_deficient_tangent_directions():
    """On a rank-r matrix the derivative is exact along directions that keep the rank:
    A(t) = (G1 + t E) G2 and G1 (G2 + t F)."""
    rng = np.random.default_rng(3)
    n, m, r = 9, 6, 3
    G1 = rng.standard_normal((n, r))
    G2 = rng.standard_normal((r, m))
    A = G1 @ G2
    y = rng.standard_normal(n)
    xt = rng.standard_normal(m)
    X, gA, gy = adj.adjoint(A, y, 2 * (adj.pinv_rank(A, r) @ y - xt), rank=r)
    for _ in range(12):
        E = rng.standard_normal((n, r))
        F = rng.standard_normal((r, m))
        for dA, Ap_, Am_ in (
            (E @ G2, (G1 + H * E) @ G2, (G1 - H * E) @ G2),
            (G1 @ F, G1 @ (G2 + H * F), G1 @ (G2 - H * F)),
        ):
            fd = (loss(adj.pinv_rank(Ap_, r) @ y, xt) - loss(adj.pinv_rank(Am_, r) @ y, xt)) / (2 * H)
            an = float(np.sum(gA * dA))
            assert abs(fd - an) <= 1e-7 * max(abs(fd), 1.0)
    assert rel(gy, fd_grad_y(A, y, xt, r)) < 1e-7


def test_identity_closed_form():
    """A = I: X = y, so dL/dy = g and dL/dA = -g y^T (the other terms vanish)."""
    rng = np.random.default_rng(5)
    y = rng.standard_normal(6)
    g = rng.standard_normal(6)
    X, gA, gy = adj.adjoint(np.eye(6), y, g, rank=6)
    np.testing.assert_allclose(X, y, rtol=0, atol=1e-15)
    np.testing.assert_allclose(gy, g, rtol=0, atol=1e-15)
    np.testing.assert_allclose(gA, -np.outer(g, y), rtol=0, atol=1e-14)


def test_factors_of_the_fp64_oracle_give_the_same_adjoint():
    rng = np.random.default_rng(8)
    n, m, r = 30, 10, 4
    A = rng.standard_normal((n, r)) @ rng.standard_normal((r, m))
    y = rng.standard_normal(n)
    g = rng.standard_normal(m)
    o = fp64.solve(A, y, tol=1e-10)
    assert o.rank == r
    X1, gA1, gy1 = adj.adjoint_from_factors(A, y, g, o.Ct, o.Pinv)
    X2, gA2, gy2 = adj.adjoint(A, y, g, rank=r)
    assert rel(X1, X2) < 1e-12 and rel(gA1, gA2) < 1e-10 and rel(gy1, gy2) < 1e-10


@pytest.mark.parametrize("mutation", [1, 2, 3, 4])
def test_planted_mistakes_fail_a_pin(mutation):
    rng = np.random.default_rng(11)
    n, m, r = 9, 6, 3
    G1 = rng.standard_normal((n, r))
    G2 = rng.standard_normal((r, m))
    A = G1 @ G2
    y = rng.standard_normal(n)
    xt = rng.standard_normal(m)
    g = 2 * (adj.pinv_rank(A, r) @ y - xt)
    _, gA, _ = adj.adjoint(A, y, g, rank=r, mutation=mutation)
    worst = 0.0
    for _ in range(6):
        E = rng.standard_normal((n, r))
        F = rng.standard_normal((r, m))
        for dA, Ap_, Am_ in (((E @ G2), (G1 + H * E) @ G2, (G1 - H * E) @ G2),
                             ((G1 @ F), G1 @ (G2 + H * F), G1 @ (G2 - H * F))):
            fd = (loss(adj.pinv_rank(Ap_, r) @ y, xt) - loss(adj.pinv_rank(Am_, r) @ y, xt)) / (2 * H)
            worst = max(worst, abs(fd - float(np.sum(gA * dA))) / max(abs(fd), 1.0))
    assert worst > 1e-4
