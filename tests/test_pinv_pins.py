"""Pins of the oracle's pseudoinverse update (Theorems label_th_pinv_indep and
label_th_pinv_lindep, `fp64.pinv`) to things other than itself: exact-rational Theorem 1 on
integer data, the SVD pseudoinverse, the closed form of [I_n; 1^T], the Penrose equations,
and planted mistakes that must each fail a pin."""
import numpy as np
import pytest

from oracle import checks, exact, fp64
from paper_2106_11594_gb300 import inputs


def _rank_deficient(n, m, r, seed):
    rng = np.random.default_rng(1000 + seed)
    return rng.standard_normal((n, r)) @ rng.standard_normal((r, m))


@pytest.mark.parametrize("n,m,r", [(40, 12, 5), (12, 30, 7), (25, 25, 25), (30, 8, 8), (6, 50, 6)])
def test_pinv_update_matches_svd_pseudoinverse(n, m, r):
    A = _rank_deficient(n, m, r, n + m)
    Ap, rank, _ = fp64.pinv(A, 1e-10)
    assert rank == min(n, m, r)
    assert Ap.shape == (m, n)
    ref = np.linalg.pinv(A, rcond=1e-10)
    assert checks.rel_err(Ap, ref) < 1e-10, checks.rel_err(Ap, ref)


def test_pinv_update_at_every_prefix():
    """The update's result after j rows is A_j^+ for every prefix j (checked at each j
    on a small stream with zero and repeated rows)."""
    A = _rank_deficient(18, 7, 4, 3)
    A[4] = 0.0
    A[9] = A[2] - 2 * A[5]
    for j in range(1, A.shape[0] + 1):
        Ap, rank, _ = fp64.pinv(A[:j], 1e-10)
        assert rank == np.linalg.matrix_rank(A[:j])
        assert checks.rel_err(Ap, np.linalg.pinv(A[:j], rcond=1e-10)) < 1e-11


@pytest.mark.parametrize("case", range(3))
def test_pinv_update_matches_exact_theorem1(case):
    n, m, r = [(8, 5, 3), (6, 9, 4), (7, 7, 7)][case]
    A, _ = inputs.integer_lowrank(n, m, r, case)
    ref, _, _ = exact.pinv_theorem1(exact.to_fractions(A))
    ref = np.array([[float(x) for x in row] for row in ref])
    Ap, _, _ = fp64.pinv(A, 1e-10)
    assert ref.shape == Ap.shape
    assert checks.rel_err(Ap, ref) < 1e-12, checks.rel_err(Ap, ref)


def test_pinv_update_closed_form_identity_plus_ones_row():
    """A = [I_n; 1^T] has A^+ = (I - 1 1^T / (n + 1)) [I_n 1]."""
    n = 9
    A = np.vstack([np.eye(n), np.ones((1, n))])
    ref = (np.eye(n) - np.ones((n, n)) / (n + 1)) @ np.hstack([np.eye(n), np.ones((n, 1))])
    Ap, rank, indep = fp64.pinv(A, 1e-10)
    assert rank == n and list(indep) == [1] * n + [0]
    assert np.abs(Ap - ref).max() < 1e-14


def test_pinv_update_penrose_and_agreement_with_the_solution():
    s = inputs.large_stream(300, 40, 9)
    Ap, rank, indep = fp64.pinv(s.A, 1e-10)
    o = fp64.solve(s.A, s.Y, tol=1e-10)
    assert rank == o.rank == 9
    np.testing.assert_array_equal(indep, o.indep)
    assert max(checks.penrose_residuals(s.A, Ap)) < 1e-11
    assert checks.rel_err(Ap @ s.Y, o.X) < 1e-11  # Theorems 2/3 and Theorems 4/5 agree


@pytest.mark.parametrize("mutation", [10, 11, 12])
def test_pinv_planted_mistakes_fail_a_pin(mutation):
    A = _rank_deficient(40, 12, 5, 7)
    Ap, _, _ = fp64.pinv(A, 1e-10, mutation=mutation)
    assert checks.rel_err(Ap, np.linalg.pinv(A, rcond=1e-10)) > 1e-6
