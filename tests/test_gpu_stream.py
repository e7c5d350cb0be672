"""Single-stream parity: CUDA path (through the C ABI) vs the CPU oracle.

Bar: FP64 mode ||X - X_ref|| / ||X_ref|| <= 1e-10, mixed mode <= 1e-4 (the tolerances the
target states), and identical rank trajectories (per-row independence flags and basis-row
indices compared as integer arrays)."""
import numpy as np
import pytest

from gpu_helpers import run_stream, torch_cuda
from oracle import checks, fp64
from paper_2106_11594_gb300 import inputs, rg

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOLMIX = 1e-4


def assert_parity(g, o, tol, compare_state=True):
    assert g["rank"] == o.rank
    np.testing.assert_array_equal(g["indep"], o.indep)
    np.testing.assert_array_equal(g["basis"], o.basis_rows)
    assert checks.rel_err(g["X"], o.X) <= tol, checks.rel_err(g["X"], o.X)
    if compare_state:
        np.testing.assert_array_equal(g["C"], o.C)  # the basis rows are input rows, verbatim
        assert checks.rel_err(g["Ct"], o.Ct) <= 1e3 * tol
        assert checks.rel_err(g["Pinv"], o.Pinv) <= 1e3 * tol


@pytest.mark.parametrize("k", [1, 3, 32, 256])
def test_small_stream_fp64(k):
    s = inputs.small_stream()
    o = fp64.solve(s.A, s.Y, tol=1e-10)
    g = run_stream(s.A, s.Y, k)
    assert_parity(g, o, TOL64)


@pytest.mark.parametrize("k", [1, 32, 256])
def test_small_stream_mixed(k):
    s = inputs.small_stream()
    o = fp64.solve(s.A, s.Y, tol=1e-10)
    g = run_stream(s.A, s.Y, k, mode=rg.RG_MIXED)
    assert g["rank"] == o.rank
    np.testing.assert_array_equal(g["indep"], o.indep)
    np.testing.assert_array_equal(g["basis"], o.basis_rows)
    assert checks.rel_err(g["X"], o.X) <= TOLMIX
    # orthonormal variant: the exported basis has orthonormal rows spanning span(C)
    Q = g["C"]
    assert np.linalg.norm(Q @ Q.T - np.eye(g["rank"])) <= 1e-10
    assert np.linalg.norm(o.C - (o.C @ Q.T) @ Q) <= 1e-10 * np.linalg.norm(o.C)


@pytest.mark.parametrize("n,m,r,k", [(4096, 1024, 64, 32), (4096, 1024, 64, 4096),
                                     (3001, 1000, 48, 1000), (2500, 333, 40, 77)])
def test_large_stream_fp64(n, m, r, k):
    s = inputs.large_stream(n, m, r)
    o = fp64.solve(s.A, s.Y, tol=1e-10)
    g = run_stream(s.A, s.Y, k)
    assert_parity(g, o, TOL64)


@pytest.mark.parametrize("n,m,r,k", [(4096, 1024, 64, 32), (3001, 1000, 48, 3001)])
def test_large_stream_mixed(n, m, r, k):
    s = inputs.large_stream(n, m, r)
    o = fp64.solve(s.A, s.Y, tol=1e-10)
    g = run_stream(s.A, s.Y, k, mode=rg.RG_MIXED)
    assert g["rank"] == o.rank
    np.testing.assert_array_equal(g["indep"], o.indep)
    np.testing.assert_array_equal(g["basis"], o.basis_rows)
    assert checks.rel_err(g["X"], o.X) <= TOLMIX


def test_full_size_large_stream_fp64_k32():
    """The benchmark's workload at full size (n=65536, m=1024, r=64) in the benchmark's
    launch configuration (32 rows per call): full oracle comparison plus properties."""
    s = inputs.large_stream()
    g = run_stream(s.A, s.Y, 32, export=True)
    o = fp64.solve(s.A, s.Y, tol=1e-10)
    assert_parity(g, o, TOL64, compare_state=False)
    assert g["rank"] == 64 and list(g["basis"]) == list(range(64))
    assert checks.normal_eq_residual(s.A, g["X"], s.Y) <= 1e-13
    assert checks.rowspace_residual(g["X"], g["Ct"], g["C"]) <= 1e-12


def test_full_size_large_stream_mixed_one_call():
    s = inputs.large_stream()
    g = run_stream(s.A, s.Y, s.n, mode=rg.RG_MIXED, export=False)
    assert g["rank"] == 64
    np.testing.assert_array_equal(np.nonzero(g["indep"])[0], np.arange(64))
    o = fp64.solve(s.A, s.Y, tol=1e-10)
    assert checks.rel_err(g["X"], o.X) <= TOLMIX


def _late_growth_stream(n, m, rank, late, seed):
    """Rows in a rank-`rank` row space (the first `rank` rows grow it), except the rows in
    `late`, which each bring one new direction; Y = A x + noise 1e-3."""
    rng = np.random.default_rng(seed)
    extra = len(late)
    G2 = rng.standard_normal((rank + extra, m))
    F = np.zeros((n, rank + extra))
    F[:, :rank] = rng.standard_normal((n, rank))
    for q, j in enumerate(late):
        F[j, rank + q] = 1.0 + rng.random()
    A = np.ascontiguousarray(F @ G2)
    Y = A @ rng.standard_normal(m) + 1e-3 * rng.standard_normal(n)
    return A, Y


@pytest.mark.parametrize("case", ["ragged", "late_growth", "rank_80", "odd_m"])
def test_mixed_large_calls_tensor_core_blocks(case):
    """One mixed-mode call of >= 8192 rows runs its blocks of >= 8192 rows through the
    tensor-core chunk path on the whole GPU. After the rank-growth sections the blocks grow
    x4 from 64 rows (64, 256, 1024, 4096), so the block after them holds the rest of the
    call:
      ragged      - m = 512, rank 40: an 8200-row block at row 5504 (64 chunks and one of
                    8 rows);
      late_growth - as ragged, plus two new directions at rows 10000 and 10001, inside that
                    block: the chunks' fused sums are discarded, the 4496 rows before the
                    first are summed again from G, and the FP64 section takes both;
      rank_80     - m = 512, rank 80 (above the shared-memory staging of the fused sums):
                    an 8250-row block at row 5536 sums its rows from G;
      odd_m       - m = 333 (row starts off 16-byte boundaries), rank 40: an 8300-row block.
    Flags and basis rows as integer arrays and X within 1e-4 of the FP64 oracle."""
    n, m, rank = {"ragged": (13704, 512, 40), "late_growth": (13704, 512, 40),
                  "rank_80": (13786, 512, 80), "odd_m": (13804, 333, 40)}[case]
    late = [10000, 10001] if case == "late_growth" else []
    seed = {"ragged": 11, "late_growth": 12, "rank_80": 13, "odd_m": 14}[case]
    A, Y = _late_growth_stream(n, m, rank, late, seed=seed)
    o = fp64.solve(A, Y, tol=1e-10)
    assert o.rank == rank + len(late)
    g = run_stream(A, Y, n, mode=rg.RG_MIXED, export=True)
    assert g["rank"] == o.rank
    np.testing.assert_array_equal(g["indep"], o.indep)
    np.testing.assert_array_equal(g["basis"], o.basis_rows)
    assert checks.rel_err(g["X"], o.X) <= TOLMIX, checks.rel_err(g["X"], o.X)


# ------------------------------------------------------------------ edge cases

def test_zero_and_duplicate_rows():
    s = inputs.large_stream(600, 96, 12)
    A = s.A.copy()
    A[5] = 0.0
    A[40:44] = 0.0
    A[100] = A[3]
    A[200] = A[0]
    o = fp64.solve(A, s.Y, tol=1e-10)
    for k in (1, 16, 600):
        assert_parity(run_stream(A, s.Y, k), o, TOL64)


def test_all_zero_stream_and_empty_call():
    torch, dev = torch_cuda()
    A = np.zeros((50, 7))
    g = run_stream(A, np.ones(50), 8)
    assert g["rank"] == 0 and not g["X"].any() and not g["indep"].any()
    st = rg.RankGreville(7)
    st.add_rows(torch.zeros((0, 7), dtype=torch.float64, device=dev),
                torch.zeros(0, dtype=torch.float64, device=dev))
    assert st.rank() == 0 and st.rows_seen() == 0


def test_single_column():
    A = np.array([[2.0], [0.0], [4.0], [-1.0]])
    Y = np.array([1.0, 5.0, 2.0, 3.0])
    o = fp64.solve(A, Y, tol=1e-10)
    assert_parity(run_stream(A, Y, 1), o, TOL64)
    assert_parity(run_stream(A, Y, 4), o, TOL64)


@pytest.mark.parametrize("mode,tol", [(rg.RG_FP64, TOL64), (rg.RG_MIXED, TOLMIX)])
def test_full_rank_square_and_wide(mode, tol):
    rng = inputs.rng_for(300, 0)
    A = rng.standard_normal((48, 48))
    Y = rng.standard_normal(48)
    g = run_stream(A, Y, 16, mode=mode)
    assert g["rank"] == 48
    assert checks.rel_err(g["X"], np.linalg.solve(A, Y)) <= tol * 100
    W = rng.standard_normal((20, 90))  # n < m: minimum-norm interpolation
    g = run_stream(W, Y[:20], 7, mode=mode)
    assert g["rank"] == 20
    assert checks.rel_err(g["X"], np.linalg.pinv(W) @ Y[:20]) <= tol


def test_capacity_overflow():
    rng = inputs.rng_for(301, 0)
    A = rng.standard_normal((40, 12)) @ np.diag(np.ones(12))
    Y = rng.standard_normal(40)
    o = fp64.solve(A, Y, tol=1e-10, r_max=5)
    assert o.status == 4 and o.rows_done == 5
    g = run_stream(A, Y, 40, r_max=5, export=False, raise_errors=False)
    assert g["err"] is not None and g["err"].code == rg.RG_ECAPACITY
    assert g["rows_seen"] == 5 and g["rank"] == 5
    assert checks.rel_err(g["X"], o.X) <= TOL64
    assert (g["indep"][5:] == 0xFF).all()


def test_nonfinite_row_stops_and_state_survives():
    torch, dev = torch_cuda()
    s = inputs.large_stream(300, 64, 10)
    A = s.A.copy()
    A[77, 3] = np.nan
    st = rg.RankGreville(64)
    At = torch.from_numpy(A).to(dev)
    Yt = torch.from_numpy(s.Y).to(dev)
    st.add_rows(At[:100], Yt[:100])
    with pytest.raises(rg.RGError) as ei:
        st.sync()
    assert ei.value.code == rg.RG_ENONFINITE
    assert st.rows_seen() == 77
    X = torch.empty(64, dtype=torch.float64, device=dev)
    st.solution(X)
    o = fp64.solve(A[:77], s.Y[:77], tol=1e-10)
    assert checks.rel_err(X.cpu().numpy(), o.X) <= TOL64
    # the error was reported once; the stream continues with clean rows
    st.add_rows(At[78:300], Yt[78:300])
    st.solution(X)
    keep = np.r_[0:77, 78:300]
    o2 = fp64.solve(A[keep], s.Y[keep], tol=1e-10)
    assert checks.rel_err(X.cpu().numpy(), o2.X) <= TOL64


def test_paper_threshold_mode_and_default_eps():
    s = inputs.large_stream(400, 64, 9)
    A = s.A * 1e-3  # row norms < 1: PAPER and REL differ in principle
    for test in (rg.RG_TEST_REL, rg.RG_TEST_PAPER):
        for tol in (1e-10, 0.0):
            o = fp64.solve(A, s.Y, tol=tol, test_mode=test)
            assert_parity(run_stream(A, s.Y, 50, tol=tol, test=test), o, TOL64)


def test_reset_rerun_is_bit_identical_and_host_api_matches():
    torch, dev = torch_cuda()
    s = inputs.large_stream(2000, 256, 24)
    g1 = run_stream(s.A, s.Y, 64, export=False)
    st = g1["state"]
    st.reset()
    At = torch.from_numpy(s.A).to(dev)
    Yt = torch.from_numpy(s.Y).to(dev)
    for j0 in range(0, 2000, 64):
        st.add_rows(At[j0:j0 + 64], Yt[j0:j0 + 64])
    X = torch.empty(256, dtype=torch.float64, device=dev)
    st.solution(X)
    np.testing.assert_array_equal(X.cpu().numpy(), g1["X"])
    # host-buffer entry points
    st.reset()
    ind = np.zeros(2000, dtype=np.uint8)
    for j0 in range(0, 2000, 64):
        st.add_rows_host(s.A[j0:j0 + 64], s.Y[j0:j0 + 64], ind[j0:j0 + 64])
    Xh = np.empty(256)
    assert st.solution_host(Xh) == 24
    np.testing.assert_array_equal(Xh, g1["X"])
    np.testing.assert_array_equal(ind, g1["indep"])


def test_invalid_arguments():
    torch, dev = torch_cuda()
    with pytest.raises(rg.RGError) as ei:
        rg.RankGreville(0)
    assert ei.value.code == rg.RG_EINVAL
    with pytest.raises(rg.RGError):
        rg.RankGreville(4, tol=float("nan"))
    st = rg.RankGreville(4)
    with pytest.raises(rg.RGError):
        st.solution(None)


@pytest.mark.parametrize("mode,tol", [(rg.RG_FP64, 1e-10), (rg.RG_MIXED, 1e-4)])
def test_solutions_and_exports_between_calls_of_mixed_sizes(mode, tol):
    """Calls of at most 64 rows defer their update of P and u to the next call; a
    solution, an export or a larger call in between must see every row so far. X after
    every call matches the oracle on the rows fed up to then."""
    torch, dev = torch_cuda()
    s = inputs.large_stream(900, 96, 12)
    At = torch.from_numpy(s.A).to(dev)
    Yt = torch.from_numpy(s.Y).to(dev)
    st = rg.RankGreville(96, 1e-10, mode)
    X = torch.empty(96, dtype=torch.float64, device=dev)
    sizes = [7, 32, 64, 65, 1, 200, 32, 32, 3, 64, 400]
    j0 = 0
    for c, k in enumerate(sizes):
        k = min(k, s.n - j0)
        st.add_rows(At[j0:j0 + k], Yt[j0:j0 + k])
        j0 += k
        if c % 3 == 2:
            cap = 96
            C = torch.zeros(cap * 96, dtype=torch.float64, device=dev)
            w = torch.zeros(cap, dtype=torch.float64, device=dev)
            st.export(C, None, None, w, None, capacity=cap)
        if c % 2 == 1 or j0 == s.n:
            st.solution(X)
            o = fp64.solve(s.A[:j0], s.Y[:j0], tol=1e-10)
            assert checks.rel_err(X.cpu().numpy(), o.X) <= tol, (c, j0)
    assert j0 == s.n
    st.close()


def test_ill_conditioned_rank_growth():
    """Workload 5 at reduced size (n 4096, m 512, r 64; singular values log-uniform on
    [1e-6, 1], 8 rank-growth phases, 5% combinations of earlier rows), tol 1e-8.

    The method projects with one classical Gram-Schmidt pass and no reorthogonalisation
    (Section 2.2; Section 4.2 finds it neither forward nor mixed stable). As directions
    with small relative rejections are appended, the orthonormal basis loses
    orthogonality and the general variant's dual basis loses accuracy, until the
    rounding noise in a dependent row's rejection exceeds tol and every later row is
    declared independent. The oracle follows the generator's rank growth up to a row d
    (past phase 0 here); over that prefix the GPU must take the oracle's decisions and
    reach an X as close to the exact solution as the oracle's. Past d both runs decide
    on rounding noise, so the full stream only checks what holds for any run: a run that
    completes ends at or above the generator's rank, and a run that stops does so by the
    capacity stop at rank m or by the breakdown check."""
    s = inputs.ill_conditioned_stream(n=4096, m=512, r=64)
    tol = 1e-8
    torch, dev = torch_cuda()
    for mode, variant in ((rg.RG_FP64, fp64.GENERAL), (rg.RG_MIXED, fp64.ORTHONORMAL)):
        o = fp64.solve(s.A, s.Y, tol=tol, variant=variant)
        d = int(np.flatnonzero(o.indep != s.growth)[0])
        assert d >= 512, d  # the oracle holds the generator's rank growth through phase 0
        od = fp64.solve(s.A[:d], s.Y[:d], tol=tol, variant=variant)
        for n_run in (d, s.n):
            At = torch.from_numpy(s.A[:n_run]).to(dev)
            Yt = torch.from_numpy(s.Y[:n_run]).to(dev)
            st = rg.RankGreville(512, tol, mode)
            if mode == rg.RG_MIXED:
                st.set_screen(1e-9)  # below the smallest relative rejection of a new direction
            ind = torch.zeros(n_run, dtype=torch.uint8, device=dev)
            for j0 in range(0, n_run, 256):
                st.add_rows(At[j0:j0 + 256], Yt[j0:j0 + 256], ind[j0:j0 + 256])
            X = torch.empty(512, dtype=torch.float64, device=dev)
            try:
                rank = st.solution(X)
            except rg.RGError as e:
                # past d the noise can declare a row independent at rank m (the stream
                # stops with RG_ECAPACITY, as the oracle does), or the noisy state can make
                # a Woodbury denominator non-positive (the breakdown check stops it with
                # RG_ENONFINITE); either way the rows from there on are not applied
                assert n_run == s.n and e.code in (rg.RG_ECAPACITY, rg.RG_ENONFINITE), (mode, e)
                rank = st.rank()
                assert o.status == 4
                assert rank == 512 or e.code == rg.RG_ENONFINITE
            got = ind.cpu().numpy()
            st.close()
            np.testing.assert_array_equal(got[:d], od.indep)
            if n_run == d:
                # The method is not forward stable (Section 4.2): on this prefix the
                # oracle itself is far from the exact minimum-norm solution (Xs, by SVD
                # at the prefix rank). The GPU run of the same method must land no
                # further from Xs than ten times the oracle's own error.
                assert rank == od.rank
                U, sv, Vt = np.linalg.svd(s.A[:d], full_matrices=False)
                r = od.rank
                Xs = Vt[:r].T @ ((U[:, :r].T @ s.Y[:d]) / sv[:r])
                floor = TOL64 if mode == rg.RG_FP64 else TOLMIX
                err_o = checks.rel_err(od.X, Xs)
                err_g = checks.rel_err(X.cpu().numpy(), Xs)
                assert err_g <= max(floor, 10 * err_o), (err_g, err_o)
            else:
                assert rank >= s.rank
