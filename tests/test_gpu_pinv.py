"""rg_pinv (the pseudoinverse formed from the stream's factorization) against the oracle's
row-by-row update of Theorems label_th_pinv_indep / label_th_pinv_lindep.

Bar: FP64 (general and orthonormal variants) within 1e-10 relative of the oracle's A^+,
after every call of a stream, or within eps kappa(P) where the basis rows make P = B^T B
ill-conditioned (the oracle's own error is of that size there); mixed mode within 1e-4. At the full size of the single-stream
workload (n 65536, m 1024, r 64) the oracle's O(m n^2) update is out of reach, so a sampled
column is compared with the oracle's least-squares solution for a unit target (column i
of A^+ is A^+ e_i), and A^+ y with the GPU solution."""
import numpy as np
import pytest

from gpu_helpers import torch_cuda
from oracle import checks, fp64
from paper_2106_11594_gb300 import inputs, rg

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOLMIX = 1e-4
ORTHO64 = rg.RG_FP64 | rg.RG_ORTHONORMAL


def gpu_pinv_after_calls(A, Y, k, mode, pad=0):
    """Feed A in calls of k rows; after each call form A^+ of the prefix. Returns the list
    of (rows so far, A^+) and the final state's solution X."""
    torch, dev = torch_cuda()
    n, m = A.shape
    At = torch.from_numpy(np.ascontiguousarray(A)).to(dev)
    Yt = torch.from_numpy(np.ascontiguousarray(Y)).to(dev)
    st = rg.RankGreville(m, 1e-10, mode)
    out = []
    for j0 in range(0, n, k):
        j1 = min(n, j0 + k)
        st.add_rows(At[j0:j1], Yt[j0:j1])
        Ap = torch.full((m, j1 + pad), 7.0, dtype=torch.float64, device=dev)
        st.pinv(At[:j1], Ap)
        Apn = Ap.cpu().numpy()
        if pad:
            assert (Apn[:, j1:] == 7.0).all()  # the padding past n is not written
        out.append((j1, Apn[:, :j1].copy()))
    X = torch.empty(m, dtype=torch.float64, device=dev)
    st.solution(X)
    st.close()
    return out, X.cpu().numpy()


@pytest.mark.parametrize("mode", [rg.RG_FP64, ORTHO64])
def test_pinv_after_every_call_small_stream(mode):
    s = inputs.small_stream()
    res, X = gpu_pinv_after_calls(s.A, s.Y, 32, mode, pad=3)
    for j, Ap in res:
        ref, _, _ = fp64.pinv(s.A[:j], 1e-10)
        assert checks.rel_err(Ap, ref) <= TOL64, (j, checks.rel_err(Ap, ref))
    assert checks.rel_err(res[-1][1] @ s.Y, X) <= TOL64


@pytest.mark.parametrize("n,m,r,k", [(2048, 256, 32, 700), (1500, 333, 40, 1500)])
@pytest.mark.parametrize("mode", [rg.RG_FP64, ORTHO64])
def test_pinv_large_stream(n, m, r, k, mode):
    """Algorithm 1's basis is the first r rows themselves, so P = B^T B carries their
    conditioning (kappa(P) ~ 5e7 on these Gaussian streams although A's nonzero singular
    values lie within a factor 2): both the oracle's A^+ and the GPU's carry errors near
    eps kappa(P) (the oracle is 1.2e-9 from the SVD pseudoinverse at n 2048). So A^+ is
    held to max(1e-10, eps kappa(P)) against the oracle, and to no further from the SVD
    pseudoinverse than the oracle itself (or 1e-10)."""
    s = inputs.large_stream(n, m, r)
    ref, rank, _ = fp64.pinv(s.A, 1e-10)
    assert rank == r
    og = fp64.solve(s.A, s.Y, tol=1e-10)
    tol_pinv = max(TOL64, np.finfo(float).eps * np.linalg.cond(og.Pinv))
    svd = np.linalg.pinv(s.A, rcond=1e-10)
    res, X = gpu_pinv_after_calls(s.A, s.Y, k, mode)
    j, Ap = res[-1]
    assert j == n
    assert checks.rel_err(Ap, ref) <= tol_pinv, (checks.rel_err(Ap, ref), tol_pinv)
    assert checks.rel_err(Ap, svd) <= max(TOL64, checks.rel_err(ref, svd))
    assert checks.rel_err(Ap @ s.Y, X) <= tol_pinv


def test_pinv_mixed_mode():
    s = inputs.large_stream(2048, 256, 32)
    ref, _, _ = fp64.pinv(s.A, 1e-10)
    res, _ = gpu_pinv_after_calls(s.A, s.Y, 2048, rg.RG_MIXED)
    assert checks.rel_err(res[-1][1], ref) <= TOLMIX


def test_pinv_edge_cases():
    rng = inputs.rng_for(302, 0)
    # zero and repeated rows, wide (n < m) and square full rank
    s = inputs.large_stream(300, 50, 7)
    A = s.A.copy()
    A[3] = 0.0
    A[10] = A[4]
    for B in (A, rng.standard_normal((20, 90)), rng.standard_normal((40, 40))):
        res, _ = gpu_pinv_after_calls(B, np.ones(B.shape[0]), 16, rg.RG_FP64)
        ref, _, _ = fp64.pinv(B, 1e-10)
        assert checks.rel_err(res[-1][1], ref) <= TOL64
        assert checks.rel_err(res[-1][1], np.linalg.pinv(B, rcond=1e-10)) <= TOL64
    # an all-zero stream has A^+ = 0
    res, _ = gpu_pinv_after_calls(np.zeros((9, 5)), np.ones(9), 4, rg.RG_FP64)
    assert all((Ap == 0.0).all() for _, Ap in res)


def test_pinv_full_size_single_stream():
    torch, dev = torch_cuda()
    s = inputs.large_stream()
    n, m = s.A.shape
    At = torch.from_numpy(s.A).to(dev)
    Yt = torch.from_numpy(s.Y).to(dev)
    st = rg.RankGreville(m, 1e-10, rg.RG_FP64)
    for j0 in range(0, n, 32):
        st.add_rows(At[j0:j0 + 32], Yt[j0:j0 + 32])
    X = torch.empty(m, dtype=torch.float64, device=dev)
    assert st.solution(X) == 64
    Ap = torch.empty((m, n), dtype=torch.float64, device=dev)
    st.pinv(At, Ap)
    st.close()
    i = 40000  # a dependent row's column
    e = np.zeros(n)
    e[i] = 1.0
    o = fp64.solve(s.A, e, tol=1e-10)
    tol_pinv = max(TOL64, np.finfo(float).eps * np.linalg.cond(o.Pinv))
    assert checks.rel_err((Ap @ Yt).cpu().numpy(), X.cpu().numpy()) <= tol_pinv
    assert checks.rel_err(Ap[:, i].cpu().numpy(), o.X) <= tol_pinv
    # A^+ A A^+ = A^+ along a random direction
    u = torch.from_numpy(inputs.rng_for(303, 0).standard_normal(n)).to(dev)
    v = Ap @ u
    assert checks.rel_err((Ap @ (At @ v)).cpu().numpy(), v.cpu().numpy()) <= tol_pinv


def test_pinv_after_capacity_stop_and_argument_checks():
    """A stream stopped by RG_ECAPACITY keeps the rows it applied: rg_pinv of those rows
    is their pseudoinverse. Bad arguments are refused on the host."""
    torch, dev = torch_cuda()
    s = inputs.large_stream(200, 40, 12)
    At = torch.from_numpy(s.A).to(dev)
    Yt = torch.from_numpy(s.Y).to(dev)
    st = rg.RankGreville(40, 1e-10, rg.RG_FP64, rg.RG_TEST_REL, 8)  # r_max 8 < rank 12
    st.add_rows(At, Yt)
    X = torch.empty(40, dtype=torch.float64, device=dev)
    with pytest.raises(rg.RGError) as ei:
        st.solution(X)
    assert ei.value.code == rg.RG_ECAPACITY
    n_ok = st.rows_seen()
    assert n_ok == 8  # the first 12 rows are independent; the ninth stops the stream
    Ap = torch.empty((40, n_ok), dtype=torch.float64, device=dev)
    st.pinv(At[:n_ok], Ap)
    ref, _, _ = fp64.pinv(s.A[:n_ok], 1e-10)
    assert checks.rel_err(Ap.cpu().numpy(), ref) <= TOL64
    Ap2 = torch.empty((40, 4), dtype=torch.float64, device=dev)
    with pytest.raises(rg.RGError) as ei:
        st.pinv(At[:n_ok], Ap2)  # row stride 4 < n
    assert ei.value.code == rg.RG_EINVAL
    st.close()
