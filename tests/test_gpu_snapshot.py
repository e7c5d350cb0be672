"""Factor snapshots (rg_snapshot / rg_restore) and gradients through intermediate
solutions X_n (autograd.lstsq_rg_path).

* Checkpoint / resume: a stream snapshotted after n1 rows and restored (into itself after
  more rows, or into a fresh state) continues to the same solution, flags and rank as an
  uninterrupted run, in FP64, the orthonormal variant and mixed mode.
* A snapshot from a state of another shape is refused (RG_EINVAL at the next sync) and
  leaves the state as it was.
* Gradients of a loss on X at two intermediate row counts and at the end agree with the
  oracle's pseudoinverse derivative on the corresponding prefixes (summed), and with
  central finite differences along rank-preserving directions (factor entries, h = 1e-6;
  dense directions of y, h = 1e-3 where L is exactly quadratic) to 1e-6 in FP64."""
import numpy as np
import pytest

from gpu_helpers import torch_cuda
from oracle import adjoint as oadj
from oracle import checks, fp64
from paper_2106_11594_gb300 import inputs, rg

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode,tol", [(rg.RG_FP64, 1e-12), (rg.RG_FP64 | rg.RG_ORTHONORMAL, 1e-12),
                                      (rg.RG_MIXED, 1e-7)])
def test_snapshot_restore_continues_the_stream(mode, tol):
    torch, dev = torch_cuda()
    s = inputs.large_stream(3000, 200, 24)
    A = torch.from_numpy(s.A).to(dev)
    Y = torch.from_numpy(s.Y).to(dev)
    n1 = 17  # mid rank growth: the snapshot holds a partial basis
    ref = rg.RankGreville(200, 1e-10, mode)
    ind_ref = torch.zeros(s.n, dtype=torch.uint8, device=dev)
    for j0 in range(0, s.n, 100):
        ref.add_rows(A[j0:j0 + 100], Y[j0:j0 + 100], ind_ref[j0:j0 + 100])
    X_ref = torch.empty(200, dtype=torch.float64, device=dev)
    assert ref.solution(X_ref) == 24
    st = rg.RankGreville(200, 1e-10, mode)
    st.add_rows(A[:n1], Y[:n1])
    buf = st.new_snapshot_buffer()
    st.snapshot(buf)
    st.add_rows(A[n1:2000], Y[n1:2000])  # move on, then go back
    st.restore(buf)
    assert st.rows_seen() == n1 and st.rank() == n1
    fresh = rg.RankGreville(200, 1e-10, mode)
    fresh.restore(buf)
    for h in (st, fresh):
        ind = torch.zeros(s.n - n1, dtype=torch.uint8, device=dev)
        h.add_rows(A[n1:], Y[n1:], ind)
        X = torch.empty(200, dtype=torch.float64, device=dev)
        assert h.solution(X) == 24
        assert h.rows_seen() == s.n
        assert torch.equal(ind, ind_ref[n1:])
        assert checks.rel_err(X.cpu().numpy(), X_ref.cpu().numpy()) <= tol
        o = fp64.solve(s.A, s.Y, tol=1e-10)
        assert checks.rel_err(X.cpu().numpy(), o.X) <= (1e-10 if tol < 1e-9 else 1e-4)
        h.close()
    ref.close()


def test_restore_refuses_a_foreign_snapshot():
    torch, dev = torch_cuda()
    a = rg.RankGreville(64, 1e-10, rg.RG_FP64)
    b = rg.RankGreville(64, 1e-10, rg.RG_FP64, r_max=32)  # other r_max: other layout
    s = inputs.small_stream()
    a.add_rows(torch.from_numpy(s.A).to(dev), torch.from_numpy(s.Y).to(dev))
    buf = a.new_snapshot_buffer()
    a.snapshot(buf)
    b.add_rows(torch.from_numpy(s.A[:5]).to(dev), torch.from_numpy(s.Y[:5]).to(dev))
    b.restore(buf[:b.snapshot_size()])
    with pytest.raises(rg.RGError) as ei:
        b.sync()
    assert ei.value.code == rg.RG_EINVAL
    assert b.rows_seen() == 5 and b.rank() == 5  # unchanged
    junk = torch.zeros(a.snapshot_size(), dtype=torch.uint8, device=dev)
    a.restore(junk)
    with pytest.raises(rg.RGError):
        a.sync()
    assert a.rank() == 8
    with pytest.raises(rg.RGError):  # too small: refused on the host
        a.restore(buf[:100])
    a.close()
    b.close()


def _path_loss_grads(A, y, counts, targets, mode=rg.RG_FP64):
    torch, dev = torch_cuda()
    from paper_2106_11594_gb300.autograd import lstsq_rg_path
    At = torch.from_numpy(A).to(dev).requires_grad_(True)
    yt = torch.from_numpy(y).to(dev).requires_grad_(True)
    T = torch.from_numpy(targets).to(dev)
    Xs = lstsq_rg_path(At, yt, counts, 1e-10, mode)
    L = ((Xs - T) ** 2).sum()
    L.backward()
    return Xs.detach().cpu().numpy(), At.grad.cpu().numpy(), yt.grad.cpu().numpy()


def test_gradients_through_intermediate_solutions_match_the_oracle():
    n, m, r = 2048, 256, 32
    G1, G2, x, e = inputs.factor_stream_factors(n, m, r, 1e-3, inputs.rng_for(4, 7))
    A = G1 @ G2
    y = A @ x + e
    counts = [20, 700, 2048]  # rank 20 (full row rank), then rank 32 twice
    targets = inputs.rng_for(4, 1 << 21).standard_normal((len(counts), m))
    Xs, gA, gy = _path_loss_grads(A, y, counts, targets)
    gA_ref = np.zeros_like(A)
    gy_ref = np.zeros_like(y)
    for i, n_i in enumerate(counts):
        o = fp64.solve(A[:n_i], y[:n_i], tol=1e-10)
        assert o.rank == min(n_i, r)
        assert checks.rel_err(Xs[i], o.X) <= 1e-10
        Xo, gAo, gyo = oadj.adjoint(A[:n_i], y[:n_i], 2.0 * (Xs[i] - targets[i]), rank=o.rank)
        gA_ref[:n_i] += gAo
        gy_ref[:n_i] += gyo
    assert checks.rel_err(gA, gA_ref) <= 1e-9, checks.rel_err(gA, gA_ref)
    assert checks.rel_err(gy, gy_ref) <= 1e-9, checks.rel_err(gy, gy_ref)


def test_gradients_through_intermediate_solutions_finite_differences():
    torch, dev = torch_cuda()
    from paper_2106_11594_gb300.autograd import lstsq_rg_path
    n, m, r = 2048, 256, 32
    G1, G2, x, e = inputs.factor_stream_factors(n, m, r, 1e-3, inputs.rng_for(4, 8))
    A = G1 @ G2
    y = A @ x + e
    counts = [700, 1500, 2048]
    targets = inputs.rng_for(4, 1 << 22).standard_normal((len(counts), m))
    T = torch.from_numpy(targets).to(dev)
    _, gA, gy = _path_loss_grads(A, y, counts, targets)

    def loss(Anp, ynp):
        with torch.no_grad():
            Xs = lstsq_rg_path(torch.from_numpy(Anp).to(dev), torch.from_numpy(ynp).to(dev), counts)
            return float(((Xs - T) ** 2).sum().item())

    h = 1e-6
    rng = np.random.default_rng(78)
    fds, ans = [], []
    for s_ in range(48):
        dA = np.zeros_like(A)
        if s_ % 2 == 0:  # G1[i, k]: row i of A moves along G2[k] (rank-preserving)
            i, k = int(rng.integers(n)), int(rng.integers(r))
            dA[i] = G2[k]
        else:  # G2[k, c]: column c moves along G1[:, k]
            k, c = int(rng.integers(r)), int(rng.integers(m))
            dA[:, c] = G1[:, k]
        fds.append((loss(A + h * dA, y) - loss(A - h * dA, y)) / (2 * h))
        ans.append(float(np.sum(gA * dA)))
    h_y = 1e-3  # L is exactly quadratic in y for fixed A
    fdy, any_ = [], []
    for s_ in range(12):
        dy = rng.standard_normal(n)
        fdy.append((loss(A, y + h_y * dy) - loss(A, y - h_y * dy)) / (2 * h_y))
        any_.append(float(gy @ dy))
    errA = np.linalg.norm(np.array(fds) - np.array(ans)) / np.linalg.norm(ans)
    erry = np.linalg.norm(np.array(fdy) - np.array(any_)) / np.linalg.norm(any_)
    assert errA <= 1e-6 and erry <= 1e-6, (errA, erry)


def test_path_counts_are_validated():
    torch, dev = torch_cuda()
    from paper_2106_11594_gb300.autograd import lstsq_rg_path
    A = torch.zeros((10, 4), dtype=torch.float64, device=dev)
    y = torch.zeros(10, dtype=torch.float64, device=dev)
    for bad in ([5, 5], [6, 3], [11], [-1, 2]):
        with pytest.raises(ValueError):
            lstsq_rg_path(A, y, bad)
