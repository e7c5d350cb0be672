"""Helpers for the GPU parity tests: run a stream / batch through the C ABI (via the
ctypes binding) and run the same rows through the CPU oracle."""
import numpy as np

from oracle import fp64
from paper_2106_11594_gb300 import rg


def torch_cuda():
    import torch
    return torch, torch.device("cuda:0")


def run_stream(A, Y, k, tol=1e-10, mode=rg.RG_FP64, test=rg.RG_TEST_REL, r_max=0,
               export=True, raise_errors=True):
    """Feed A's rows in calls of k rows; return a dict of results (numpy)."""
    torch, dev = torch_cuda()
    n, m = A.shape
    At = torch.from_numpy(np.ascontiguousarray(A)).to(dev)
    Yt = torch.from_numpy(np.ascontiguousarray(Y)).to(dev)
    ind = torch.full((max(n, 1),), 7, dtype=torch.uint8, device=dev)
    st = rg.RankGreville(m, tol, mode, test, r_max)
    err = None
    for j0 in range(0, n, max(k, 1)):
        st.add_rows(At[j0:j0 + k], Yt[j0:j0 + k], ind[j0:j0 + k])
    X = torch.empty(m, dtype=torch.float64, device=dev)
    try:
        rank = st.solution(X)
    except rg.RGError as e:
        if raise_errors:
            raise
        err = e
        rank = st.rank()
        st.solution(X, with_rank=False)
    out = dict(X=X.cpu().numpy(), rank=rank, indep=ind[:n].cpu().numpy(), err=err,
               rows_seen=st.rows_seen())
    if export:
        cap = max(rank, 1)
        C = torch.zeros(cap * m, dtype=torch.float64, device=dev)
        Ct = torch.zeros(cap * m, dtype=torch.float64, device=dev)
        P = torch.zeros(cap * cap, dtype=torch.float64, device=dev)
        w = torch.zeros(cap, dtype=torch.float64, device=dev)
        basis = torch.zeros(cap, dtype=torch.int64, device=dev)
        r2 = st.export(C, Ct, P, w, basis, capacity=cap)
        out.update(C=C[:r2 * m].cpu().numpy().reshape(r2, m),
                   Ct=Ct[:r2 * m].cpu().numpy().reshape(r2, m),
                   Pinv=P[:r2 * r2].cpu().numpy().reshape(r2, r2), w=w[:r2].cpu().numpy(),
                   basis=basis[:r2].cpu().numpy())
    out["state"] = st
    return out


def run_batch(batch, tol=1e-10, mode=rg.RG_FP64, calls=1):
    """Run a Batch through rg_batch_* (rows of each instance split into `calls` calls)."""
    torch, dev = torch_cuda()
    m = np.array([s.m for s in batch.streams], dtype=np.int64)
    bt = rg.RankGrevilleBatch(m, tol, mode)
    n = np.array([s.n for s in batch.streams], dtype=np.int64)
    total_rows = int(n.sum())
    ind = torch.full((max(total_rows, 1),), 7, dtype=torch.uint8, device=dev)
    # split every instance's rows into `calls` consecutive chunks
    row_base = np.concatenate([[0], np.cumsum(n)])
    for c in range(calls):
        lo = (n * c) // calls
        hi = (n * (c + 1)) // calls
        cnt = hi - lo
        ro = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
        eo = np.concatenate([[0], np.cumsum(cnt * m)]).astype(np.int64)
        Ap = np.concatenate([s.A[lo[b]:hi[b]].reshape(-1) for b, s in enumerate(batch.streams)]
                            + [np.zeros(0)])
        Yp = np.concatenate([s.Y[lo[b]:hi[b]] for b, s in enumerate(batch.streams)] + [np.zeros(0)])
        A_t = torch.from_numpy(np.ascontiguousarray(Ap)).to(dev)
        Y_t = torch.from_numpy(np.ascontiguousarray(Yp)).to(dev)
        ind_c = torch.full((max(int(cnt.sum()), 1),), 7, dtype=torch.uint8, device=dev)
        bt.add_rows(A_t, torch.from_numpy(ro).to(dev), torch.from_numpy(eo).to(dev), Y_t, ind_c)
        torch.cuda.synchronize()
        ic = ind_c.cpu().numpy()
        for b in range(batch.B):
            ind[int(row_base[b] + lo[b]):int(row_base[b] + hi[b])] = torch.from_numpy(
                ic[ro[b]:ro[b + 1]].copy()).to(dev)
    xo = np.concatenate([[0], np.cumsum(m)]).astype(np.int64)
    X = torch.empty(int(xo[-1]), dtype=torch.float64, device=dev)
    ranks = torch.empty(batch.B, dtype=torch.int64, device=dev)
    bt.solution(X, torch.from_numpy(xo).to(dev), ranks)
    bt.sync()
    return dict(X=X.cpu().numpy(), ranks=ranks.cpu().numpy(), indep=ind[:total_rows].cpu().numpy(),
                xo=xo, row_base=row_base, handle=bt)


def oracle_batch(batch, tol=1e-10):
    res = [fp64.solve(s.A, s.Y, tol=tol) for s in batch.streams]
    return res
