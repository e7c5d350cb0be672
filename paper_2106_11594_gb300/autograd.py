"""torch.autograd.Function around the rank-Greville solve: X = A^+ y forward on the GPU
(rg_init / rg_add_rows / rg_solution), and the adjoint kernel (rg_adjoint) backward.

The gradient is the derivative of the minimum-norm least-squares solution on the manifold
of matrices of fixed rank: for a rank-deficient A it is exact along perturbations that
keep the rank (for example perturbations of the factors of A = G1 G2); a generic
perturbation of a rank-deficient A changes the rank, where A^+ is not differentiable.
"""
from __future__ import annotations

import torch

from . import rg


class _LstsqRG(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, y, tol, mode):
        A = A.contiguous()
        y = y.contiguous()
        st = rg.RankGreville(A.shape[1], tol, mode)
        if A.shape[0] > 0:
            st.add_rows(A, y)
        X = torch.empty(A.shape[1], dtype=torch.float64, device=A.device)
        st.solution(X, with_rank=False)
        ctx.st = st
        ctx.save_for_backward(A, y)
        return X

    @staticmethod
    def backward(ctx, gX):
        A, y = ctx.saved_tensors
        gA = torch.empty_like(A)
        gy = torch.empty_like(y)
        ctx.st.adjoint(A, y, gX.contiguous(), gA, gy)
        return gA, gy, None, None


def lstsq_rg(A, y, tol: float = 1e-10, mode: int = rg.RG_FP64):
    """X = A^+ y for A (n, m) and y (n,) float64 CUDA tensors, differentiable in A and y."""
    return _LstsqRG.apply(A, y, tol, mode)


class _LstsqRGBatch(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A_packed, y_packed, row_offsets, elem_offsets, m_list, tol, mode):
        bt = rg.RankGrevilleBatch(m_list, tol, mode)
        bt.add_rows(A_packed, row_offsets, elem_offsets, y_packed)
        X = torch.empty(int(sum(int(m) for m in m_list)), dtype=torch.float64, device=A_packed.device)
        bt.solution(X)
        ctx.bt = bt
        ctx.save_for_backward(A_packed, y_packed, row_offsets, elem_offsets)
        return X

    @staticmethod
    def backward(ctx, gX):
        A, y, ro, eo = ctx.saved_tensors
        gA = torch.empty_like(A)
        gy = torch.empty_like(y)
        ctx.bt.adjoint(A, ro, eo, y, y.numel(), gX.contiguous(), gA, gy)
        return gA, gy, None, None, None, None, None


def lstsq_rg_batch(A_packed, y_packed, row_offsets, elem_offsets, m_list, tol: float = 1e-10,
                   mode: int = rg.RG_FP64):
    """X_packed (instances back to back by m_b) for a packed batch (rg_batch_add_rows
    layout), differentiable in A_packed and y_packed."""
    return _LstsqRGBatch.apply(A_packed, y_packed, row_offsets, elem_offsets, list(m_list), tol, mode)


class _LstsqRGPath(torch.autograd.Function):
    """X_n = A_n^+ y_n at several row counts n_1 < n_2 < ... of one stream. The forward
    feeds the rows once and takes a factor snapshot (rg_snapshot) at every n_i; the
    backward restores each snapshot into a scratch state and runs the adjoint kernel on
    the rows [0, n_i), so the gradient of a loss on intermediate solutions needs no second
    pass over the stream."""

    @staticmethod
    def forward(ctx, A, y, counts, tol, mode):
        A = A.contiguous()
        y = y.contiguous()
        m = A.shape[1]
        st = rg.RankGreville(m, tol, mode)
        Xs = torch.empty((len(counts), m), dtype=torch.float64, device=A.device)
        snaps = []
        prev = 0
        for i, n_i in enumerate(counts):
            if n_i > prev:
                st.add_rows(A[prev:n_i], y[prev:n_i])
            st.solution(Xs[i], with_rank=False)
            buf = st.new_snapshot_buffer(A.device)
            st.snapshot(buf)
            snaps.append(buf)
            prev = n_i
        st.sync()
        st.close()
        ctx.snaps = snaps
        ctx.counts = counts
        ctx.tol, ctx.mode = tol, mode
        ctx.save_for_backward(A, y)
        return Xs

    @staticmethod
    def backward(ctx, gX):
        A, y = ctx.saved_tensors
        gA = torch.zeros_like(A)
        gy = torch.zeros_like(y)
        st = rg.RankGreville(A.shape[1], ctx.tol, ctx.mode)
        for i, n_i in enumerate(ctx.counts):
            g = gX[i].contiguous()
            if n_i == 0 or not bool(torch.any(g != 0)):
                continue
            st.restore(ctx.snaps[i])
            gA_i = torch.empty((n_i, A.shape[1]), dtype=torch.float64, device=A.device)
            gy_i = torch.empty(n_i, dtype=torch.float64, device=A.device)
            st.adjoint(A[:n_i], y[:n_i], g, gA_i, gy_i)
            gA[:n_i] += gA_i
            gy[:n_i] += gy_i
        st.sync()
        st.close()
        return gA, gy, None, None, None


def lstsq_rg_path(A, y, counts, tol: float = 1e-10, mode: int = rg.RG_FP64):
    """Solutions X_{n_i} = A_{n_i}^+ y_{n_i} after the first n_i rows, for increasing row
    counts `counts`, as a (len(counts), m) tensor differentiable in A and y (gradients flow
    through every intermediate solution via factor snapshots)."""
    counts = [int(c) for c in counts]
    if any(b <= a for a, b in zip(counts, counts[1:])) or (counts and (counts[0] < 0 or counts[-1] > A.shape[0])):
        raise ValueError("counts must increase strictly and lie in [0, n]")
    return _LstsqRGPath.apply(A, y, counts, tol, mode)
