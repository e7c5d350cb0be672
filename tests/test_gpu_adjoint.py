"""Adjoint parity: rg_adjoint / rg_batch_adjoint (through the autograd Functions) against
the oracle's pseudoinverse-derivative formula, and against central finite differences of
the GPU forward along rank-preserving directions (h = 1e-6 for the entries of the factors;
h = 1e-3 along y, where the loss is exactly quadratic; <= 1e-6 relative, FP64)."""
import numpy as np
import pytest

from gpu_helpers import torch_cuda
from oracle import adjoint as oadj
from oracle import checks, fp64
from paper_2106_11594_gb300 import inputs, rg

pytestmark = pytest.mark.gpu

CASES = [(60, 20, 20), (15, 40, 15), (200, 30, 6), (256, 64, 8), (300, 130, 100)]


def _case(n, m, r, seed):
    rng = inputs.rng_for(500, seed)
    A = rng.standard_normal((n, r)) @ rng.standard_normal((r, m))
    y = A @ rng.standard_normal(m) + 1e-3 * rng.standard_normal(n)
    g = rng.standard_normal(m)
    return A, y, g


@pytest.mark.parametrize("mode,tol", [(rg.RG_FP64, 1e-9), (rg.RG_FP64 | rg.RG_ORTHONORMAL, 1e-9),
                                      (rg.RG_MIXED, 1e-3)])
def test_adjoint_matches_oracle(mode, tol):
    torch, dev = torch_cuda()
    from paper_2106_11594_gb300.autograd import lstsq_rg
    for k, (n, m, r) in enumerate(CASES):
        A, y, g = _case(n, m, r, k)
        o = fp64.solve(A, y, tol=1e-10)
        assert o.rank == min(n, m, r)
        Xo, gAo, gyo = oadj.adjoint(A, y, g, rank=o.rank)
        At = torch.from_numpy(A).to(dev).requires_grad_(True)
        yt = torch.from_numpy(y).to(dev).requires_grad_(True)
        X = lstsq_rg(At, yt, 1e-10, mode)
        X.backward(torch.from_numpy(g).to(dev))
        assert checks.rel_err(X.detach().cpu().numpy(), Xo) <= max(tol, 1e-10), (n, m, r)
        assert checks.rel_err(At.grad.cpu().numpy(), gAo) <= tol, (n, m, r, checks.rel_err(At.grad.cpu().numpy(), gAo))
        assert checks.rel_err(yt.grad.cpu().numpy(), gyo) <= tol, (n, m, r)


def test_finite_differences_along_factor_directions():
    """Workload-4 shape (n 2048, m 256, r 32): 64 sampled entries of the factors G1, G2
    (each a rank-preserving direction of A = G1 G2) and 16 random directions of y;
    L = ||X - x_t||^2."""
    torch, dev = torch_cuda()
    from paper_2106_11594_gb300.autograd import lstsq_rg
    n, m, r = 2048, 256, 32
    G1, G2, x, e = inputs.factor_stream_factors(n, m, r, 1e-3, inputs.rng_for(4, 0))
    A = G1 @ G2
    y = A @ x + e
    xt = inputs.rng_for(4, 1 << 20).standard_normal(m)
    xt_t = torch.from_numpy(xt).to(dev)
    At = torch.from_numpy(A).to(dev).requires_grad_(True)
    yt = torch.from_numpy(y).to(dev).requires_grad_(True)
    L = ((lstsq_rg(At, yt) - xt_t) ** 2).sum()
    L.backward()
    gA = At.grad.cpu().numpy()
    gy = yt.grad.cpu().numpy()

    def loss(Anp, ynp):
        with torch.no_grad():
            X = lstsq_rg(torch.from_numpy(Anp).to(dev), torch.from_numpy(ynp).to(dev))
            return float(((X - xt_t) ** 2).sum().item())

    h = 1e-6
    rng = np.random.default_rng(77)
    fds, ans = [], []
    for s in range(64):
        if s % 2 == 0:  # G1[i, k]: row i of A moves along G2[k]
            i, k = int(rng.integers(n)), int(rng.integers(r))
            dA = np.zeros_like(A)
            dA[i] = G2[k]
        else:  # G2[k, c]: column c of A moves along G1[:, k]
            k, c = int(rng.integers(r)), int(rng.integers(m))
            dA = np.zeros_like(A)
            dA[:, c] = G1[:, k]
        fds.append((loss(A + h * dA, y) - loss(A - h * dA, y)) / (2 * h))
        ans.append(float(np.sum(gA * dA)))
    # y: dense random directions (a single entry of y moves L by ~1e-2 of its value per
    # unit, so at h = 1e-6 its difference quotient would be mostly FP64 rounding of L).
    # For fixed A, L = ||A^+ y - x_t||^2 is exactly quadratic in y, so a central difference
    # has no truncation error at any step: h_y = 1e-3 keeps the quotient clear of the
    # forward's rounding (at 1e-6 that rounding alone is ~1e-6 of the derivative).
    h_y = 1e-3
    fdy, any_ = [], []
    for s in range(16):
        dy = rng.standard_normal(n)
        fdy.append((loss(A, y + h_y * dy) - loss(A, y - h_y * dy)) / (2 * h_y))
        any_.append(float(gy @ dy))
    # norm-wise relative error over the sampled directional derivatives
    errA = np.linalg.norm(np.array(fds) - np.array(ans)) / np.linalg.norm(ans)
    erry = np.linalg.norm(np.array(fdy) - np.array(any_)) / np.linalg.norm(any_)
    assert errA <= 1e-6 and erry <= 1e-6, (errA, erry)


def test_gradcheck_full_rank():
    torch, dev = torch_cuda()
    from paper_2106_11594_gb300.autograd import lstsq_rg
    rng = np.random.default_rng(9)
    A = torch.from_numpy(rng.standard_normal((7, 4))).to(dev).requires_grad_(True)
    y = torch.from_numpy(rng.standard_normal(7)).to(dev).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda a, b: lstsq_rg(a, b), (A, y), eps=1e-6, atol=1e-8, rtol=1e-6)


@pytest.mark.parametrize("mode,tol", [(rg.RG_FP64, 1e-9), (rg.RG_FP64 | rg.RG_ORTHONORMAL, 1e-9),
                                      (rg.RG_MIXED, 1e-3)])
def test_batch_adjoint_matches_oracle(mode, tol):
    torch, dev = torch_cuda()
    from paper_2106_11594_gb300.autograd import lstsq_rg_batch
    shapes = [(2048, 256, 32)] * 3 + [(n, m, r) for (n, m, r) in CASES]
    mats = []
    for k, (n, m, r) in enumerate(shapes):
        mats.append(_case(n, m, r, 100 + k))
    n = np.array([a.shape[0] for a, _, _ in mats])
    m = np.array([a.shape[1] for a, _, _ in mats])
    ro = np.concatenate([[0], np.cumsum(n)]).astype(np.int64)
    eo = np.concatenate([[0], np.cumsum(n * m)]).astype(np.int64)
    Ap = torch.from_numpy(np.concatenate([a.reshape(-1) for a, _, _ in mats])).to(dev).requires_grad_(True)
    yp = torch.from_numpy(np.concatenate([y for _, y, _ in mats])).to(dev).requires_grad_(True)
    gp = torch.from_numpy(np.concatenate([g for _, _, g in mats])).to(dev)
    X = lstsq_rg_batch(Ap, yp, torch.from_numpy(ro).to(dev), torch.from_numpy(eo).to(dev), m, 1e-10, mode)
    X.backward(gp)
    gA = Ap.grad.cpu().numpy()
    gy = yp.grad.cpu().numpy()
    xo = np.concatenate([[0], np.cumsum(m)])
    for b, (A, y, g) in enumerate(mats):
        o = fp64.solve(A, y, tol=1e-10)
        Xo, gAo, gyo = oadj.adjoint(A, y, g, rank=o.rank)
        assert checks.rel_err(X.detach().cpu().numpy()[xo[b]:xo[b + 1]], Xo) <= max(tol, 1e-10), b
        assert checks.rel_err(gA[eo[b]:eo[b + 1]].reshape(A.shape), gAo) <= tol, b
        assert checks.rel_err(gy[ro[b]:ro[b + 1]], gyo) <= tol, b
