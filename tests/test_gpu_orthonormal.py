"""Orthonormal variant (Section 2.2, alpha = 1/||Gamma_r||) and orthogonal variant (alpha = 1)
on the GPU against the oracle's variants of the same names. Orthonormal: against the
oracle's orthonormal variant: FP64 mode with RG_ORTHONORMAL (every step in FP64) to the
FP64 bar, and the state that mixed mode keeps (the same variant with FP32 projections).

Bar: identical rank trajectories and basis-row indices; X within 1e-10 (FP64) or 1e-4
(mixed) relative; the exported orthonormal basis Q and P^-1 within the same bar scaled
by 1e3, as for the general variant."""
import numpy as np
import pytest

from gpu_helpers import run_batch, run_stream, torch_cuda
from oracle import checks, fp64
from paper_2106_11594_gb300 import inputs, rg

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOLMIX = 1e-4
ORTHO64 = rg.RG_FP64 | rg.RG_ORTHONORMAL


def assert_ortho_parity(g, o, tol, tol_state):
    assert g["rank"] == o.rank
    np.testing.assert_array_equal(g["indep"], o.indep)
    np.testing.assert_array_equal(g["basis"], o.basis_rows)
    assert checks.rel_err(g["X"], o.X) <= tol, checks.rel_err(g["X"], o.X)
    np.testing.assert_array_equal(g["Ct"], g["C"])  # the dual basis is Q itself
    assert checks.rel_err(g["C"], o.C) <= tol_state, checks.rel_err(g["C"], o.C)
    assert checks.rel_err(g["Pinv"], o.Pinv) <= tol_state, checks.rel_err(g["Pinv"], o.Pinv)
    Q = g["C"]
    assert np.abs(Q @ Q.T - np.eye(g["rank"])).max() <= 1e-12


@pytest.mark.parametrize("k", [1, 3, 32, 256])
def test_small_stream_fp64_orthonormal(k):
    s = inputs.small_stream()
    o = fp64.solve(s.A, s.Y, tol=1e-10, variant=fp64.ORTHONORMAL)
    assert_ortho_parity(run_stream(s.A, s.Y, k, mode=ORTHO64), o, TOL64, 1e3 * TOL64)


@pytest.mark.parametrize("n,m,r,k", [(4096, 1024, 64, 32), (3001, 1000, 48, 3001),
                                     (2500, 333, 40, 77)])
def test_large_stream_fp64_orthonormal(n, m, r, k):
    s = inputs.large_stream(n, m, r)
    o = fp64.solve(s.A, s.Y, tol=1e-10, variant=fp64.ORTHONORMAL)
    assert_ortho_parity(run_stream(s.A, s.Y, k, mode=ORTHO64), o, TOL64, 1e3 * TOL64)
    # both variants reach the same minimum-norm solution
    og = fp64.solve(s.A, s.Y, tol=1e-10)
    assert checks.rel_err(o.X, og.X) <= TOL64


@pytest.mark.parametrize("k", [32, 4096])
def test_mixed_mode_state_is_the_orthonormal_variant(k):
    """Mixed mode keeps Q in FP64 (appends are decided and formed in FP64), so Q matches
    the oracle's orthonormal variant to the FP64 bar; P^-1 accumulates FP32 partial sums
    and is held to the mixed bar."""
    s = inputs.large_stream(4096, 1024, 64)
    o = fp64.solve(s.A, s.Y, tol=1e-10, variant=fp64.ORTHONORMAL)
    g = run_stream(s.A, s.Y, k, mode=rg.RG_MIXED)
    assert g["rank"] == o.rank
    np.testing.assert_array_equal(g["indep"], o.indep)
    np.testing.assert_array_equal(g["basis"], o.basis_rows)
    assert checks.rel_err(g["X"], o.X) <= TOLMIX
    assert checks.rel_err(g["C"], o.C) <= 1e3 * TOL64, checks.rel_err(g["C"], o.C)
    assert checks.rel_err(g["Pinv"], o.Pinv) <= TOLMIX, checks.rel_err(g["Pinv"], o.Pinv)


def test_fp64_orthonormal_edge_cases():
    """Zero rows, duplicates, a rank reaching m, and n < m."""
    s = inputs.large_stream(600, 96, 12)
    A = s.A.copy()
    A[5] = 0.0
    A[40:44] = 0.0
    A[100] = A[3]
    o = fp64.solve(A, s.Y, tol=1e-10, variant=fp64.ORTHONORMAL)
    for k in (1, 16, 600):
        assert_ortho_parity(run_stream(A, s.Y, k, mode=ORTHO64), o, TOL64, 1e3 * TOL64)
    rng = inputs.rng_for(301, 0)
    B = rng.standard_normal((60, 40))
    Y = rng.standard_normal(60)
    o = fp64.solve(B, Y, tol=1e-10, variant=fp64.ORTHONORMAL)
    g = run_stream(B, Y, 16, mode=ORTHO64)
    assert_ortho_parity(g, o, TOL64, 1e3 * TOL64)
    assert g["rank"] == 40
    W = rng.standard_normal((20, 90))
    g = run_stream(W, Y[:20], 7, mode=ORTHO64)
    assert g["rank"] == 20
    assert checks.rel_err(g["X"], np.linalg.pinv(W) @ Y[:20]) <= TOL64


def test_noalloc_fp64_orthonormal():
    torch, dev = torch_cuda()
    s = inputs.large_stream(2048, 256, 32)
    o = fp64.solve(s.A, s.Y, tol=1e-10, variant=fp64.ORTHONORMAL)
    X = torch.empty(256, dtype=torch.float64, device=dev)
    rank = rg.solve_noalloc(torch.from_numpy(s.A).to(dev), torch.from_numpy(s.Y).to(dev), X,
                            1e-10, ORTHO64)
    assert rank == o.rank
    assert checks.rel_err(X.cpu().numpy(), o.X) <= TOL64


@pytest.mark.parametrize("calls", [1, 2])
def test_batch_fp64_orthonormal(calls):
    """The batched kernel's FP64 orthonormal instantiation against the oracle's orthonormal
    variant, instance by instance (32 instances spread over the uneven batch). The bar of
    an ill-conditioned instance is max(1e-10, 1e3 eps kappa_2(A)), as for the general
    variant."""
    batch = inputs.uneven_batch(4096, instances=list(range(0, 4096, 128)))
    ores = [fp64.solve(s.A, s.Y, tol=1e-10, variant=fp64.ORTHONORMAL) for s in batch.streams]
    g = run_batch(batch, mode=ORTHO64, calls=calls)
    for b, (s, o) in enumerate(zip(batch.streams, ores)):
        assert g["ranks"][b] == o.rank, b
        rb = int(g["row_base"][b])
        np.testing.assert_array_equal(g["indep"][rb:rb + s.n], o.indep, err_msg=f"instance {b}")
        X = g["X"][g["xo"][b]:g["xo"][b + 1]]
        sv = np.linalg.svd(s.A, compute_uv=False)
        sv = sv[sv > sv[0] * 1e-12]
        tb = max(TOL64, 1e3 * np.finfo(float).eps * sv[0] / sv[-1])
        assert checks.rel_err(X, o.X) <= tb, (b, checks.rel_err(X, o.X), tb)


# ---------------------------------------------------------------------------------------
# Orthogonal variant (Section 2.2, alpha = 1): C holds the raw rejections (orthogonal rows),
# Ct the same rows over their squared norms; appends leave older rows unchanged.
# ---------------------------------------------------------------------------------------
ORTHOG64 = rg.RG_FP64 | rg.RG_ORTHOGONAL


def assert_orthog_parity(g, o, tol, tol_state):
    assert g["rank"] == o.rank
    np.testing.assert_array_equal(g["indep"], o.indep)
    np.testing.assert_array_equal(g["basis"], o.basis_rows)
    assert checks.rel_err(g["X"], o.X) <= tol, checks.rel_err(g["X"], o.X)
    assert checks.rel_err(g["C"], o.C) <= tol_state, checks.rel_err(g["C"], o.C)
    assert checks.rel_err(g["Ct"], o.Ct) <= tol_state, checks.rel_err(g["Ct"], o.Ct)
    assert checks.rel_err(g["Pinv"], o.Pinv) <= tol_state, checks.rel_err(g["Pinv"], o.Pinv)
    C = g["C"]
    G = C @ C.T  # orthogonal rows: a diagonal Gram matrix
    d = np.sqrt(np.diag(G))
    assert np.abs(G / np.outer(d, d) - np.eye(g["rank"])).max() <= 1e-12
    np.testing.assert_allclose(g["Ct"] * (d ** 2)[:, None], C, rtol=1e-13, atol=0)


@pytest.mark.parametrize("k", [1, 3, 32, 256])
def test_small_stream_fp64_orthogonal(k):
    s = inputs.small_stream()
    o = fp64.solve(s.A, s.Y, tol=1e-10, variant=fp64.ORTHOGONAL)
    assert_orthog_parity(run_stream(s.A, s.Y, k, mode=ORTHOG64), o, TOL64, 1e3 * TOL64)


@pytest.mark.parametrize("n,m,r,k", [(4096, 1024, 64, 32), (3001, 1000, 48, 3001),
                                     (2500, 333, 40, 77)])
def test_large_stream_fp64_orthogonal(n, m, r, k):
    s = inputs.large_stream(n, m, r)
    o = fp64.solve(s.A, s.Y, tol=1e-10, variant=fp64.ORTHOGONAL)
    assert_orthog_parity(run_stream(s.A, s.Y, k, mode=ORTHOG64), o, TOL64, 1e3 * TOL64)
    og = fp64.solve(s.A, s.Y, tol=1e-10)
    assert checks.rel_err(o.X, og.X) <= TOL64


def test_fp64_orthogonal_edge_cases_noalloc_and_batch():
    s = inputs.large_stream(600, 96, 12)
    A = s.A.copy()
    A[5] = 0.0
    A[100] = A[3]
    o = fp64.solve(A, s.Y, tol=1e-10, variant=fp64.ORTHOGONAL)
    for k in (1, 16, 600):
        assert_orthog_parity(run_stream(A, s.Y, k, mode=ORTHOG64), o, TOL64, 1e3 * TOL64)
    torch, dev = torch_cuda()
    X = torch.empty(96, dtype=torch.float64, device=dev)
    rank = rg.solve_noalloc(torch.from_numpy(A).to(dev), torch.from_numpy(s.Y).to(dev), X, 1e-10, ORTHOG64)
    assert rank == o.rank and checks.rel_err(X.cpu().numpy(), o.X) <= TOL64
    batch = inputs.uneven_batch(4096, instances=list(range(3, 4096, 256)))
    ores = [fp64.solve(b.A, b.Y, tol=1e-10, variant=fp64.ORTHOGONAL) for b in batch.streams]
    g = run_batch(batch, mode=ORTHOG64, calls=2)
    for b, (sb, ob) in enumerate(zip(batch.streams, ores)):
        assert g["ranks"][b] == ob.rank, b
        rb = int(g["row_base"][b])
        np.testing.assert_array_equal(g["indep"][rb:rb + sb.n], ob.indep)
        sv = np.linalg.svd(sb.A, compute_uv=False)
        sv = sv[sv > sv[0] * 1e-12]
        tb = max(TOL64, 1e3 * np.finfo(float).eps * sv[0] / sv[-1])
        assert checks.rel_err(g["X"][g["xo"][b]:g["xo"][b + 1]], ob.X) <= tb, b


def test_orthogonal_excludes_mixed_and_orthonormal():
    for flags in (rg.RG_ORTHOGONAL | rg.RG_MIXED, rg.RG_ORTHOGONAL | rg.RG_ORTHONORMAL):
        with pytest.raises(rg.RGError) as ei:
            rg.RankGreville(16, 1e-10, flags)
        assert ei.value.code == rg.RG_EINVAL
