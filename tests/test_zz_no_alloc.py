"""rg_solve_noalloc: the allocation-free entry point for callers that cannot call
cudaMalloc (a latency-critical loop that cannot take cudaMalloc's implicit device
synchronisation, or a host whose device memory belongs to its own allocator).

Checked through the C ABI against the allocating entry points (rg_init, rg_add_rows,
rg_solution) and directly against the CPU oracle, on two calls in a row: the second call
reuses the fixed device array that the first one left behind, so it also checks that each
call clears what must start at zero. This file is collected last on purpose."""
import numpy as np
import pytest

from gpu_helpers import run_stream, torch_cuda
from oracle import checks, fp64
from paper_2106_11594_gb300 import inputs, rg

pytestmark = pytest.mark.gpu


def noalloc(A, Y, mode=rg.RG_FP64, r_max=0):
    torch, dev = torch_cuda()
    At = torch.from_numpy(np.ascontiguousarray(A)).to(dev)
    Yt = torch.from_numpy(np.ascontiguousarray(Y)).to(dev)
    X = torch.full((A.shape[1],), np.nan, dtype=torch.float64, device=dev)
    rank = rg.solve_noalloc(At, Yt, X, tol=1e-10, mode=mode, r_max=r_max)
    return X.cpu().numpy(), rank


def test_noalloc_matches_allocating_api_two_calls_in_a_row():
    first = inputs.large_stream(4096, 256, 24)
    second = inputs.small_stream()  # different m: the array's layout changes between calls
    for s in (first, second):
        X, rank = noalloc(s.A, s.Y)
        ref = run_stream(s.A, s.Y, s.n, export=False)
        assert rank == ref["rank"]
        assert checks.rel_err(X, ref["X"]) <= 1e-10
        o = fp64.solve(s.A, s.Y, tol=1e-10)  # and the oracle itself
        assert rank == o.rank == s.rank
        assert checks.rel_err(X, o.X) <= 1e-10


def test_noalloc_mixed_matches_allocating_api():
    s = inputs.large_stream(3000, 200, 20)
    for _ in range(2):
        X, rank = noalloc(s.A, s.Y, mode=rg.RG_MIXED)
        ref = run_stream(s.A, s.Y, s.n, mode=rg.RG_MIXED, export=False)
        assert rank == ref["rank"] == 20
        assert checks.rel_err(X, ref["X"]) <= 1e-4
        o = fp64.solve(s.A, s.Y, tol=1e-10, variant=fp64.ORTHONORMAL)
        assert checks.rel_err(X, o.X) <= 1e-4


def test_noalloc_asynchronous_call_matches_synchronous():
    """rank_out NULL: the call returns without waiting; after a synchronisation X equals
    the synchronous call's, bit for bit (same kernels, same order)."""
    torch, dev = torch_cuda()
    s = inputs.large_stream(2048, 128, 16)
    At = torch.from_numpy(s.A).to(dev)
    Yt = torch.from_numpy(s.Y).to(dev)
    X1 = torch.full((128,), np.nan, dtype=torch.float64, device=dev)
    X2 = torch.full((128,), np.nan, dtype=torch.float64, device=dev)
    assert rg.solve_noalloc(At, Yt, X1) == 16
    assert rg.solve_noalloc(At, Yt, X2, with_rank=False) is None
    torch.cuda.synchronize()
    assert torch.equal(X1, X2)
    assert checks.rel_err(X2.cpu().numpy(), fp64.solve(s.A, s.Y, tol=1e-10).X) <= 1e-10


def test_noalloc_rejects_sizes_beyond_the_fixed_array():
    torch, dev = torch_cuda()
    m = 2048
    A = torch.zeros((4, m), dtype=torch.float64, device=dev)
    Y = torch.zeros(4, dtype=torch.float64, device=dev)
    X = torch.zeros(m, dtype=torch.float64, device=dev)
    with pytest.raises(rg.RGError) as ei:
        rg.solve_noalloc(A, Y, X)
    assert ei.value.code == rg.RG_EINVAL
    assert "fixed maximum" in str(ei.value)
    # the same problem fits once r_max is lowered
    assert rg.solve_noalloc(A, Y, X, r_max=64) == 0
