"""Full-size batched parity: EVERY instance of the 4096-instance uneven batch and of the
1024-instance uniform batch (n 2048, m 256, r 32) through rg_batch_* in FP64 and in mixed
mode, compared instance by instance with the batched CPU oracle (plain FP64 Algorithm 1,
OpenMP over instances on all host cores):

  * the per-row rank decisions (independence flags) as integer arrays,
  * the rank of every instance,
  * X within 1e-10 relative (FP64) and 1e-4 (mixed).

A few instances of the uneven batch are unstable for the method itself: their first r rows
are ill-conditioned (kappa ~1e5, a growth row with a relative rejection of ~5e-5), the
single Gram-Schmidt pass of Algorithm 1 amplifies the rounding in the dual basis past tol,
and the FP64 oracle leaves the generator's rank growth (Section 4.2's stability caveat).
After that row both sides decide on rounding noise. For those instances the GPU must take
the oracle's decisions over the prefix the oracle resolves (rows before its departure), and
the set is pinned as measured (7 of 4096, all seeded).

The instances are generated on the host by the seeded generators (the same draws as the
sampled tests), uploaded into one packed device batch, and the oracle runs on each host
chunk right after it is uploaded, so host memory holds one chunk at a time."""
import numpy as np
import pytest

from oracle import checks, fp64
from paper_2106_11594_gb300 import inputs, rg

pytestmark = pytest.mark.gpu

CHUNK = 256  # instances generated (and checked by the oracle) at a time


def kappa_tol(A, tol):
    """The stated FP64 tolerance holds on well-conditioned inputs; an ill-conditioned
    instance may differ between two correct FP64 runs by ~2 e eps_M kappa_2(A) with the
    paper's stability factor e up to ~3e2 (Section 4.2, Table table_e_random)."""
    sv = np.linalg.svd(A, compute_uv=False)
    sv = sv[sv > sv[0] * 1e-12]
    return max(tol, 1e3 * np.finfo(float).eps * sv[0] / sv[-1])


def build_full_batch(make_stream, shapes):
    """Upload every instance into packed device buffers and run the oracle chunk by chunk.
    make_stream(b) returns instance b's inputs.Stream. Returns the device tensors, the
    offsets and the oracle's X, ranks and flags."""
    import torch
    dev = torch.device("cuda:0")
    n = np.array([s[0] for s in shapes], dtype=np.int64)
    m = np.array([s[1] for s in shapes], dtype=np.int64)
    B = len(shapes)
    ro = np.concatenate([[0], np.cumsum(n)]).astype(np.int64)
    eo = np.concatenate([[0], np.cumsum(n * m)]).astype(np.int64)
    xo = np.concatenate([[0], np.cumsum(m)]).astype(np.int64)
    A = torch.empty(int(eo[-1]), dtype=torch.float64, device=dev)
    Y = torch.empty(int(ro[-1]), dtype=torch.float64, device=dev)
    oX = np.zeros(int(xo[-1]))
    oR = np.zeros(B, dtype=np.int64)
    oI = np.zeros(int(ro[-1]), dtype=np.uint8)
    for c0 in range(0, B, CHUNK):
        ids = range(c0, min(B, c0 + CHUNK))
        streams = [make_stream(b) for b in ids]
        Ah = np.concatenate([s.A.reshape(-1) for s in streams])
        Yh = np.concatenate([s.Y for s in streams])
        A[eo[c0]:eo[ids[-1] + 1]] = torch.from_numpy(Ah).to(dev)
        Y[ro[c0]:ro[ids[-1] + 1]] = torch.from_numpy(Yh).to(dev)
        lro = ro[c0:ids[-1] + 2] - ro[c0]
        leo = eo[c0:ids[-1] + 2] - eo[c0]
        lxo = xo[c0:ids[-1] + 2] - xo[c0]
        X, R, I = fp64.solve_batch(Ah, Yh, lro, leo, lxo, tol=1e-10, with_indep=True)
        oX[xo[c0]:xo[ids[-1] + 1]] = X
        oR[c0:ids[-1] + 1] = R
        oI[ro[c0]:ro[ids[-1] + 1]] = I
    return A, Y, ro, eo, xo, m, oX, oR, oI


def oracle_departures(oI, ro, r_gen):
    """Per instance, the first row where the oracle's flags leave the generator's rank
    growth (for Gaussian factors the first min(n, r) rows grow the rank), or -1."""
    dep = np.full(len(r_gen), -1, dtype=np.int64)
    for b in range(len(r_gen)):
        f = oI[ro[b]:ro[b + 1]]
        g = np.zeros_like(f)
        g[:min(len(f), int(r_gen[b]))] = 1
        bad = np.flatnonzero(f != g)
        if bad.size:
            dep[b] = bad[0]
    return dep


def check_full_batch(A, Y, ro, eo, xo, m, oX, oR, oI, make_stream, dep):
    import torch
    dev = A.device
    ro_t, eo_t, xo_t = (torch.from_numpy(a).to(dev) for a in (ro, eo, xo))
    B = len(m)
    report = {}
    for mode, tol in ((rg.RG_FP64, 1e-10), (rg.RG_MIXED, 1e-4)):
        bt = rg.RankGrevilleBatch(m, 1e-10, mode)
        ind = torch.full((int(ro[-1]),), 7, dtype=torch.uint8, device=dev)
        X = torch.empty(int(xo[-1]), dtype=torch.float64, device=dev)
        ranks = torch.empty(B, dtype=torch.int64, device=dev)
        bt.add_rows(A, ro_t, eo_t, Y, ind)
        bt.solution(X, xo_t, ranks)
        bt.sync()
        bt.close()
        gX, gR, gI = X.cpu().numpy(), ranks.cpu().numpy(), ind.cpu().numpy()
        stable = dep < 0
        np.testing.assert_array_equal(gR[stable], oR[stable])
        # trajectories: every row's decision, as integers (unstable instances: the prefix
        # the oracle resolves)
        for b in range(B):
            f, fo = gI[ro[b]:ro[b + 1]], oI[ro[b]:ro[b + 1]]
            n_cmp = len(f) if dep[b] < 0 else int(dep[b])
            bad_rows = np.flatnonzero(f[:n_cmp] != fo[:n_cmp])
            assert bad_rows.size == 0, (mode, b, bad_rows[:10])
        worst = 0.0
        for b in np.flatnonzero(stable):
            e = checks.rel_err(gX[xo[b]:xo[b + 1]], oX[xo[b]:xo[b + 1]])
            if e > tol:  # FP64 only: allow for the instance's conditioning (Section 4.2)
                assert mode == rg.RG_FP64, (b, e)
                tb = kappa_tol(make_stream(b).A, tol)
                assert e <= tb, (b, e, tb)
            worst = max(worst, e)
        report[mode] = worst
    return report


def test_uneven_batch_all_4096_instances():
    n3, m3, r3 = inputs.uneven_batch_shapes()
    shapes = [(int(a), int(b), int(c)) for a, b, c in zip(n3, m3, r3)]

    def make(b):
        return inputs.factor_stream(shapes[b][0], shapes[b][1], shapes[b][2], 1e-4,
                                    inputs.rng_for(3, b))

    A, Y, ro, eo, xo, m, oX, oR, oI = build_full_batch(make, shapes)
    dep = oracle_departures(oI, ro, r3)
    unstable = np.flatnonzero(dep >= 0)
    print("instances where the oracle leaves the generator's rank growth:", unstable.tolist(),
          "at rows", dep[unstable].tolist())
    # as measured (the oracle is built without FMA contraction: the same set on every host)
    assert unstable.tolist() == [267, 1576, 1588, 2110, 2849, 3371, 3628]
    np.testing.assert_array_equal(oR[dep < 0], r3[dep < 0])
    rep = check_full_batch(A, Y, ro, eo, xo, m, oX, oR, oI, make, dep)
    print("worst rel err vs oracle: FP64 %.3e, mixed %.3e" % (rep[rg.RG_FP64], rep[rg.RG_MIXED]))


def test_uniform_batch_all_1024_instances():
    shapes = [(2048, 256, 32)] * 1024

    def make(b):
        return inputs.factor_stream(2048, 256, 32, 1e-3, inputs.rng_for(4, b))

    A, Y, ro, eo, xo, m, oX, oR, oI = build_full_batch(make, shapes)
    assert (oR == 32).all()
    dep = oracle_departures(oI, ro, np.full(1024, 32))
    assert (dep < 0).all()
    rep = check_full_batch(A, Y, ro, eo, xo, m, oX, oR, oI, make, dep)
    print("worst rel err vs oracle: FP64 %.3e, mixed %.3e" % (rep[rg.RG_FP64], rep[rg.RG_MIXED]))
