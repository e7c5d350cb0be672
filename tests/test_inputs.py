"""The seeded input recipe: each generator builds what the workload description states
(shapes, ranges, rank, noise level) and is reproducible from its seed alone."""
import numpy as np

from paper_2106_11594_gb300 import inputs


def test_factor_stream_matches_its_draws():
    """A = G1 G2 and Y = A x_true + eps, from the raw draws in the same order."""
    s = inputs.factor_stream(300, 40, 6, 1e-3, inputs.rng_for(9, 2))
    G1, G2, x, e = inputs.factor_stream_factors(300, 40, 6, 1e-3, inputs.rng_for(9, 2))
    np.testing.assert_array_equal(s.A, G1 @ G2)
    np.testing.assert_array_equal(s.Y, s.A @ x + e)
    assert np.linalg.matrix_rank(s.A) == s.rank == 6
    assert 0.8e-3 < np.std(e) < 1.2e-3  # noise standard deviation 1e-3


def test_workload_shapes_and_ranks():
    s1 = inputs.small_stream()
    assert s1.A.shape == (256, 64) and np.linalg.matrix_rank(s1.A) == 8
    s2 = inputs.large_stream(2048, 256, 32)  # the large-stream construction at a small size
    assert s2.A.shape == (2048, 256) and np.linalg.matrix_rank(s2.A) == 32
    # the first r rows grow the rank one per row
    assert np.linalg.matrix_rank(s2.A[:32]) == 32


def test_uneven_batch_shapes_follow_the_recipe():
    n, m, r = inputs.uneven_batch_shapes()
    assert len(n) == len(m) == len(r) == 4096
    assert m.min() >= 32 and m.max() <= 512
    assert (r >= 2).all() and (r <= np.maximum(2, m // 4)).all()
    assert (n >= m).all() and (n <= 8 * m).all()
    assert abs(m.mean() - 272) < 10  # U{32..512} has mean 272
    n2, m2, r2 = inputs.uneven_batch_shapes()
    np.testing.assert_array_equal(n, n2)  # reproducible
    # a subset draws exactly what the full batch draws for those instances
    sub = inputs.uneven_batch(4096, instances=[5, 77])
    assert [s_.A.shape for s_ in sub.streams] == [(int(n[5]), int(m[5])), (int(n[77]), int(m[77]))]
    again = inputs.uneven_batch(4096, instances=[77])
    np.testing.assert_array_equal(sub.streams[1].A, again.streams[0].A)


def test_uniform_batch_and_packing():
    b = inputs.uniform_batch(1024, instances=range(3))
    assert all(s_.A.shape == (2048, 256) and s_.rank == 32 for s_ in b.streams)
    Ap, Yp, ro, eo, xo = b.packed()
    assert list(ro) == [0, 2048, 4096, 6144] and list(eo) == [0, 2048 * 256, 2 * 2048 * 256, 3 * 2048 * 256]
    assert list(xo) == [0, 256, 512, 768]
    np.testing.assert_array_equal(Ap[eo[1]:eo[2]].reshape(2048, 256), b.streams[1].A)


def test_ill_conditioned_stream_recipe():
    s = inputs.ill_conditioned_stream(n=1024, m=128, r=32)
    assert s.A.shape == (1024, 128) and int(s.growth.sum()) == 32
    # the row space of every phase is spanned by the directions active in it: rows of
    # phase p lie in a subspace of dimension 4 (p + 1)
    per = 1024 // 8
    for p in range(8):
        sv = np.linalg.svd(s.A[:(p + 1) * per], compute_uv=False)
        assert (sv > sv[0] * 1e-9).sum() == 4 * (p + 1)
