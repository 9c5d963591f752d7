"""The seeded generators produce the shapes and distributions their recipes state."""
import numpy as np

import synthetic as S


def test_sparse_zipf_slice_is_unique_in_range_and_reproducible():
    cfg = S.workload("sparse_binary_zipf")
    dims = (300, 200, 100)
    idx, val = S.sparse_slice(cfg, 1, nnz=5000, dims=dims)
    assert idx.shape == (5000, 3) and idx.dtype == np.int32 and np.all(val == 1)
    assert np.all(idx >= 0) and np.all(idx < np.array(dims))
    key = (idx[:, 0].astype(np.int64) * dims[1] + idx[:, 1]) * dims[2] + idx[:, 2]
    assert np.unique(key).size == 5000
    idx2, _ = S.sparse_slice(cfg, 1, nnz=5000, dims=dims)
    assert np.array_equal(idx, idx2)
    idx3, _ = S.sparse_slice(cfg, 2, nnz=5000, dims=dims)
    assert not np.array_equal(idx, idx3)
    # heavy head: the most frequent row of each mode carries several percent of the nonzeros
    for k in range(3):
        assert np.bincount(idx[:, k]).max() > 0.03 * 5000


def test_dense_slices_have_the_stated_noise():
    cfg = S.workload("dense_gaussian_2way")
    X, s = S.dense_slice(cfg, 3)
    A = S.truth(cfg)
    M = np.einsum("ir,jr,r->ij", A[0], A[1], s)
    assert X.shape == (20, 30) and X.dtype == np.float64
    assert 0.07 < (X - M).std() < 0.13
    assert np.all((s >= 0.5) & (s <= 1.5))
    cfg = S.workload("dense_poisson_3way")
    X, s = S.dense_slice(cfg, 1)
    assert X.dtype == np.float32 and np.all(X == np.round(X)) and 0.5 < X.mean() < 1.5


def test_batched_shapes_follow_the_recipe():
    cfg = S.workload("batched_streams")
    sh = S.batched_stream_shapes(cfg)
    assert len(sh) == 64
    for s, (dims, rank, loss) in enumerate(sh):
        assert all(32 <= n <= 160 for n in dims) and rank in cfg["rank_choices"]
        assert loss == ("gaussian" if s % 2 == 0 else "poisson")
