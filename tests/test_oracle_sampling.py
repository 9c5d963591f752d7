"""Pins of the oracle's stratified sampling (Alg. 5 / Alg. 6, Sec. 4.3).

The sampled gradient is pinned by (i) a per-sample brute-force sum for a fixed
sample list, (ii) unbiasedness against the exact dense gradient, and (iii)
distributional checks of the zero sampler.
"""
import numpy as np
import pytest

from oracle import gcp


def _tiny_sparse(rng, dims, density):
    X = (rng.random(dims) < density) * rng.integers(1, 4, dims)
    idx = np.argwhere(X != 0)
    rng.shuffle(idx)
    val = X[tuple(idx.T)].astype(float)
    return X.astype(float), idx, val


def test_zero_samples_are_zeros_and_in_range():
    rng = np.random.default_rng(10)
    dims = (7, 6, 5)
    X, idx, val = _tiny_sparse(rng, dims, 0.3)
    keys = np.sort(gcp.linear_keys(idx, dims))
    zc, att = gcp.zero_sample_coords(dims, 5000, 99, 3, 7, gcp.PURPOSE["grad_z"], keys, 64)
    assert np.all(zc >= 0) and np.all(zc < np.array(dims))
    assert np.all(X[tuple(zc.T)] == 0)
    assert att.min() == 0 and att.max() > 0          # some slots needed a retry at 30% density


def test_zero_sampler_is_uniform_over_zeros():
    rng = np.random.default_rng(11)
    dims = (4, 3, 2)
    X, idx, val = _tiny_sparse(rng, dims, 0.4)
    keys = np.sort(gcp.linear_keys(idx, dims))
    n = 60000
    zc, _ = gcp.zero_sample_coords(dims, n, 5, 1, 0, gcp.PURPOSE["grad_z"], keys, 200)
    zk = gcp.linear_keys(zc, dims)
    zeros = np.sort(gcp.linear_keys(np.argwhere(X == 0), dims))
    counts = np.array([(zk == z).sum() for z in zeros])
    assert counts.sum() == n
    e = n / len(zeros)
    chi2 = ((counts - e) ** 2 / e).sum()
    assert chi2 < len(zeros) + 6 * np.sqrt(2 * len(zeros))


def test_nonzero_sampler_is_uniform_over_entries():
    ids = gcp.nonzero_sample_ids(13, 130000, 77, 2, 0, gcp.PURPOSE["grad_nz"])
    counts = np.bincount(ids, minlength=13)
    chi2 = ((counts - 10000.0) ** 2 / 10000.0).sum()
    assert chi2 < 40.0


def test_sampling_limit_raises_for_a_full_slice():
    dims = (2, 2)
    idx = np.array(list(np.ndindex(*dims)))
    with pytest.raises(gcp.SamplingLimit):
        gcp.zero_sample_coords(dims, 3, 1, 1, 0, 1, np.sort(gcp.linear_keys(idx, dims)), 8)
    # with no zeros at all the stratified draw drops its zero stratum (q := 0)
    c, x, w = gcp.stratified_samples(idx, np.ones(4), dims, 5, 5, 1, 1, 0, 0, 1, 8)
    assert c.shape[0] == 5 and np.all(w == 4 / 5)


def test_sampled_gradient_equals_per_sample_sum():
    """Y~_(k) Z_k diag(s) over the merged sample tensor equals the plain per-sample sum."""
    rng = np.random.default_rng(12)
    dims = (5, 4, 3)
    R = 3
    X, idx, val = _tiny_sparse(rng, dims, 0.3)
    A = [rng.standard_normal((n, R)) for n in dims]
    s = rng.standard_normal(R)
    p, q = 40, 30
    G, gs, F = gcp.sampled_gradient(idx, val, dims, s, A, "gaussian", p, q, 4, 2, 9)
    coords, x, w = gcp.stratified_samples(idx, val, dims, p, q, 4, 2, 9, 0, 1)
    eta = idx.shape[0]
    zeta = np.prod(dims) - eta
    assert np.allclose(w[:p], eta / p) and np.allclose(w[p:], zeta / q)
    Gref = [np.zeros((n, R)) for n in dims]
    gsref = np.zeros(R)
    Fref = 0.0
    for c in range(p + q):                 # one sample at a time, no merging
        i = coords[c]
        m = sum(s[j] * A[0][i[0], j] * A[1][i[1], j] * A[2][i[2], j] for j in range(R))
        y = w[c] * 2.0 * (m - x[c])
        Fref += w[c] * (x[c] - m) ** 2
        for j in range(R):
            Gref[0][i[0], j] += y * s[j] * A[1][i[1], j] * A[2][i[2], j]
            Gref[1][i[1], j] += y * s[j] * A[0][i[0], j] * A[2][i[2], j]
            Gref[2][i[2], j] += y * s[j] * A[0][i[0], j] * A[1][i[1], j]
            gsref[j] += y * A[0][i[0], j] * A[1][i[1], j] * A[2][i[2], j]
    for k in range(3):
        np.testing.assert_allclose(G[k], Gref[k], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(gs, gsref, rtol=1e-12, atol=1e-12)
    assert abs(F - Fref) < 1e-10 * max(1.0, abs(Fref))


@pytest.mark.parametrize("loss", ["poisson", "bernoulli_logit"])
def test_sampled_gradient_and_objective_are_unbiased(loss):
    """E[Y~] = Y and E[F~] = F (Sec. 4.3): the mean over many draws matches the exact values."""
    rng = np.random.default_rng(13)
    dims = (4, 3, 3)
    R = 2
    X, idx, val = _tiny_sparse(rng, dims, 0.35)
    if loss == "bernoulli_logit":
        val = np.ones_like(val)
        X = (X != 0).astype(float)
    A = [rng.random((n, R)) + 0.2 for n in dims]
    s = rng.random(R) + 0.5
    Gex, gsex, Fex = gcp.dense_gradient(X, s, A, loss)
    ndraw, p, q = 3000, 6, 6
    acc = [np.zeros_like(g) for g in Gex]
    acc2 = [np.zeros_like(g) for g in Gex]
    accs, accs2 = np.zeros(R), np.zeros(R)
    Fs = []
    for dr in range(ndraw):
        G, gs, F = gcp.sampled_gradient(idx, val, dims, s, A, loss, p, q, 17, 5, dr)
        for k in range(3):
            acc[k] += G[k]
            acc2[k] += G[k] ** 2
        accs += gs
        accs2 += gs ** 2
        Fs.append(F)
    for k in range(3):
        mean = acc[k] / ndraw
        sd = np.sqrt(np.maximum(acc2[k] / ndraw - mean ** 2, 1e-30) / ndraw)
        assert np.all(np.abs(mean - Gex[k]) <= 5 * sd + 1e-12)
    mean = accs / ndraw
    sd = np.sqrt(np.maximum(accs2 / ndraw - mean ** 2, 1e-30) / ndraw)
    assert np.all(np.abs(mean - gsex) <= 5 * sd)
    Fs = np.array(Fs)
    assert abs(Fs.mean() - Fex) <= 5 * Fs.std() / np.sqrt(ndraw)


def test_counter_streams_are_distinct():
    """Different draws, purposes and time steps give different samples; equal inputs give equal samples."""
    a = gcp.nonzero_sample_ids(1000, 64, 5, 3, 0, 0)
    assert np.array_equal(a, gcp.nonzero_sample_ids(1000, 64, 5, 3, 0, 0))
    for other in [(5, 3, 1, 0), (5, 4, 0, 0), (5, 3, 0, 2), (6, 3, 0, 0)]:
        b = gcp.nonzero_sample_ids(1000, 64, other[0], other[1], other[2], other[3])
        assert not np.array_equal(a, b)
