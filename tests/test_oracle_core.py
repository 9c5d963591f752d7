"""Pins of the oracle's core arithmetic against closed forms, brute force and finite differences.

Each test checks the oracle against something other than itself: a published
test vector, an explicit outer-product sum, the Gaussian normal equations,
central differences of the objective, or a probabilistic identity.
"""
import os

import numpy as np
import pytest

from oracle import gcp
from oracle.philox import philox4x32_10, bounded

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_factors(rng, dims, R, nonneg=False):
    if nonneg:
        return [rng.random((n, R)) + 0.1 for n in dims]
    return [rng.standard_normal((n, R)) for n in dims]


# ----------------------------------------------------------------------------- Philox
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox4x32_10([v[0:4]], (v[4], v[5]))[0]
        assert [int(x) for x in out] == v[6:10]


def test_bounded_integer_range_and_extremes():
    u = np.array([0, 1, 2**31, 2**32 - 1], np.uint64)
    for n in (1, 7, 1000, 2**31 - 1):
        b = bounded(u, n)
        assert b[0] == 0 and b[-1] == n - 1
        assert np.all((b >= 0) & (b < n))
    # multiply-shift of uniform words is uniform up to n / 2^32
    ctr = np.stack([np.arange(200000), np.zeros(200000), np.zeros(200000), np.zeros(200000)], 1)
    w = philox4x32_10(ctr, (123, 456))[:, 0]
    counts = np.bincount(bounded(w, 10), minlength=10)
    chi2 = ((counts - 20000.0) ** 2 / 20000.0).sum()
    assert chi2 < 35.0   # 9 dof, p ~ 1e-4


# ----------------------------------------------------------------------------- model
@pytest.mark.parametrize("dims", [(4, 5), (3, 4, 5), (2, 3, 2, 4)])
def test_kruskal_value_matches_outer_product_sum(dims):
    rng = np.random.default_rng(1)
    R = 3
    A = _rand_factors(rng, dims, R)
    s = rng.standard_normal(R)
    M = np.zeros(dims)
    for idx in np.ndindex(*dims):        # explicit sum over j of s_j prod_k a^(k)_{i_k j}
        M[idx] = sum(s[j] * np.prod([A[k][idx[k], j] for k in range(len(dims))]) for j in range(R))
    coords = np.array(list(np.ndindex(*dims)))
    np.testing.assert_allclose(gcp.kruskal_value(s, A, coords), M.reshape(-1), rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(gcp.kruskal_full_bruteforce(s, A), M, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(gcp.dense_model(s, A), M, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dims", [(4, 5), (3, 4, 5), (2, 3, 2, 4)])
def test_unfold_khatri_rao_conventions(dims):
    """M_(k) = A^(k) diag(s) Z_k' and vec(M) = Z s (Kolda & Bader identities)."""
    rng = np.random.default_rng(2)
    R = 3
    A = _rand_factors(rng, dims, R)
    s = rng.standard_normal(R)
    M = gcp.kruskal_full_bruteforce(s, A)
    for k in range(len(dims)):
        np.testing.assert_allclose(gcp.unfold(M, k), A[k] @ np.diag(s) @ gcp.Zk(A, k).T, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(gcp.fold(gcp.unfold(M, k), k, list(dims)), M)
    np.testing.assert_allclose(gcp.vec(M), gcp.Zall(A) @ s, rtol=1e-12, atol=1e-12)


# ----------------------------------------------------------------------------- losses
@pytest.mark.parametrize("loss", gcp.LOSSES)
def test_loss_derivative_matches_central_difference(loss):
    rng = np.random.default_rng(3)
    x = rng.integers(0, 3, 50).astype(float) if loss != "gaussian" else rng.standard_normal(50)
    if loss.startswith("bernoulli"):
        x = np.minimum(x, 1.0)
    m = rng.random(50) * 3 + 0.2
    h = 1e-6
    fd = (gcp.loss_f(loss, x, m + h) - gcp.loss_f(loss, x, m - h)) / (2 * h)
    np.testing.assert_allclose(gcp.loss_dfdm(loss, x, m), fd, rtol=1e-7, atol=1e-8)


def test_loss_closed_forms():
    # Gaussian (x - m)^2, Poisson m - x log m, odds log(m+1) - x log m, logit log(1+e^m) - x m
    assert gcp.loss_f("gaussian", 3.0, 1.0, 0.0) == 4.0
    assert abs(gcp.loss_f("poisson", 2.0, np.e, 0.0) - (np.e - 2.0)) < 1e-15
    assert abs(gcp.loss_f("bernoulli_odds", 1.0, 1.0, 0.0) - np.log(2.0)) < 1e-15
    assert abs(gcp.loss_f("bernoulli_logit", 0.0, 0.0) - np.log(2.0)) < 1e-15
    assert abs(gcp.loss_f("bernoulli_logit", 1.0, 800.0) - 0.0) < 1e-12    # no overflow
    assert abs(gcp.loss_dfdm("bernoulli_logit", 1.0, 0.0) + 0.5) < 1e-15
    assert gcp.default_lower_bound("poisson") == 0.0
    assert gcp.default_lower_bound("gaussian") == -np.inf


# ----------------------------------------------------------------------------- dense gradient
@pytest.mark.parametrize("dims", [(5, 6), (4, 5, 3), (3, 2, 4, 3)])
def test_dense_gaussian_gradient_matches_normal_equations(dims):
    """Gaussian: dF/dA^(k) = 2(A^(k) diag(s) Z_k'Z_k diag(s) - X_(k) Z_k diag(s)),
    dF/ds = 2(Z'Z s - Z' vec X)  (least-squares CP gradient, Sec. 5 with the sign of eq. gcp_grad_A)."""
    rng = np.random.default_rng(4)
    R = 3
    A = _rand_factors(rng, dims, R)
    s = rng.standard_normal(R)
    X = rng.standard_normal(dims)
    G, gs, F = gcp.dense_gradient(X, s, A, "gaussian")
    for k in range(len(dims)):
        Z = gcp.Zk(A, k)
        ref = 2.0 * (A[k] @ np.diag(s) @ Z.T @ Z @ np.diag(s) - gcp.unfold(X, k) @ Z @ np.diag(s))
        np.testing.assert_allclose(G[k], ref, rtol=1e-11, atol=1e-11)
    Z = gcp.Zall(A)
    np.testing.assert_allclose(gs, 2.0 * (Z.T @ Z @ s - Z.T @ gcp.vec(X)), rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(F, ((X - gcp.kruskal_full_bruteforce(s, A)) ** 2).sum(), rtol=1e-12)
    _, gs_explicit, _ = gcp.dense_gradient(X, s, A, "gaussian", explicit_Z=True)
    np.testing.assert_allclose(gs, gs_explicit, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("loss", gcp.LOSSES)
@pytest.mark.parametrize("dims", [(3, 4), (3, 2, 4)])
def test_dense_gradient_matches_finite_differences(loss, dims):
    rng = np.random.default_rng(5)
    R = 2
    nonneg = loss in ("poisson", "bernoulli_odds")
    A = _rand_factors(rng, dims, R, nonneg)
    s = rng.random(R) + 0.5 if nonneg else rng.standard_normal(R)
    if loss == "gaussian":
        X = rng.standard_normal(dims)
    elif loss == "poisson":
        X = rng.poisson(2.0, dims).astype(float)
    else:
        X = (rng.random(dims) < 0.4).astype(float)
    G, gs, F = gcp.dense_gradient(X, s, A, loss)
    h = 1e-6
    for k in range(len(dims)):
        fd = np.zeros_like(A[k])
        for idx in np.ndindex(*A[k].shape):
            Ap = [a.copy() for a in A]; Ap[k][idx] += h
            Am = [a.copy() for a in A]; Am[k][idx] -= h
            fd[idx] = (gcp.dense_objective(X, s, Ap, loss) - gcp.dense_objective(X, s, Am, loss)) / (2 * h)
        np.testing.assert_allclose(G[k], fd, rtol=1e-6, atol=1e-6)
    fds = np.zeros(R)
    for j in range(R):
        sp = s.copy(); sp[j] += h
        sm = s.copy(); sm[j] -= h
        fds[j] = (gcp.dense_objective(X, sp, A, loss) - gcp.dense_objective(X, sm, A, loss)) / (2 * h)
    np.testing.assert_allclose(gs, fds, rtol=1e-6, atol=1e-6)


def test_noise_free_planted_gaussian_gradient_vanishes():
    """Gaussian GCP = CP: at the planted factors of a noise-free slice the gradient is zero."""
    rng = np.random.default_rng(6)
    A = _rand_factors(rng, (6, 5, 4), 3)
    s = rng.random(3) + 0.5
    X = gcp.kruskal_full_bruteforce(s, A)
    G, gs, F = gcp.dense_gradient(X, s, A, "gaussian")
    assert abs(F) < 1e-24
    assert max(np.abs(g).max() for g in G) < 1e-12 and np.abs(gs).max() < 1e-12
