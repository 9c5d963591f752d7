"""Pins of the oracle's reconstruction losses and K-tensor score (Sec. 6, Sec. 6.1)."""
import itertools

import numpy as np
import pytest

from oracle import gcp


def test_exact_sparse_loss_gaussian_and_poisson_closed_forms():
    """Exact loss over every entry of a sparse slice, against closed forms that never build the
    full tensor: Gaussian sum (x - m)^2 = ||X||^2 - 2 <X, M> + s'(*_k A_k'A_k)s; Poisson
    sum m - x log(m + eps) = s'(prod_k A_k' 1) - sum_nnz x log(m + eps)."""
    rng = np.random.default_rng(1)
    dims, R = (6, 5, 4), 3
    A = [rng.random((n, R)) + 0.1 for n in dims]
    s = rng.random(R) + 0.5
    lin = rng.choice(int(np.prod(dims)), 25, replace=False)
    idx = np.stack(np.unravel_index(lin, dims), axis=1)
    val = rng.integers(1, 4, 25).astype(float)
    X = gcp.coo_to_dense(idx, val, dims)
    m = gcp.kruskal_value(s, A, idx)
    Fg, n2 = gcp.exact_slice_loss(X, s, A, "gaussian")
    Gam = gcp.hadamard_gram(A, A)
    assert Fg == pytest.approx((val ** 2).sum() - 2 * (val * m).sum() + s @ Gam @ s, rel=1e-12)
    assert n2 == pytest.approx((val ** 2).sum(), rel=1e-15)
    Fp, _ = gcp.exact_slice_loss(X, s, A, "poisson")
    colsum = np.prod([a.sum(axis=0) for a in A], axis=0)
    assert Fp == pytest.approx(s @ colsum - (val * np.log(m + 1e-10)).sum(), rel=1e-12)


def test_sampled_loss_is_unbiased_for_the_exact_loss():
    """E[sampled numerator] = exact numerator (Alg. 5 weights eta/p, zeta/q): the mean over seeds is
    within 5 standard errors."""
    rng = np.random.default_rng(2)
    dims, R = (8, 7, 6), 2
    A = [rng.random((n, R)) for n in dims]
    s = rng.random(R) + 0.5
    lin = rng.choice(int(np.prod(dims)), 40, replace=False)
    idx = np.stack(np.unravel_index(lin, dims), axis=1)
    val = np.ones(40)
    F, _ = gcp.exact_slice_loss(gcp.coo_to_dense(idx, val, dims), s, A, "bernoulli_logit")
    est = [gcp.sampled_slice_loss(idx, val, dims, s, A, "bernoulli_logit", 10, 10, seed, 1)[0] for seed in range(2000)]
    assert abs(np.mean(est) - F) < 5 * np.std(est) / np.sqrt(len(est))


def test_congruence_of_a_ktensor_with_a_permuted_rescaled_copy_is_one():
    rng = np.random.default_rng(3)
    A = [rng.standard_normal((n, 5)) for n in (7, 6, 4)]
    perm = [3, 0, 4, 1, 2]
    scales = rng.random(5) + 0.5
    signs = [np.where(rng.random(5) < 0.5, -1.0, 1.0) for _ in A]
    B = [a[:, perm] * scales * sg for a, sg in zip(A, signs)]
    score, match = gcp.kruskal_score(A, B)
    assert score == pytest.approx(1.0, abs=1e-13)
    assert [perm[c] for c in match] == list(range(5))   # b_c is a_{perm[c]}


def test_best_matching_equals_the_assignment_solution_and_greedy_is_not_better():
    """R <= 8: the brute-force best matching equals scipy's linear_sum_assignment on Q (maximise);
    for larger R the greedy matching is a valid permutation scoring at most the optimum."""
    from scipy.optimize import linear_sum_assignment
    rng = np.random.default_rng(4)
    for R in (2, 5, 8):
        A = [rng.standard_normal((n, R)) for n in (6, 5, 7)]
        B = [rng.standard_normal((n, R)) for n in (6, 5, 7)]
        Q = gcp.congruence_matrix(A, B)
        r, c = linear_sum_assignment(-Q)
        score, perm = gcp.kruskal_score(A, B)
        assert score == pytest.approx(Q[r, c].sum() / R, rel=1e-13)
    R = 12
    A = [rng.standard_normal((n, R)) for n in (9, 8)]
    B = [rng.standard_normal((n, R)) for n in (9, 8)]
    Q = gcp.congruence_matrix(A, B)
    score, perm = gcp.kruskal_score(A, B)
    assert sorted(perm) == list(range(R))
    assert score == pytest.approx(Q[np.arange(R), perm].mean(), rel=1e-13)
    r, c = linear_sum_assignment(-Q)
    assert score <= Q[r, c].mean() + 1e-13


def test_congruence_matrix_hand_example():
    """Two 2-way rank-2 K-tensors with known cosines: A = identity columns, B columns at 60 degrees."""
    A = [np.eye(2), np.eye(2)]
    B = [np.array([[1.0, np.cos(np.pi / 3)], [0.0, np.sin(np.pi / 3)]]), np.eye(2)]
    Q = gcp.congruence_matrix(A, B)
    np.testing.assert_allclose(Q, [[1.0, 0.0], [0.0, np.sin(np.pi / 3)]], atol=1e-15)
    assert gcp.kruskal_score(A, B)[0] == pytest.approx((1 + np.sin(np.pi / 3)) / 2, rel=1e-15)
