"""GPU parity of the evaluation metrics of Sec. 6: the local / global reconstruction loss terms
(sgcp_slice_loss, sampled and exact, dense and sparse) and the K-tensor score of Sec. 6.1
(sgcp_kruskal_score), against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synthetic as S
from oracle import gcp

LOSSES = ["gaussian", "poisson", "bernoulli_odds", "bernoulli_logit"]


@pytest.fixture(scope="module")
def sg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2110_14514_gb300 as sg
    return sg


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def close(a, b, tol):
    return abs(a - b) <= tol * max(abs(b), 1.0)


def positive_case(rng, dims, R, loss):
    A = [(0.4 * rng.random((n, R)) + 0.05).astype(np.float32) for n in dims]
    s = (rng.random(R) + 0.5).astype(np.float32)
    if loss in ("gaussian", "bernoulli_logit"):
        A = [(0.5 * rng.standard_normal((n, R))).astype(np.float32) for n in dims]
    return A, s


@pytest.mark.parametrize("loss", LOSSES)
def test_dense_slice_loss_is_exact(sg, loss):
    dims, R = (40, 36, 30), 16
    rng = np.random.default_rng(1)
    A, s = positive_case(rng, dims, R, loss)
    X = rng.poisson(1.0, dims).astype(np.float32)
    if loss.startswith("bernoulli"):
        X = (X > 0).astype(np.float32)
    with sg.Context(sg.params(dims, R, loss), [dev(a) for a in A]) as ctx:
        F, n2 = ctx.slice_loss(dev(s), [dev(a) for a in A], X=dev(X))
    Fo, n2o = gcp.exact_slice_loss(X, s, A, loss)
    assert close(F, Fo, 1e-4) and close(n2, n2o, 1e-6), (F, Fo, n2, n2o)


def test_dense_2way_fp64_slice_loss(sg):
    cfg = S.workload("dense_gaussian_2way")
    A = S.init_factors(cfg)
    X, s = S.dense_slice(cfg, 1)
    with sg.Context(sg.params(cfg["dims"], cfg["rank"], "gaussian", precision=sg.PREC_F64), [dev(a) for a in A]) as ctx:
        F, n2 = ctx.slice_loss(dev(s), [dev(a) for a in A], X=dev(X))
    Fo, n2o = gcp.exact_slice_loss(X, s, A, "gaussian")
    assert close(F, Fo, 1e-12) and close(n2, n2o, 1e-12)


@pytest.mark.parametrize("loss", LOSSES)
@pytest.mark.parametrize("dims", [(60, 50, 40), (300, 70)])
def test_sparse_slice_loss_sampled_and_exact(sg, loss, dims):
    """Sampled: the objective sample set at time index t (the oracle's samples); exact: every entry
    of the slice, zeros included (the oracle builds the full tensor)."""
    R = 8
    rng = np.random.default_rng(len(dims) + LOSSES.index(loss))
    A, s = positive_case(rng, dims, R, loss)
    lin = rng.choice(int(np.prod(dims)), 3000, replace=False)
    idx = np.stack(np.unravel_index(lin, dims), axis=1).astype(np.int32)
    val = np.ones(3000, np.float32) if loss.startswith("bernoulli") else (1 + lin % 3).astype(np.float32)
    p = sg.params(dims, R, loss, p_obj=1500, q_obj=2500, seed=9)
    with sg.Context(p, [dev(a) for a in A]) as ctx:
        Fs, n2s = ctx.slice_loss(dev(s), [dev(a) for a in A], idx=dev(idx), vals=dev(val), t=4)
        Fe, n2e = ctx.slice_loss(dev(s), [dev(a) for a in A], idx=dev(idx), vals=dev(val), exact=True)
    Fso, n2o = gcp.sampled_slice_loss(idx, val, dims, s, A, loss, 1500, 2500, 9, 4)
    Feo, _ = gcp.exact_slice_loss(gcp.coo_to_dense(idx, val, dims), s, A, loss)
    assert close(Fs, Fso, 1e-4), (Fs, Fso)
    assert close(Fe, Feo, 1e-5), (Fe, Feo)
    assert close(n2s, n2o, 1e-6) and close(n2e, n2o, 1e-6)


@pytest.mark.parametrize("loss", ["gaussian", "poisson"])
def test_exact_loss_of_a_full_size_sparse_slice(sg, loss):
    """Every one of the 10000 x 5000 x 2000 = 1e11 entries of a 1e6-nonzero Zipf slice, R = 32,
    against closed forms that need only the nonzeros and the factor Grams: Gaussian
    ||X||^2 - 2 sum_nnz x m + s'(*_k A_k'A_k) s; Poisson s'(prod_k A_k'1) - sum_nnz x log(m + eps)."""
    cfg = S.workload("sparse_binary_zipf")
    idx, val = S.sparse_slice(cfg, 1)
    dims, R = cfg["dims"], cfg["rank"]
    rng = np.random.default_rng(12)
    A = [(0.02 * rng.random((n, R)) + 0.001).astype(np.float32) for n in dims]
    s = (rng.random(R) + 0.5).astype(np.float32)
    with sg.Context(sg.params(dims, R, loss), [dev(a) for a in A]) as ctx:
        F, n2 = ctx.slice_loss(dev(s), [dev(a) for a in A], idx=dev(idx), vals=dev(val), exact=True)
    A64 = [a.astype(np.float64) for a in A]
    m = gcp.kruskal_value(s.astype(np.float64), A64, idx)
    x = val.astype(np.float64)
    if loss == "gaussian":
        Fo = (x * x).sum() - 2 * (x * m).sum() + s @ gcp.hadamard_gram(A64, A64) @ s
    else:
        Fo = s @ np.prod([a.sum(axis=0) for a in A64], axis=0) - (x * np.log(m + 1e-10)).sum()
    assert close(F, Fo, 1e-4), (F, Fo)
    assert close(n2, (x * x).sum(), 1e-7)


@pytest.mark.parametrize("R,dtype", [(5, np.float32), (8, np.float64), (16, np.float32), (40, np.float64)])
def test_kruskal_score_matches_the_oracle(sg, R, dtype):
    """R <= 8: the best of all matchings; above: greedy.  A noisy, permuted, rescaled copy (score
    near 1, the permutation recovered) and an unrelated K-tensor."""
    rng = np.random.default_rng(R)
    dims = (50, 40, 30, 20)
    A = [rng.standard_normal((n, R)).astype(dtype) for n in dims]
    perm = rng.permutation(R)
    B = [(a[:, perm] * (rng.random(R) + 0.5) + 0.05 * rng.standard_normal(a.shape)).astype(dtype) for a in A]
    C = [rng.standard_normal((n, R)).astype(dtype) for n in dims]
    for other in (B, C):
        sc, pm = sg.kruskal_score([dev(a) for a in A], [dev(b) for b in other])
        so, po = gcp.kruskal_score(A, other)
        assert abs(sc - so) < 1e-9, (sc, so)
        assert pm == po
    sc, pm = sg.kruskal_score([dev(a) for a in A], [dev(b) for b in B])
    assert sc > 0.9 and [perm[c] for c in pm] == list(range(R))
