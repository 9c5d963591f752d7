"""Pins of the oracle's stored-slice history variant (Sec. 4.1, eq. gcp_stream_problem_1)."""
import numpy as np
import pytest

from oracle import gcp, solver


def explicit_objective(X, s, A, hist, P):
    """sum_i f(x_i, m_i) + sum_h w_h sum_i f(x_ih, m_ih) + lambda/2 sum ||A_k||^2 with every model
    built as an explicit outer-product sum."""
    F = float(gcp.loss_f(P.loss, X, gcp.kruskal_full_bruteforce(s, A)).sum())
    for Xh, sh, wh in hist:
        F += wh * float(gcp.loss_f(P.loss, Xh, gcp.kruskal_full_bruteforce(sh, A)).sum())
    return F + 0.5 * P.lam * sum(float((a ** 2).sum()) for a in A)


@pytest.mark.parametrize("loss", ["gaussian", "poisson", "bernoulli_logit"])
def test_stored_history_gradient_matches_finite_differences(loss):
    rng = np.random.default_rng(5)
    dims, R = (4, 3, 5), 2
    A = [rng.random((n, R)) + 0.2 for n in dims]
    s = rng.random(R) + 0.5
    X = rng.poisson(1.0, dims).astype(float) if loss != "gaussian" else rng.standard_normal(dims)
    if loss == "bernoulli_logit":
        X = (X > 0).astype(float)
    hist = [(rng.poisson(1.0, dims).astype(float), rng.random(R) + 0.5, w) for w in (0.7, 1.3)]
    P = solver.Params(dims=dims, rank=R, loss=loss, lam=0.05, kappa_f=1, tau_f=1)
    Xs = solver.Slice(dims=dims, X=X)
    hX = [solver.Slice(dims=dims, X=h[0]) for h in hist]
    G = solver.factor_gradient(Xs, A, s, None, [], [], P, 1, 0)
    H = solver.stored_history_gradient(A, hX, [1, 2], [h[1] for h in hist], [h[2] for h in hist], P, 3, 0)
    step = 1e-6
    for k in range(len(A)):
        for idx in np.ndindex(*A[k].shape):
            Ap = [a.copy() for a in A]
            Am = [a.copy() for a in A]
            Ap[k][idx] += step
            Am[k][idx] -= step
            fd = (explicit_objective(X, s, Ap, hist, P) - explicit_objective(X, s, Am, hist, P)) / (2 * step)
            assert G[k][idx] + H[k][idx] == pytest.approx(fd, rel=1e-6, abs=1e-6)


def test_stored_history_special_cases():
    """w = 0 leaves the plain gradient; a stored slice equal to the current one with the same
    weights scales the loss gradient by (1 + w)."""
    rng = np.random.default_rng(6)
    dims, R = (5, 4, 3), 3
    A = [rng.standard_normal((n, R)) for n in dims]
    s = rng.random(R) + 0.5
    X = rng.standard_normal(dims)
    P = solver.Params(dims=dims, rank=R, loss="gaussian")
    Xs = solver.Slice(dims=dims, X=X)
    G = solver.factor_gradient(Xs, A, s, None, [], [], P, 2, 0)
    H0 = solver.stored_history_gradient(A, [Xs], [1], [s], [0.0], P, 2, 0)
    H = solver.stored_history_gradient(A, [Xs], [1], [s], [0.4], P, 2, 0)
    for k in range(3):
        assert np.array_equal(H0[k], np.zeros_like(A[k]))
        np.testing.assert_allclose(G[k] + H[k], 1.4 * G[k], rtol=1e-12, atol=1e-12)
    Fh = solver.stored_history_objective(A, [Xs], [1], [s], [0.4], P, 2)
    assert Fh == pytest.approx(0.4 * gcp.dense_objective(X, s, A, "gaussian"), rel=1e-13)


def test_stored_history_stream_decreases_the_objective_and_keeps_the_slices():
    rng = np.random.default_rng(7)
    dims, R = (8, 7, 6), 2
    At = [rng.random((n, R)) + 0.1 for n in dims]
    P = solver.Params(dims=dims, rank=R, loss="gaussian", H=2, w=1.0, theta=0.9, kappa_w=2, tau_w=10,
                      alpha_w=0.05, kappa_f=2, tau_f=10, alpha_f=0.01, history="slices", seed=3)
    og = solver.OnlineGCP(P, [a + 0.1 * rng.standard_normal(a.shape) for a in At])
    slices = [solver.Slice(dims=dims, X=gcp.kruskal_full_bruteforce(rng.random(R) + 0.5, At)) for _ in range(4)]
    for X in slices:
        n0 = len(og.log_f)
        og.step(X)
        for e in og.log_f[n0:]:
            if e["passed"]:
                assert e["F_new"] <= e["F_old"]
    assert len(og.hist_X) == 2 and all(og.hist_X[j] is slices[og.hist_t[j] - 1] for j in range(2))
