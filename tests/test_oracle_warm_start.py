"""Pins of the oracle's warm start (static GCP-SGD on the first slices stacked as a (d+1)-way tensor,
Sec. 4.4 and Sec. 6) and of the OnlineSGD special case of OnlineGCP (Sec. 5)."""
import math

import numpy as np
import pytest

from oracle import gcp, solver

LOSSES = ["gaussian", "poisson", "bernoulli_odds", "bernoulli_logit"]


def stacked_case(rng, loss, dims=(5, 4), R=3, n=4):
    A = [rng.random((k, R)) + 0.1 for k in dims]
    S = rng.random((n, R)) + 0.2
    if loss == "gaussian":
        slices = [rng.standard_normal(dims) for _ in range(n)]
    else:
        slices = [(rng.random(dims) < 0.4).astype(float) * (1 + (loss == "poisson")) for _ in range(n)]
    return A, S, slices


@pytest.mark.parametrize("loss", LOSSES)
def test_stacked_gradient_equals_the_gradient_of_the_explicit_stacked_tensor(loss):
    """Slice by slice (G^(k) = sum_h Y_h(k) Z_k diag(S_h), g_{S_h} = Z' vec(Y_h)) against the
    oracle's (d+1)-way dense gradient of the stacked array X[i_1, .., i_d, h] with factors
    (A^(1), .., A^(d), S) and unit weights -- a different unfolding and Khatri-Rao product."""
    rng = np.random.default_rng(len(loss))
    A, S, slices = stacked_case(rng, loss)
    dims = tuple(a.shape[0] for a in A)
    P = solver.Params(dims=dims, rank=3, loss=loss)
    Xs = [solver.Slice(dims=dims, X=x) for x in slices]
    G, GS = solver.stacked_loss_gradient(Xs, A, S, P, draw=0)
    Gfull, _, Ffull = gcp.dense_gradient(np.stack(slices, axis=-1), np.ones(3), A + [S], loss)
    for k in range(len(A)):
        np.testing.assert_allclose(G[k], Gfull[k], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(GS, Gfull[-1], rtol=1e-12, atol=1e-12)
    assert solver.stacked_objective(Xs, A, S, P) == pytest.approx(Ffull, rel=1e-12)


def test_stacked_objective_regularises_every_factor_matrix():
    rng = np.random.default_rng(3)
    A, S, slices = stacked_case(rng, "gaussian")
    dims = tuple(a.shape[0] for a in A)
    Xs = [solver.Slice(dims=dims, X=x) for x in slices]
    P0 = solver.Params(dims=dims, rank=3, loss="gaussian")
    P1 = solver.Params(dims=dims, rank=3, loss="gaussian", lam=0.3)
    extra = 0.15 * (sum((a ** 2).sum() for a in A) + (S ** 2).sum())
    assert solver.stacked_objective(Xs, A, S, P1) == pytest.approx(solver.stacked_objective(Xs, A, S, P0) + extra,
                                                                   rel=1e-13)
    # explicit loss of the stacked model, entry by entry
    M = gcp.kruskal_full_bruteforce(np.ones(3), A + [S])
    F = sum(((slices[h] - M[..., h]) ** 2).sum() for h in range(len(slices)))
    assert solver.stacked_objective(Xs, A, S, P0) == pytest.approx(F, rel=1e-12)


def test_static_gcp_sgd_fits_a_planted_stacked_tensor():
    """Noise-free planted stacked tensor (Gaussian): the fit lowers the stacked objective by more
    than 10x from a perturbed start, and every accepted epoch does not increase it."""
    rng = np.random.default_rng(5)
    dims, R, n = (12, 10), 3, 6
    At = [rng.random((k, R)) + 0.2 for k in dims]
    St = rng.random((n, R)) + 0.5
    slices = [solver.Slice(dims=dims, X=gcp.kruskal_full_bruteforce(St[h], At)) for h in range(n)]
    A0 = [a + 0.3 * rng.standard_normal(a.shape) for a in At]
    S0 = np.ones((n, R))
    P = solver.Params(dims=dims, rank=R, loss="gaussian", kappa_f=8, tau_f=60, alpha_f=0.02)
    F0 = solver.stacked_objective(slices, A0, S0, P)
    log = []
    A, S, F = solver.static_gcp_sgd(slices, A0, S0, P, log=log)
    assert F < 0.1 * F0
    for e in log:
        if e["passed"]:
            assert e["F_new"] <= e["F_old"]
    assert F == pytest.approx(solver.stacked_objective(slices, A, S, P), rel=1e-12)


def test_warm_start_window_and_state():
    """After a warm start on n <= H slices the stream stands at t = n with the fitted factors as
    Abar, the window (1..n) holding the fitted rows S_h, and s = S_n."""
    rng = np.random.default_rng(6)
    dims, R, n = (6, 5), 2, 3
    slices = [solver.Slice(dims=dims, X=rng.standard_normal(dims)) for _ in range(n)]
    A0 = [rng.standard_normal((k, R)) for k in dims]
    P = solver.Params(dims=dims, rank=R, loss="gaussian", H=5, kappa_f=2, tau_f=4, alpha_f=0.01)
    og, S, F = solver.warm_start(slices, A0, np.ones((n, R)), P)
    A, S2, F2 = solver.static_gcp_sgd(slices, A0, np.ones((n, R)), P)
    assert og.t == n and og.hist_t == [1, 2, 3]
    for h in range(n):
        assert np.array_equal(og.hist_s[h], S[h])
    for a, b in zip(og.Abar, A):
        assert np.array_equal(a, b)
    assert np.array_equal(og.s, S[-1]) and F == F2


def test_online_sgd_special_case_first_step_closed_form():
    """OnlineGCP with the Gaussian loss, the least-squares temporal solve, the dense gradient, no
    history window and one factor iteration per slice (Sec. 5: the OnlineSGD special case).  Its
    first step is, in closed form: s = (A1'A1 * A2'A2)^-1 (A1' X A2 diagonal sums), then one
    ADAM step from zero moments, a <- a - alpha g / (|g| + eps / sqrt(1 - beta2)), with g the
    Gaussian gradient 2 (A^(k) diag(s) Gamma_k diag(s) - X_(k) A^(other) diag(s)), kept when it
    does not raise ||X - M||^2 (else the start is kept)."""
    rng = np.random.default_rng(7)
    I, J, R = 7, 6, 3
    A1, A2 = rng.standard_normal((I, R)), rng.standard_normal((J, R))
    X = rng.standard_normal((I, J))
    P = solver.Params(dims=(I, J), rank=R, loss="gaussian", temporal="lsq", H=0, kappa_f=1, tau_f=1,
                      alpha_f=0.05)
    og = solver.OnlineGCP(P, [A1, A2])
    out = og.step(solver.Slice(dims=(I, J), X=X))
    # closed form, written out with explicit sums
    Gam = (A1.T @ A1) * (A2.T @ A2)
    rhs = np.array([sum(A1[i, r] * X[i, j] * A2[j, r] for i in range(I) for j in range(J)) for r in range(R)])
    s = np.linalg.solve(Gam, rhs)
    np.testing.assert_allclose(out["s"], s, rtol=1e-10)
    D = np.diag(s)
    g1 = 2.0 * (A1 @ D @ (A2.T @ A2) @ D - X @ A2 @ D)
    g2 = 2.0 * (A2 @ D @ (A1.T @ A1) @ D - X.T @ A1 @ D)
    step = lambda a, g: a - P.alpha_f * g / (np.abs(g) + P.adam_eps / math.sqrt(1.0 - P.beta2))
    B1, B2 = step(A1, g1), step(A2, g2)
    F_old = ((X - A1 @ D @ A2.T) ** 2).sum()
    F_new = ((X - B1 @ D @ B2.T) ** 2).sum()
    E1, E2 = (B1, B2) if F_new <= F_old else (A1, A2)
    np.testing.assert_allclose(og.Abar[0], E1, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(og.Abar[1], E2, rtol=1e-10, atol=1e-12)
    assert out["F_f"] == pytest.approx(min(F_new, F_old), rel=1e-10)
    assert og.i == (1 if F_new <= F_old else 0)
