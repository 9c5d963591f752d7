"""Pins of the oracle's history penalty, streaming gradient and solvers (Sec. 4, Alg. 1-4)."""
import math

import numpy as np
import pytest

from oracle import gcp, solver


def _setup(rng, dims=(4, 3, 5), R=3, H=3):
    A = [rng.standard_normal((n, R)) for n in dims]
    Abar = [a + 0.3 * rng.standard_normal(a.shape) for a in A]
    s_hist = [rng.standard_normal(R) for _ in range(H)]
    w_h = rng.random(H) + 0.5
    return A, Abar, s_hist, w_h


def test_history_objective_gram_form_matches_explicit_tensors():
    rng = np.random.default_rng(20)
    for dims in [(4, 5), (4, 3, 5), (2, 3, 2, 3)]:
        A, Abar, s_hist, w_h = _setup(rng, dims)
        bf = gcp.history_objective_bruteforce(s_hist, w_h, A, Abar)
        assert bf > 0
        assert abs(gcp.history_objective(s_hist, w_h, A, Abar) - bf) < 1e-10 * bf


def test_history_terms_vanish_when_factors_are_unchanged():
    rng = np.random.default_rng(21)
    A, _, s_hist, w_h = _setup(rng)
    assert abs(gcp.history_objective_bruteforce(s_hist, w_h, A, A)) == 0.0
    for k in range(3):
        assert np.abs(gcp.history_gradient(A, A, s_hist, w_h, k)).max() < 1e-12


def test_history_gradient_matches_finite_differences():
    """eq. spatial_gcp_grad history term = derivative of 1/2 sum_h w_h ||Mbar_h - M_h||^2."""
    rng = np.random.default_rng(22)
    A, Abar, s_hist, w_h = _setup(rng, dims=(3, 4, 2), R=2, H=2)
    h = 1e-6
    for k in range(3):
        g = gcp.history_gradient(A, Abar, s_hist, w_h, k)
        ge = gcp.history_gradient(A, Abar, s_hist, w_h, k, explicit_Z=True)
        np.testing.assert_allclose(g, ge, rtol=1e-12, atol=1e-12)
        fd = np.zeros_like(A[k])
        for idx in np.ndindex(*A[k].shape):
            Ap = [a.copy() for a in A]; Ap[k][idx] += h
            Am = [a.copy() for a in A]; Am[k][idx] -= h
            fd[idx] = (gcp.history_objective_bruteforce(s_hist, w_h, Ap, Abar)
                       - gcp.history_objective_bruteforce(s_hist, w_h, Am, Abar)) / (2 * h)
        np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-7)


def test_full_streaming_gradient_matches_finite_differences():
    """Factor gradient of eq. gcp_stream_objective (loss + lambda + history) on a dense slice."""
    rng = np.random.default_rng(23)
    dims, R = (3, 4, 2), 2
    A, Abar, s_hist, w_h = _setup(rng, dims, R, H=2)
    s = rng.standard_normal(R)
    X = rng.standard_normal(dims)
    P = solver.Params(dims=dims, rank=R, loss="gaussian", lam=0.3)
    Xs = solver.Slice(dims=dims, X=X)
    G = solver.factor_gradient(Xs, A, s, Abar, s_hist, w_h, P, 1, 0)
    h = 1e-6
    for k in range(3):
        fd = np.zeros_like(A[k])
        for idx in np.ndindex(*A[k].shape):
            Ap = [a.copy() for a in A]; Ap[k][idx] += h
            Am = [a.copy() for a in A]; Am[k][idx] -= h
            fd[idx] = (solver.full_objective(Xs, Ap, s, Abar, s_hist, w_h, P)
                       - solver.full_objective(Xs, Am, s, Abar, s_hist, w_h, P)) / (2 * h)
        np.testing.assert_allclose(G[k], fd, rtol=1e-6, atol=1e-6)


def test_history_weights_are_exponential():
    np.testing.assert_allclose(gcp.history_weights([1, 3, 4], 5, 2.0, 0.5), [2 * 0.5 ** 4, 2 * 0.5 ** 2, 2 * 0.5])


# ----------------------------------------------------------------------------- ADAM (Alg. 2)
def test_adam_steps_have_length_alpha_for_a_constant_gradient():
    """With a constant gradient g the bias-corrected ADAM step is alpha * sign(g) at every i
    (up to epsilon); an off-by-one in the bias exponent breaks this at i = 0, 1."""
    ad = solver.Adam(0.01, 0.9, 0.999, 1e-12, -np.inf, 0.1)
    a = np.array([1.0, -2.0])
    ad.init(a)
    g = np.array([3.0, -0.5])
    for i in range(5):
        a_new = ad.step(a, g, i)
        np.testing.assert_allclose(a - a_new, 0.01 * np.sign(g), rtol=1e-9)
        a = a_new


def test_adam_rollback_restores_checkpoint_and_decays_alpha():
    ad = solver.Adam(0.5, 0.9, 0.999, 1e-8, 0.0, 0.1)
    a0 = np.array([1.0, 2.0])
    ad.init(a0)
    a1 = ad.step(a0, np.array([1.0, -1.0]), 0)
    a1 = ad.update(a1, True)
    u1, v1 = ad.u.copy(), ad.v.copy()
    a2 = ad.step(a1, np.array([100.0, 100.0]), 1)
    assert np.all(a2 >= 0.0)                           # lower bound l = 0
    back = ad.update(a2, False)
    assert np.array_equal(back, a1) and np.array_equal(ad.u, u1) and np.array_equal(ad.v, v1)
    assert ad.alpha == pytest.approx(0.05)
    # a first-epoch rejection returns the initial point, not zeros
    ad2 = solver.Adam(0.5, 0.9, 0.999, 1e-8, -np.inf, 0.1)
    ad2.init(a0)
    a = ad2.step(a0, np.array([1.0, 1.0]), 0)
    assert np.array_equal(ad2.update(a, False), a0)


# ----------------------------------------------------------------------------- reservoir (Alg. 1)
def test_reservoir_window_is_a_uniform_sample():
    """After step T every earlier step is in the window with probability H / T (Vitter)."""
    H, T, nseed = 4, 12, 3000
    counts = np.zeros(T + 1)
    for seed in range(nseed):
        win = []
        for t in range(1, T + 1):
            if len(win) < H:
                win.append(t)
            else:
                j = solver.reservoir_index(seed, t)
                assert 1 <= j <= t
                if j <= H:
                    win[j - 1] = t
        for h in win:
            counts[h] += 1
    p = H / T
    sd = math.sqrt(nseed * p * (1 - p))
    assert np.all(np.abs(counts[1:] - nseed * p) < 5 * sd)


# ----------------------------------------------------------------------------- solvers
def test_lsq_temporal_recovers_planted_weights():
    rng = np.random.default_rng(30)
    dims, R = (6, 5, 4), 3
    A = [rng.standard_normal((n, R)) for n in dims]
    s = rng.random(R) + 0.5
    X = gcp.kruskal_full_bruteforce(s, A)
    P = solver.Params(dims=dims, rank=R, loss="gaussian")
    np.testing.assert_allclose(solver.lsq_temporal(solver.Slice(dims=dims, X=X), A, P), s, rtol=1e-10)
    idx = np.argwhere(np.ones(dims))
    Xs = solver.Slice(dims=dims, idx=idx, val=X[tuple(idx.T)])
    np.testing.assert_allclose(solver.lsq_temporal(Xs, A, P), s, rtol=1e-10)


def test_lsq_temporal_with_ridge_minimises_the_penalised_residual():
    """mu > 0: the solve returns the minimiser of ||x - Z s||^2 + (mu / 2) ||s||^2, checked against
    a least-squares solve of the augmented system [Z; sqrt(mu / 2) I] s = [x; 0] with Z built from
    explicit rank-one tensors."""
    rng = np.random.default_rng(35)
    dims, R, mu = (5, 4, 6), 3, 0.7
    A = [rng.standard_normal((n, R)) for n in dims]
    X = rng.standard_normal(dims)
    P = solver.Params(dims=dims, rank=R, loss="gaussian", mu=mu)
    s = solver.lsq_temporal(solver.Slice(dims=dims, X=X), A, P)
    Z = np.stack([np.einsum("i,j,k->ijk", A[0][:, r], A[1][:, r], A[2][:, r]).ravel() for r in range(R)], axis=1)
    Zaug = np.vstack([Z, np.sqrt(mu / 2) * np.eye(R)])
    xaug = np.concatenate([X.ravel(), np.zeros(R)])
    ref = np.linalg.lstsq(Zaug, xaug, rcond=None)[0]
    np.testing.assert_allclose(s, ref, rtol=1e-10, atol=1e-12)


def test_temporal_and_factor_solvers_decrease_the_objective():
    rng = np.random.default_rng(31)
    dims, R = (6, 5, 4), 2
    A_true = [rng.random((n, R)) + 0.2 for n in dims]
    s_true = rng.random(R) + 0.5
    X = rng.poisson(gcp.kruskal_full_bruteforce(s_true, A_true)).astype(float)
    P = solver.Params(dims=dims, rank=R, loss="poisson", kappa_w=4, tau_w=20, alpha_w=0.05,
                      kappa_f=3, tau_f=20, alpha_f=0.01)
    Xs = solver.Slice(dims=dims, X=X)
    A0 = [a + 0.05 for a in A_true]
    log = []
    s, Fw = solver.wght_gcp_sgd(Xs, A0, P, 1, log=log)
    F_start = solver.estimate_objective(Xs, A0, np.zeros(R), None, [], [], 0.0, 0.0, P, 1, True)
    assert Fw < F_start
    accepted = [e["F_new"] for e in log if e["passed"]]
    assert all(b <= a for a, b in zip(accepted, accepted[1:]))
    ad = solver.Adam(P.alpha_f, P.beta1, P.beta2, P.adam_eps, 0.0, P.alpha_decay)
    ad.init(solver._flat(A0))
    log = []
    A1, i, Ff = solver.fac_gcp_sgd(Xs, A0, s, A0, [], [], P, 1, 0, ad, log=log)
    F0 = solver.estimate_objective(Xs, A0, s, A0, [], [], 0.0, 0.0, P, 1, False)
    assert Ff <= F0 and i == sum(P.tau_f for e in log if e["passed"])


def test_teacher_forced_rejection_restores_the_factors():
    rng = np.random.default_rng(32)
    dims, R = (4, 3, 3), 2
    A0 = [rng.standard_normal((n, R)) for n in dims]
    X = rng.standard_normal(dims)
    P = solver.Params(dims=dims, rank=R, loss="gaussian", kappa_f=2, tau_f=5, alpha_f=0.1)
    Xs = solver.Slice(dims=dims, X=X)
    ad = solver.Adam(P.alpha_f, P.beta1, P.beta2, P.adam_eps, -np.inf, P.alpha_decay)
    ad.init(solver._flat(A0))
    A1, i, _ = solver.fac_gcp_sgd(Xs, A0, np.ones(R), A0, [], [], P, 1, 0, ad,
                                  decisions=iter([False, False]))
    assert i == 0
    for a, b in zip(A1, A0):
        assert np.array_equal(a, b)


def test_temporal_solver_rejection_restores_s_F_and_the_iteration_count():
    """Alg. 3 rejection branch (restore s, F <- F_old, i <- i - tau_w, decay alpha), pinned by two
    invariants on a dense Gaussian slice (exact gradient, so the draw counter plays no part):
    (1) two rejected epochs return the starting point s = 0 and the objective there, which for the
        Gaussian loss is sum x^2 in closed form;
    (2) a rejected epoch followed by an accepted one equals a single epoch run with the decayed
        rate from scratch.  That holds only if the rejection restored s and the moments and also
        rolled i back: with i left at tau_w the second epoch's bias correction would use
        1 - beta^(tau_w + j + 1) instead of 1 - beta^(j + 1)."""
    rng = np.random.default_rng(33)
    dims, R = (5, 4, 3), 3
    A = [rng.standard_normal((n, R)) for n in dims]
    X = rng.standard_normal(dims)
    Xs = solver.Slice(dims=dims, X=X)
    kw = dict(dims=dims, rank=R, loss="gaussian", tau_w=7, alpha_w=0.05, alpha_decay=0.1)
    P = solver.Params(kappa_w=2, **kw)
    log = []
    s, F = solver.wght_gcp_sgd(Xs, A, P, 1, decisions=iter([False, False]), log=log)
    assert np.array_equal(s, np.zeros(R))
    assert F == pytest.approx(float((X ** 2).sum()), rel=1e-14)
    assert log[1]["F_old"] == log[0]["F_old"]          # the second epoch starts from the restored F
    s2, F2 = solver.wght_gcp_sgd(Xs, A, P, 1, decisions=iter([False, True]))
    P1 = solver.Params(kappa_w=1, **dict(kw, alpha_w=0.05 * 0.1))
    s1, F1 = solver.wght_gcp_sgd(Xs, A, P1, 1, decisions=iter([True]))
    assert np.allclose(s2, s1, rtol=1e-13, atol=0.0) and F2 == pytest.approx(F1, rel=1e-13)
    # and the rolled-back counter matters: the un-decayed single epoch is a different point
    s3, _ = solver.wght_gcp_sgd(Xs, A, solver.Params(kappa_w=1, **kw), 1, decisions=iter([True]))
    assert not np.allclose(s3, s1)


def test_lbfgs_two_loop_equals_the_explicit_inverse_bfgs_update():
    """The two-loop recursion returns H g for the matrix built by the inverse BFGS update
    H <- (I - rho s y') H (I - rho y s') + rho s s' (Nocedal & Wright eq. 6.17), applied to the
    pairs oldest first from H_0 = gamma I with gamma = s'y / y'y of the newest pair."""
    rng = np.random.default_rng(8)
    n, m = 9, 5
    Q = rng.standard_normal((n, n))
    B = Q @ Q.T + n * np.eye(n)                     # SPD curvature, so every s'y > 0
    S = [rng.standard_normal(n) for _ in range(m)]
    Yv = [B @ sv for sv in S]
    g = rng.standard_normal(n)
    r = solver.lbfgs_direction(g, S, Yv)
    gamma = (S[-1] @ Yv[-1]) / (Yv[-1] @ Yv[-1])
    H = gamma * np.eye(n)
    for sv, yv in zip(S, Yv):
        rho = 1.0 / (yv @ sv)
        V = np.eye(n) - rho * np.outer(yv, sv)
        H = V.T @ H @ V + rho * np.outer(sv, sv)
    np.testing.assert_allclose(r, H @ g, rtol=1e-10, atol=1e-12)
    # with no pairs the direction is the scaled gradient; the secant equation holds for the newest pair
    np.testing.assert_allclose(solver.lbfgs_direction(g, [], []), g / np.linalg.norm(g), rtol=1e-14)
    np.testing.assert_allclose(solver.lbfgs_direction(Yv[-1], S, Yv), S[-1], rtol=1e-9, atol=1e-12)


def test_lbfgs_decreases_the_exact_objective():
    rng = np.random.default_rng(33)
    dims, R = (5, 4, 3), 2
    A_true = [rng.standard_normal((n, R)) for n in dims]
    s = np.array([1.0, 0.7])
    X = gcp.kruskal_full_bruteforce(s, A_true)
    A0 = [a + 0.2 * rng.standard_normal(a.shape) for a in A_true]
    P = solver.Params(dims=dims, rank=R, loss="gaussian", lbfgs_iters=30)
    Xs = solver.Slice(dims=dims, X=X)
    F0 = solver.full_objective(Xs, A0, s, A0, [], [], P)
    A1, F1 = solver.fac_lbfgs(Xs, A0, s, A0, [], [], P, 1)
    assert F1 < 1e-3 * F0


def _congruence(A, B, sa, sb):
    """K-tensor score: mean over components of the product of |cosines| (best permutation)."""
    import itertools
    R = len(sa)
    best = 0.0
    for perm in itertools.permutations(range(R)):
        sc = 0.0
        for j in range(R):
            c = 1.0
            for a, b in zip(A, B):
                x, y = a[:, j], b[:, perm[j]]
                c *= abs(x @ y) / (np.linalg.norm(x) * np.linalg.norm(y))
            sc += c
        best = max(best, sc / R)
    return best


def test_online_gcp_tracks_a_noise_free_planted_stream():
    """OnlineGCP (Alg. 1) with the LSQ temporal solve on a noise-free low-rank stream started
    near the truth: the temporal weights are recovered and the factors stay congruent."""
    rng = np.random.default_rng(34)
    dims, R = (8, 7, 6), 2
    A_true = [rng.standard_normal((n, R)) for n in dims]
    A0 = [a + 0.02 * rng.standard_normal(a.shape) for a in A_true]
    P = solver.Params(dims=dims, rank=R, loss="gaussian", H=3, w=1.0, kappa_f=2, tau_f=10,
                      alpha_f=1e-3, temporal="lsq")
    og = solver.OnlineGCP(P, A0)
    for t in range(1, 7):
        s_t = rng.random(R) + 0.5
        X = gcp.kruskal_full_bruteforce(s_t, A_true)
        og.step(solver.Slice(dims=dims, X=X))
        assert len(og.hist_t) == min(t, P.H)
    assert _congruence(og.Abar, A_true, og.s, s_t) > 0.99
    M = gcp.kruskal_full_bruteforce(og.s, og.Abar)
    assert np.linalg.norm(M - X) < 0.05 * np.linalg.norm(X)
