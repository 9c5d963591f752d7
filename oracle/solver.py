"""FP64 CPU oracle of the OnlineGCP solvers: ADAM, WghtGcpSgd, FacGcpSgd, OnlineGCP.

TEST INFRASTRUCTURE ONLY (see ``oracle/gcp.py``).

Follows arXiv 2110.14514 Sec. 4.4: Alg. 1 (OnlineGCP with reservoir-sampled
history window), Alg. 2 (ADAM with epoch checkpoint / rollback), Alg. 3
(temporal-weight solver), Alg. 4 (factor solver), Alg. 5 (objective estimate);
and Sec. 5 (least-squares temporal solve for the Gaussian loss).  The
L-BFGS factor solver is not in the paper; it follows Nocedal & Wright,
"Numerical Optimization", Alg. 7.4 (two-loop recursion) with a projected
backtracking Armijo line search.

Readings of points the paper leaves open:

* R-bias  ADAM bias correction uses exponent i+1 (Alg. 2 would divide by
          1 - beta1^0 = 0 at i = 0; Kingma & Ba count steps from 1).
* R-init  ADAM Init sets the checkpoint a_o to the initial point (a zero
          checkpoint would zero the variables on a first-epoch rejection).
* R-decay "Decrease learning rate" multiplies alpha by alpha_decay (0.1);
          alpha restarts at its base value at every solver call.  The factor
          solver's moments and iteration counter i persist across slices
          (Sec. 4.4 prose after Alg. 1).
* R-tol   The stop test F > tol is taken literally; tol = -inf runs exactly
          kappa epochs.
* R-draw  Sample draws of the gradient are numbered by a per-(solver call)
          draw counter that is never rolled back, so a re-run epoch after a
          rejection sees fresh samples; objective samples use draw 0 and their
          own purposes, hence one fixed sample set per solver per slice.
* R-win   The window used at step t holds only steps h < t; Alg. 1 adds t
          after solving.  Reservoir: j = 1 + U(out0, t) from counter
          (0, 0, 0, reservoir << 24 | t); slot j is replaced when j <= H.
* R-lsq   Least-squares temporal solve minimises sum (x - m)^2 + mu/2 ||s||^2
          exactly: (Gamma + mu/2 I) s = Z' vec(X), Gamma = *_k A^(k)'A^(k),
          then s <- max(s, l).

Teacher forcing: a solver given ``decisions`` (an iterator of booleans) takes
the accept/reject outcome of each epoch from it instead of its own F
comparison, and records both in ``log``.
"""
from dataclasses import dataclass, field
import math
import numpy as np

from . import gcp
from .philox import philox4x32_10, bounded


@dataclass
class Params:
    """Table 1 / Table 2 arguments of OnlineGCP (Sec. 4.3, Sec. 6)."""
    dims: tuple
    rank: int
    loss: str = "gaussian"
    lower: float = None          # None -> loss default (Sec. 4.1)
    eps: float = 1e-10
    H: int = 0
    w: float = 1.0
    theta: float = 1.0
    lam: float = 0.0
    mu: float = 0.0
    p: int = 0                   # gradient nonzero samples (sparse slices)
    q: int = 0                   # gradient zero samples
    p_obj: int = 0               # objective nonzero samples
    q_obj: int = 0               # objective zero samples
    tol_w: float = -math.inf
    tol_f: float = -math.inf
    kappa_w: int = 5
    kappa_f: int = 5
    tau_w: int = 100
    tau_f: int = 100
    alpha_w: float = 0.1
    alpha_f: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    adam_eps: float = 1e-8
    alpha_decay: float = 0.1
    cap: int = 64
    temporal: str = "adam"       # "adam" | "lsq"
    optimizer: str = "adam"      # "adam" | "lbfgs" (factor solver)
    lbfgs_mem: int = 5
    lbfgs_iters: int = 10
    seed: int = 0
    history: str = "model"       # "model": eq. gcp_stream_problem_2; "slices": eq. gcp_stream_problem_1

    def lower_bound(self):
        return gcp.default_lower_bound(self.loss) if self.lower is None else self.lower


@dataclass
class Slice:
    """One streamed slice: dense (X) or sparse COO (idx, val)."""
    dims: tuple
    X: np.ndarray = None
    idx: np.ndarray = None
    val: np.ndarray = None

    @property
    def dense(self):
        return self.X is not None


# ----------------------------------------------------------------------------
# Alg. 2: ADAM with epoch checkpoint
# ----------------------------------------------------------------------------
class Adam:
    def __init__(self, alpha, beta1, beta2, eps, lower, decay):
        self.alpha0 = alpha
        self.alpha = alpha
        self.beta1, self.beta2, self.eps = beta1, beta2, eps
        self.lower = lower
        self.decay = decay

    def init(self, a):
        """Zero moments; checkpoint = initial point (R-init)."""
        a = np.asarray(a, np.float64)
        self.u = np.zeros_like(a)
        self.v = np.zeros_like(a)
        self.u_o = np.zeros_like(a)
        self.v_o = np.zeros_like(a)
        self.a_o = a.copy()
        self.alpha = self.alpha0

    def step(self, a, g, i):
        self.u = self.beta1 * self.u + (1.0 - self.beta1) * g
        self.v = self.beta2 * self.v + (1.0 - self.beta2) * g * g
        at = self.alpha * math.sqrt(1.0 - self.beta2 ** (i + 1)) / (1.0 - self.beta1 ** (i + 1))
        a = a - at * self.u / (np.sqrt(self.v) + self.eps)
        return np.maximum(a, self.lower)

    def update(self, a, passed):
        if passed:
            self.u_o = self.u.copy()
            self.v_o = self.v.copy()
            self.a_o = np.array(a, np.float64, copy=True)
            return a
        self.u = self.u_o.copy()
        self.v = self.v_o.copy()
        self.alpha *= self.decay
        return self.a_o.copy()


# ----------------------------------------------------------------------------
# Objective and gradient pieces of one solver
# ----------------------------------------------------------------------------
def _loss_estimate(X, s, A, P, t, temporal):
    """Sample part of Alg. 5 (sparse: p', q' fixed samples; dense: exact)."""
    if X.dense:
        return gcp.dense_objective(X.X, s, A, P.loss, P.eps)
    pn, pz = ("tobj_nz", "tobj_z") if temporal else ("obj_nz", "obj_z")
    coords, x, w = gcp.stratified_samples(X.idx, X.val, X.dims, P.p_obj, P.q_obj, P.seed, t, 0,
                                          gcp.PURPOSE[pn], gcp.PURPOSE[pz], P.cap)
    return gcp.sampled_loss(coords, x, w, s, A, P.loss, P.eps)


def estimate_objective(X, A, s, Abar, s_hist, w_h, lam, mu, P, t, temporal):
    """Alg. 5: sampled loss + 1/2 sum_h w_h ||Mbar_h - M_h||^2 + lambda/2 sum ||A||^2 + mu/2 ||s||^2."""
    F = _loss_estimate(X, s, A, P, t, temporal)
    if len(s_hist):
        F += gcp.history_objective(s_hist, w_h, A, Abar)
    return F + gcp.regularization_objective(A, s, lam, mu)


def loss_gradient(X, s, A, P, t, draw, temporal):
    """Y~_(k) Z_k diag(s) and Z' y~ from one stratified draw (sparse) or exactly (dense)."""
    if X.dense:
        G, gs, _ = gcp.dense_gradient(X.X, s, A, P.loss, P.eps)
        return G, gs
    G, gs, _ = gcp.sampled_gradient(X.idx, X.val, X.dims, s, A, P.loss, P.p, P.q, P.seed, t, draw,
                                    temporal=temporal, eps=P.eps, cap=P.cap)
    return G, gs


def factor_gradient(X, A, s, Abar, s_hist, w_h, P, t, draw):
    """eq. spatial_gcp_grad: Y~_(k) Z_k diag(s) + lambda A^(k) + history term, k = 1..d."""
    G, _ = loss_gradient(X, s, A, P, t, draw, temporal=False)
    out = []
    for k in range(len(A)):
        g = G[k] + P.lam * np.asarray(A[k], np.float64)
        if len(s_hist):
            g = g + gcp.history_gradient(A, Abar, s_hist, w_h, k)
        out.append(g)
    return out


# ----------------------------------------------------------------------------
# Stored-slice history (Sec. 4.1, eq. gcp_stream_problem_1): the window keeps the slices X_h
# themselves and the history term is sum_h w_h sum_i f(x_ih, m_ih) with M_h = [[s_h; A]] (old
# weights, current factors).  Sparse stored slices are sampled like the current one, with their
# own purposes, counter t-field h and draw t * kappa_f * tau_f + d (d = 0 for the objective).
# ----------------------------------------------------------------------------
def stored_history_gradient(A, hist_X, hist_t, s_hist, w_h, P, t, draw):
    """sum_h w_h Y_h(k) Z_k diag(s_h), k = 1..d, over the stored slices."""
    G = [np.zeros(np.shape(a)) for a in A]
    base = t * P.kappa_f * P.tau_f
    for X, h, sh, wh in zip(hist_X, hist_t, s_hist, w_h):
        if X.dense:
            Gh, _, _ = gcp.dense_gradient(X.X, sh, A, P.loss, P.eps)
        else:
            Gh, _, _ = gcp.sampled_gradient(X.idx, X.val, X.dims, sh, A, P.loss, P.p, P.q, P.seed, h, base + draw,
                                            eps=P.eps, cap=P.cap, purposes=("hgrad_nz", "hgrad_z"))
        for k in range(len(A)):
            G[k] += wh * Gh[k]
    return G


def stored_history_objective(A, hist_X, hist_t, s_hist, w_h, P, t):
    """sum_h w_h sum_i f(x_ih, m_ih) (sampled for sparse stored slices)."""
    F = 0.0
    base = t * P.kappa_f * P.tau_f
    for X, h, sh, wh in zip(hist_X, hist_t, s_hist, w_h):
        if X.dense:
            F += wh * gcp.dense_objective(X.X, sh, A, P.loss, P.eps)
        else:
            coords, x, w = gcp.stratified_samples(X.idx, X.val, X.dims, P.p_obj, P.q_obj, P.seed, h, base,
                                                  gcp.PURPOSE["hobj_nz"], gcp.PURPOSE["hobj_z"], P.cap)
            F += wh * gcp.sampled_loss(coords, x, w, sh, A, P.loss, P.eps)
    return F


def _decide(F_new, F_old, decisions, log):
    own = not (F_new > F_old)
    passed = own if decisions is None else bool(next(decisions))
    log.append({"F_new": F_new, "F_old": F_old, "own": own, "passed": passed})
    return passed


# ----------------------------------------------------------------------------
# Alg. 3: temporal weights solver
# ----------------------------------------------------------------------------
def wght_gcp_sgd(X, A, P, t, decisions=None, log=None, s_init=None):
    log = [] if log is None else log
    R = P.rank
    s = np.zeros(R) if s_init is None else np.array(s_init, np.float64)
    adam = Adam(P.alpha_w, P.beta1, P.beta2, P.adam_eps, P.lower_bound(), P.alpha_decay)
    adam.init(s)
    F = estimate_objective(X, A, s, None, [], [], 0.0, P.mu, P, t, temporal=True)
    i = 0
    draw = 0
    epoch = 0
    while F > P.tol_w and epoch < P.kappa_w:
        F_old = F
        for _ in range(P.tau_w):
            _, gs = loss_gradient(X, s, A, P, t, draw, temporal=True)
            g = gs + P.mu * s
            s = adam.step(s, g, i)
            i += 1
            draw += 1
        F = estimate_objective(X, A, s, None, [], [], 0.0, P.mu, P, t, temporal=True)
        if not _decide(F, F_old, decisions, log):
            s = adam.update(s, False)
            F = F_old
            i -= P.tau_w
        else:
            s = adam.update(s, True)
        epoch += 1
    return s, F


def lsq_temporal(X, A, P):
    """Least-squares temporal solve for the Gaussian loss (Sec. 5, R-lsq)."""
    R = P.rank
    Gam = gcp.hadamard_gram(A, A)
    if X.dense:
        rhs = gcp.Zall(A).T @ gcp.vec(np.asarray(X.X, np.float64))
    else:
        rhs = gcp.sparse_temporal(np.asarray(X.idx, np.int64).reshape(-1, len(A)), X.val, A)
    s = np.linalg.solve(Gam + 0.5 * P.mu * np.eye(R), rhs)
    return np.maximum(s, P.lower_bound())


# ----------------------------------------------------------------------------
# Alg. 4: factor matrix solver (ADAM) and the L-BFGS alternative
# ----------------------------------------------------------------------------
def _flat(A):
    return np.concatenate([np.asarray(a, np.float64).ravel() for a in A])


def _unflat(v, A):
    out, o = [], 0
    for a in A:
        n = a.size
        out.append(v[o:o + n].reshape(a.shape).copy())
        o += n
    return out


def fac_gcp_sgd(X, A, s, Abar, s_hist, w_h, P, t, i, adam, decisions=None, log=None, hist_X=None, hist_t=None):
    """Alg. 4.  ``adam`` is the persistent AdamFac instance; returns (A, i, F).  With hist_X (the
    stored slices of the window, P.history == "slices") the history term is that of eq.
    gcp_stream_problem_1 instead of the model-based penalty."""
    log = [] if log is None else log
    adam.alpha = adam.alpha0
    a = _flat(A)
    stored = hist_X is not None

    def objective(Av):
        if stored:
            return (estimate_objective(X, Av, s, None, [], [], P.lam, 0.0, P, t, temporal=False) +
                    stored_history_objective(Av, hist_X, hist_t, s_hist, w_h, P, t))
        return estimate_objective(X, Av, s, Abar, s_hist, w_h, P.lam, 0.0, P, t, temporal=False)

    def gradient(Av, draw):
        if stored:
            G = factor_gradient(X, Av, s, None, [], [], P, t, draw)
            H = stored_history_gradient(Av, hist_X, hist_t, s_hist, w_h, P, t, draw)
            return [g + h for g, h in zip(G, H)]
        return factor_gradient(X, Av, s, Abar, s_hist, w_h, P, t, draw)

    F = objective(A)
    draw = 0
    epoch = 0
    while F > P.tol_f and epoch < P.kappa_f:
        F_old = F
        for _ in range(P.tau_f):
            G = gradient(_unflat(a, A), draw)
            a = adam.step(a, _flat(G), i)
            i += 1
            draw += 1
        F = objective(_unflat(a, A))
        if not _decide(F, F_old, decisions, log):
            a = adam.update(a, False)
            F = F_old
            i -= P.tau_f
        else:
            a = adam.update(a, True)
        epoch += 1
    return _unflat(a, A), i, F


def full_objective(X, A, s, Abar, s_hist, w_h, P):
    """eq. gcp_stream_objective evaluated exactly on a dense slice (mu term omitted: s is fixed)."""
    F = gcp.dense_objective(X.X, s, A, P.loss, P.eps)
    if len(s_hist):
        F += gcp.history_objective(s_hist, w_h, A, Abar)
    return F + gcp.regularization_objective(A, s, P.lam, 0.0)


def lbfgs_direction(g, S, Yv):
    """H g by the two-loop recursion (Nocedal & Wright Alg. 7.4) over the pairs (S[i], Yv[i]),
    oldest first, with H_0 = gamma I, gamma = s'y / y'y of the newest pair (1 / ||g|| without
    pairs)."""
    qv = g.copy()
    alphas = []
    for sv, yv in reversed(list(zip(S, Yv))):
        rho = 1.0 / (yv @ sv)
        al = rho * (sv @ qv)
        alphas.append((al, rho, sv, yv))
        qv = qv - al * yv
    gamma = (S[-1] @ Yv[-1]) / (Yv[-1] @ Yv[-1]) if S else 1.0 / max(np.linalg.norm(g), 1e-300)
    r = gamma * qv
    for al, rho, sv, yv in reversed(alphas):
        be = rho * (yv @ r)
        r = r + sv * (al - be)
    return r


def fac_lbfgs(X, A, s, Abar, s_hist, w_h, P, t):
    """Projected L-BFGS on the factor matrices of a dense slice (build-defined, not in the paper).

    Per iteration: direction p = -H g by the two-loop recursion over the last
    lbfgs_mem pairs (initial scaling gamma = s'y / y'y); step size from
    backtracking (alpha = 1, halve up to 30 times) until the projected point
    a+ = max(a + alpha p, l) satisfies F(a+) <= F(a) + 1e-4 g'(a+ - a).  A pair
    is stored only when s'y > 1e-12 * ||s|| ||y||.  Stops early when no step is
    accepted.
    """
    lower = P.lower_bound()
    a = _flat(A)

    def fg(v):
        Av = _unflat(v, A)
        F = full_objective(X, Av, s, Abar, s_hist, w_h, P)
        G = factor_gradient(X, Av, s, Abar, s_hist, w_h, P, t, 0)
        return F, _flat(G)

    F, g = fg(a)
    S, Yv = [], []
    for _ in range(P.lbfgs_iters):
        pdir = -lbfgs_direction(g, S, Yv)
        step = 1.0
        accepted = False
        for _ls in range(30):
            a_new = np.maximum(a + step * pdir, lower)
            F_new, g_new = fg(a_new)
            if F_new <= F + 1e-4 * (g @ (a_new - a)):
                accepted = True
                break
            step *= 0.5
        if not accepted:
            break
        sv, yv = a_new - a, g_new - g
        if sv @ yv > 1e-12 * np.linalg.norm(sv) * np.linalg.norm(yv):
            S.append(sv)
            Yv.append(yv)
            if len(S) > P.lbfgs_mem:
                S.pop(0)
                Yv.pop(0)
        a, F, g = a_new, F_new, g_new
    return _unflat(a, A), F


# ----------------------------------------------------------------------------
# Alg. 1: OnlineGCP
# ----------------------------------------------------------------------------
def reservoir_index(seed, t):
    """j = 1 + U(out0, t) with counter (0, 0, 0, reservoir << 24 | t) (R-win)."""
    ctr = [[0, 0, 0, gcp.counter_word3(gcp.PURPOSE["reservoir"], t)]]
    out = philox4x32_10(ctr, gcp.philox_key(seed))
    return 1 + int(bounded(out[:, 0], t)[0])


class OnlineGCP:
    """State of Alg. 1 across slices; ``step`` is one pass of its loop body."""

    def __init__(self, P, A0, hist_t=(), hist_s=()):
        self.P = P
        self.Abar = [np.array(a, np.float64, copy=True) for a in A0]
        self.hist_t = list(hist_t)
        self.hist_s = [np.array(h, np.float64) for h in hist_s]
        self.hist_X = []          # stored slices of the window (P.history == "slices")
        self.adam_f = Adam(P.alpha_f, P.beta1, P.beta2, P.adam_eps, P.lower_bound(), P.alpha_decay)
        self.adam_f.init(_flat(self.Abar))
        self.i = 0
        self.t = 0
        self.s = np.zeros(P.rank)
        self.log_w, self.log_f = [], []

    def step(self, X, decisions_w=None, decisions_f=None):
        P = self.P
        self.t += 1
        t = self.t
        A = [a.copy() for a in self.Abar]
        if P.temporal == "lsq":
            s = lsq_temporal(X, A, P)
            F_w = None
        else:
            s, F_w = wght_gcp_sgd(X, A, P, t, decisions_w, self.log_w)
        w_h = gcp.history_weights(self.hist_t, t, P.w, P.theta)
        if P.optimizer == "lbfgs":
            A, F_f = fac_lbfgs(X, A, s, self.Abar, self.hist_s, w_h, P, t)
        else:
            stored = P.history == "slices"
            A, self.i, F_f = fac_gcp_sgd(X, A, s, self.Abar, self.hist_s, w_h, P, t, self.i,
                                         self.adam_f, decisions_f, self.log_f,
                                         hist_X=self.hist_X if stored else None,
                                         hist_t=self.hist_t if stored else None)
        self.enter_window(t, s, X)
        self.Abar = [a.copy() for a in A]
        self.s = s
        return {"F_w": F_w, "F_f": F_f, "s": s}

    def enter_window(self, t, s, X=None):
        """Alg. 1's reservoir update of the history window with step t (weights s, slice X)."""
        P = self.P
        if P.H <= 0:
            return
        if len(self.hist_t) < P.H:
            self.hist_t.append(t)
            self.hist_s.append(np.array(s, np.float64, copy=True))
            self.hist_X.append(X)
        else:
            j = reservoir_index(P.seed, t)
            if j <= P.H:
                self.hist_t[j - 1] = t
                self.hist_s[j - 1] = np.array(s, np.float64, copy=True)
                self.hist_X[j - 1] = X


# ----------------------------------------------------------------------------
# Warm start: static GCP-SGD on the first slices stacked as a (d+1)-way tensor
# (Sec. 4.4: the initial factors come from a static fit of an initial set of
# slices; Sec. 6: every experiment starts from such a warm start, whose slices
# also form the initial history window).
# ----------------------------------------------------------------------------
def stacked_loss_gradient(slices, A, S, P, draw, t0=1):
    """Gradient of sum_h f(X_h, M_h), M_h = [[S_h; A^(1..d)]], the loss of the (d+1)-way tensor whose
    last mode indexes the slices, with S (n x R) that mode's factor matrix:
    dF/dA^(k) = sum_h Y_h(k) Z_k diag(S_h) and dF/dS_h = Z' vec(Y_h), one slice at a time.
    Sparse slices are sampled per slice (strata: slice x {nonzero, zero}; p + q samples each, slice
    h with time index t0 + h).  Returns (list of d gradients, n x R gradient of S)."""
    G = [np.zeros(np.shape(a)) for a in A]
    GS = np.zeros(np.shape(S))
    for h, X in enumerate(slices):
        Gh, gsh = loss_gradient(X, S[h], A, P, t0 + h, draw, temporal=False)
        for k in range(len(A)):
            G[k] += Gh[k]
        GS[h] = gsh
    return G, GS


def stacked_objective(slices, A, S, P, t0=1):
    """sum_h (sampled or exact) loss of slice h at (A, S_h) + lambda/2 (sum_k ||A^(k)||^2 + ||S||^2):
    the stacked problem regularises every factor matrix, the slice mode's included."""
    F = 0.0
    for h, X in enumerate(slices):
        F += _loss_estimate(X, S[h], A, P, t0 + h, temporal=False)
    return F + gcp.regularization_objective(list(A) + [S], np.zeros(1), P.lam, 0.0)


def static_gcp_sgd(slices, A0, S0, P, decisions=None, log=None, t0=1):
    """GCP-SGD on the stacked tensor: the epoch / ADAM / rollback loop of Alg. 4 (Alg. 2 steps,
    kappa_f epochs of tau_f iterations, rate alpha_f) over the variables (A^(1), ..., A^(d), S),
    with no history term.  Returns (A, S, F)."""
    log = [] if log is None else log
    A = [np.array(a, np.float64, copy=True) for a in A0]
    S = np.array(S0, np.float64, copy=True)
    allv = A + [S]
    adam = Adam(P.alpha_f, P.beta1, P.beta2, P.adam_eps, P.lower_bound(), P.alpha_decay)
    a = _flat(allv)
    adam.init(a)
    F = stacked_objective(slices, A, S, P, t0)
    i = 0
    draw = 0          # never rolled back (R-draw): a re-run epoch draws fresh samples
    epoch = 0
    while F > P.tol_f and epoch < P.kappa_f:
        F_old = F
        for _ in range(P.tau_f):
            cur = _unflat(a, allv)
            G, GS = stacked_loss_gradient(slices, cur[:-1], cur[-1], P, draw, t0)
            g = _flat([Gk + P.lam * ak for Gk, ak in zip(G, cur[:-1])] + [GS + P.lam * cur[-1]])
            a = adam.step(a, g, i)
            i += 1
            draw += 1
        cur = _unflat(a, allv)
        F = stacked_objective(slices, cur[:-1], cur[-1], P, t0)
        if not _decide(F, F_old, decisions, log):
            a = adam.update(a, False)
            F = F_old
            i -= P.tau_f
        else:
            a = adam.update(a, True)
        epoch += 1
    cur = _unflat(a, allv)
    return cur[:-1], cur[-1], F


def warm_start(slices, A0, S0, P, decisions=None, log=None):
    """The warm start of an OnlineGCP stream: static_gcp_sgd on slices 1..n (time indices 1..n),
    then an OnlineGCP state at t = n whose factors are the fit and whose history window holds the
    warm-start slices' weights S_h, entered in order h = 1..n by the reservoir rule of Alg. 1."""
    A, S, F = static_gcp_sgd(slices, A0, S0, P, decisions, log)
    og = OnlineGCP(P, A)
    og.t = len(slices)
    for h in range(1, len(slices) + 1):
        og.enter_window(h, S[h - 1], slices[h - 1])
    og.s = S[-1].copy()
    return og, S, F
