"""FP64 CPU oracle for the streaming-GCP gradient path (plain numpy, slow, obvious).

TEST INFRASTRUCTURE ONLY.  Nothing under ``oracle/`` is part of the product:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it, and it shares no code with the CUDA library.

What it follows (Phipps, Johnson, Kolda, "Streaming Generalized Canonical
Polyadic Tensor Decompositions", arXiv 2110.14514):

* Kruskal model value m_i = sum_j s_j prod_k a^(k)_{i_k j}        (Sec. 2.1, eq. CP_model)
* losses f(x, m) and y = df/dm                                     (Sec. 2.2, eq. GCP_problem)
* dF/dA^(k) = Y_(k) Z_k diag(s),  dF/ds = Z' vec(Y)                (Sec. 2.2, eqs. gcp_grad_A, gcp_grad_lambda)
* stratified sampled gradient tensor Y~ and its weights            (Sec. 4.3, Alg. 6)
* sampled objective estimate F~                                    (Sec. 4.3, Alg. 5)
* model-based history penalty 1/2 sum_h w_h ||Mbar_h - M_h||^2,
  w_h = w theta^(t-h), and its factor gradient                    (Sec. 4.1 eq. gcp_stream_problem_2; Sec. 4.2 eq. spatial_gcp_grad)

Readings of points the paper leaves open (each is listed with its reason in
the design notes of the repository):

* R-sign  The dense Gaussian formula of Sec. 5 has the opposite sign of eq.
          gcp_grad_A with y = 2(m - x); the oracle uses eq. gcp_grad_A.
* R-mu    The temporal gradient of Sec. 4.2 / Alg. 3 writes lambda*s, the
          objective penalises mu/2 ||s||^2: the oracle uses mu.
* R-half  History objective weight is 1/2 w_h everywhere (eq.
          gcp_stream_objective, Alg. 5), consistent with eq. spatial_gcp_grad.
* R-eps   log m is evaluated as log(m + eps) (Sec. 2.2 footnote), eps a parameter.
* R-logit Bernoulli with logit link (f = log(1 + e^m) - x m) is provided in
          addition to the odds link f = log(m + 1) - x log(m + eps).
* R-rng   The random draws of Alg. 5 / Alg. 6 are fixed as follows.  Key =
          (seed mod 2^32, seed >> 32).  Counter = (slot, attempt, draw,
          purpose << 24 | (t mod 2^24)).  A nonzero sample takes COO entry
          U(out0, eta) in the caller's COO order.  A zero sample of slot c
          tries attempts a = 0, 1, ..., cap-1 with i_k = U(out_k, I_k) and
          takes the first candidate that is not a nonzero; U(u, n) =
          (u * n) >> 32.  Each slot is an independent uniform draw from the
          zeros, i.e. the same distribution as the sequential rejection loop
          of Alg. 5 / Alg. 6, but order independent.
* R-dense Dense slices use the exact full gradient and objective (every
          entry once, weight 1).
"""
import numpy as np

from .philox import philox4x32_10, bounded

LOSSES = ("gaussian", "poisson", "bernoulli_odds", "bernoulli_logit")

# Sample-stream purposes (third-word high byte of the Philox counter).
PURPOSE = {
    "grad_nz": 0, "grad_z": 1, "obj_nz": 2, "obj_z": 3, "reservoir": 4,
    "tgrad_nz": 5, "tgrad_z": 6, "tobj_nz": 7, "tobj_z": 8,
    # stored history slices (eq. gcp_stream_problem_1): counter t-field = the stored slice's own
    # time index h, draw = t * kappa_f * tau_f + (iteration of the factor solve at step t)
    "hgrad_nz": 9, "hgrad_z": 10, "hobj_nz": 11, "hobj_z": 12,
}


class SamplingLimit(RuntimeError):
    """A zero-sample slot found no zero within its attempt cap."""


# ----------------------------------------------------------------------------
# Losses (Sec. 2.2, eq. GCP_problem and its footnote)
# ----------------------------------------------------------------------------
def loss_f(loss, x, m, eps=1e-10):
    """Elementwise loss f(x, m) in float64."""
    x = np.asarray(x, np.float64)
    m = np.asarray(m, np.float64)
    if loss == "gaussian":
        return (x - m) ** 2
    if loss == "poisson":
        return m - x * np.log(m + eps)
    if loss == "bernoulli_odds":
        return np.log(m + 1.0) - x * np.log(m + eps)
    if loss == "bernoulli_logit":
        # log(1 + e^m) - x m, written so that it does not overflow
        return np.maximum(m, 0.0) + np.log1p(np.exp(-np.abs(m))) - x * m
    raise ValueError(loss)


def loss_dfdm(loss, x, m, eps=1e-10):
    """Elementwise derivative df/dm (the entries of the gradient tensor Y)."""
    x = np.asarray(x, np.float64)
    m = np.asarray(m, np.float64)
    if loss == "gaussian":
        return 2.0 * (m - x)
    if loss == "poisson":
        return 1.0 - x / (m + eps)
    if loss == "bernoulli_odds":
        return 1.0 / (m + 1.0) - x / (m + eps)
    if loss == "bernoulli_logit":
        with np.errstate(over="ignore"):   # e^-m -> inf for m << 0: 1 / (1 + inf) = 0 is the limit
            return 1.0 / (1.0 + np.exp(-m)) - x
    raise ValueError(loss)


def default_lower_bound(loss):
    """l = 0 for Poisson and Bernoulli-odds (m must stay >= 0), else -inf (Sec. 4.1)."""
    return 0.0 if loss in ("poisson", "bernoulli_odds") else -np.inf


# ----------------------------------------------------------------------------
# Kruskal model (Sec. 2.1, eq. CP_model) and Khatri-Rao algebra (Sec. 2.2)
# ----------------------------------------------------------------------------
def kruskal_value(s, A, coords):
    """m_i = sum_j s_j prod_k A[k][i_k, j] for each row i of coords (n, d)."""
    coords = np.asarray(coords, np.int64).reshape(-1, len(A))
    prod = np.broadcast_to(np.asarray(s, np.float64), (coords.shape[0], len(s))).copy()
    for k, Ak in enumerate(A):
        prod *= np.asarray(Ak, np.float64)[coords[:, k], :]
    return prod.sum(axis=1)


def kruskal_full_bruteforce(s, A):
    """Full tensor sum_j s_j a_j^(1) o ... o a_j^(d) by explicit outer products."""
    dims = [a.shape[0] for a in A]
    M = np.zeros(dims)
    for j in range(len(s)):
        outer = np.asarray(A[0][:, j], np.float64)
        for Ak in A[1:]:
            outer = np.multiply.outer(outer, np.asarray(Ak[:, j], np.float64))
        M += s[j] * outer
    return M


def khatri_rao(mats):
    """Column-wise Kronecker product mats[0] (.) mats[1] (.) ... ; the last
    matrix's row index varies fastest."""
    out = np.asarray(mats[0], np.float64)
    for B in mats[1:]:
        B = np.asarray(B, np.float64)
        out = (out[:, None, :] * B[None, :, :]).reshape(-1, out.shape[1])
    return out


def Zk(A, k):
    """Z_k = A^(d) (.) ... (.) A^(k+1) (.) A^(k-1) (.) ... (.) A^(1)."""
    return khatri_rao([A[n] for n in reversed(range(len(A))) if n != k])


def Zall(A):
    """Z = A^(d) (.) ... (.) A^(1)."""
    return khatri_rao([A[n] for n in reversed(range(len(A)))])


def unfold(T, k):
    """Mode-k matricization: row i_k, columns ordered with the lowest remaining
    mode index fastest (matches the row order of Z_k)."""
    return np.reshape(np.moveaxis(T, k, 0), (T.shape[k], -1), order="F")


def fold(Mk, k, dims):
    """Inverse of unfold."""
    rest = [dims[n] for n in range(len(dims)) if n != k]
    return np.moveaxis(np.reshape(Mk, [dims[k]] + rest, order="F"), 0, k)


def vec(T):
    """Vectorization with the first mode index fastest (matches the rows of Z)."""
    return np.reshape(T, -1, order="F")


# ----------------------------------------------------------------------------
# Exact (dense) GCP gradient, eqs. gcp_grad_A and gcp_grad_lambda
# ----------------------------------------------------------------------------
def dense_model(s, A):
    """M = fold(A^(1) diag(s) Z_1', 1): mode-1 unfolding of eq. CP_model."""
    dims = [a.shape[0] for a in A]
    M1 = (np.asarray(A[0], np.float64) * np.asarray(s, np.float64)) @ Zk(A, 0).T
    return fold(M1, 0, dims)


def dense_gradient(X, s, A, loss, eps=1e-10, explicit_Z=False):
    """Exact GCP gradient of F = sum_i f(x_i, m_i) over every entry of a dense slice.

    Returns (G, gs, F) with G[k] = Y_(k) Z_k diag(s) and gs = Z' vec(Y).
    With explicit_Z the temporal gradient forms Z itself (small tensors only);
    otherwise it uses sum_rows(A^(1) * (Y_(1) Z_1)), which equals Z' vec(Y)
    because row (i_1, rest) of Z is A^(1)[i_1] * Z_1[rest].
    """
    X = np.asarray(X, np.float64)
    s = np.asarray(s, np.float64)
    M = dense_model(s, A)
    Y = loss_dfdm(loss, X, M, eps)
    F = float(loss_f(loss, X, M, eps).sum())
    G = [unfold(Y, k) @ Zk(A, k) * s[None, :] for k in range(len(A))]
    if explicit_Z:
        gs = Zall(A).T @ vec(Y)
    else:
        gs = (np.asarray(A[0], np.float64) * (unfold(Y, 0) @ Zk(A, 0))).sum(axis=0)
    return G, gs, F


def dense_objective(X, s, A, loss, eps=1e-10):
    """Exact sum_i f(x_i, m_i) over a dense slice."""
    return float(loss_f(loss, np.asarray(X, np.float64), dense_model(s, A), eps).sum())


# ----------------------------------------------------------------------------
# Stratified sampling (Sec. 4.3, Alg. 5 and Alg. 6) with the counter layout R-rng
# ----------------------------------------------------------------------------
def philox_key(seed):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return (seed & 0xFFFFFFFF, seed >> 32)


def counter_word3(purpose, t):
    return ((int(purpose) & 0xFF) << 24) | (int(t) & 0xFFFFFF)


def linear_keys(coords, dims):
    """C-order linear index ((i_1 I_2 + i_2) I_3 + i_3 ...) as uint64."""
    coords = np.asarray(coords, np.int64)
    key = np.zeros(coords.shape[0], np.uint64)
    for k, n in enumerate(dims):
        key = key * np.uint64(n) + coords[:, k].astype(np.uint64)
    return key


def nonzero_sample_ids(nnz, p, seed, t, draw, purpose):
    """COO positions of p nonzero samples: U(out0, eta) with counter (c, 0, draw, w3)."""
    c = np.arange(p, dtype=np.uint64)
    ctr = np.stack([c, np.zeros_like(c), np.full_like(c, draw),
                    np.full_like(c, counter_word3(purpose, t))], axis=1)
    out = philox4x32_10(ctr, philox_key(seed))
    return bounded(out[:, 0], nnz)


def zero_sample_coords(dims, q, seed, t, draw, purpose, nz_sorted_keys, cap):
    """q zero coordinates, one independent bounded rejection sequence per slot.

    nz_sorted_keys: sorted uint64 linear keys of the slice's nonzeros.
    Returns (coords (q, d) int64, attempts (q,) int64: the accepted attempt).
    """
    d = len(dims)
    coords = np.zeros((q, d), np.int64)
    attempts = np.full(q, -1, np.int64)
    pending = np.arange(q, dtype=np.int64)
    dims_u = np.asarray(dims, np.uint64)
    for a in range(cap):
        if pending.size == 0:
            break
        c = pending.astype(np.uint64)
        ctr = np.stack([c, np.full_like(c, a), np.full_like(c, draw),
                        np.full_like(c, counter_word3(purpose, t))], axis=1)
        out = philox4x32_10(ctr, philox_key(seed))
        cand = np.stack([bounded(out[:, k], dims_u[k]) for k in range(d)], axis=1)
        keys = linear_keys(cand, dims)
        if len(nz_sorted_keys):
            pos = np.minimum(np.searchsorted(nz_sorted_keys, keys), len(nz_sorted_keys) - 1)
            is_nz = nz_sorted_keys[pos] == keys
        else:
            is_nz = np.zeros(len(keys), bool)
        ok = ~is_nz
        coords[pending[ok]] = cand[ok]
        attempts[pending[ok]] = a
        pending = pending[~ok]
    if pending.size:
        raise SamplingLimit(f"{pending.size} zero-sample slots hit the attempt cap {cap}")
    return coords, attempts


def stratified_samples(coo_idx, coo_val, dims, p, q, seed, t, draw, purpose_nz, purpose_z, cap=64):
    """The p + q samples of one stratified draw (Sec. 4.3).

    Returns (coords (p+q, d), x (p+q,), weight (p+q,)) where nonzero samples
    carry eta/p and zero samples carry zeta/q with zeta = prod I_k - eta.
    If the slice has no zeros, q is taken as 0.
    """
    coo_idx = np.asarray(coo_idx, np.int64).reshape(-1, len(dims))
    coo_val = np.asarray(coo_val, np.float64)
    eta = coo_idx.shape[0]
    omega = int(np.prod([int(n) for n in dims], dtype=object))
    zeta = omega - eta
    if zeta == 0:
        q = 0
    parts_c, parts_x, parts_w = [], [], []
    if p > 0 and eta > 0:
        ids = nonzero_sample_ids(eta, p, seed, t, draw, purpose_nz)
        parts_c.append(coo_idx[ids])
        parts_x.append(coo_val[ids])
        parts_w.append(np.full(p, eta / p))
    if q > 0:
        nz_keys = np.sort(linear_keys(coo_idx, dims))
        zc, _ = zero_sample_coords(dims, q, seed, t, draw, purpose_z, nz_keys, cap)
        parts_c.append(zc)
        parts_x.append(np.zeros(q))
        parts_w.append(np.full(q, zeta / q))
    if not parts_c:
        return np.zeros((0, len(dims)), np.int64), np.zeros(0), np.zeros(0)
    return np.concatenate(parts_c), np.concatenate(parts_x), np.concatenate(parts_w)


def strat_grad_tensor(coords, x, weight, s, A, loss, eps=1e-10):
    """Alg. 6 body: the sparse sampled gradient tensor Y~.

    Every sample adds weight * df/dm(x, m) to y~ at its coordinate; repeated
    coordinates add up.  Returns (unique coords, y~ values).
    """
    dims = [a.shape[0] for a in A]
    m = kruskal_value(s, A, coords)
    contrib = weight * loss_dfdm(loss, x, m, eps)
    keys = linear_keys(coords, dims)
    uniq, first, inv = np.unique(keys, return_index=True, return_inverse=True)
    ytil = np.zeros(uniq.shape[0])
    np.add.at(ytil, inv, contrib)
    return np.asarray(coords, np.int64)[first], ytil


def sparse_mttkrp(coords, yvals, s, A, k):
    """Y~_(k) Z_k diag(s) for a sparse Y~: row i_k gets y * s * prod_{n != k} A[n][i_n]."""
    R = len(s)
    rows = np.broadcast_to(np.asarray(s, np.float64), (len(yvals), R)) * np.asarray(yvals)[:, None]
    for n, An in enumerate(A):
        if n != k:
            rows = rows * np.asarray(An, np.float64)[coords[:, n], :]
    G = np.zeros((A[k].shape[0], R))
    np.add.at(G, coords[:, k], rows)
    return G


def sparse_temporal(coords, yvals, A):
    """Z' vec(Y~) for a sparse Y~: sum over entries of y * prod_k A[k][i_k]."""
    R = A[0].shape[1]
    rows = np.broadcast_to(np.asarray(yvals, np.float64)[:, None], (len(yvals), R)).copy()
    for k, Ak in enumerate(A):
        rows = rows * np.asarray(Ak, np.float64)[coords[:, k], :]
    return rows.sum(axis=0)


def sampled_loss(coords, x, weight, s, A, loss, eps=1e-10):
    """Alg. 5 sample sum: sum over samples of weight * f(x, m)."""
    m = kruskal_value(s, A, coords)
    return float((weight * loss_f(loss, x, m, eps)).sum())


def sampled_gradient(coo_idx, coo_val, dims, s, A, loss, p, q, seed, t, draw,
                     temporal=False, eps=1e-10, cap=64, purposes=None):
    """Stochastic gradient from one stratified draw (Alg. 6 then eq. gcp_grad_A / gcp_grad_lambda).

    temporal=False uses purposes grad_nz/grad_z and returns the factor
    gradients [Y~_(k) Z_k diag(s)]_k together with Z' y~; temporal=True uses the
    temporal-solver purposes.  Returns (G list, gs, sampled loss on the same samples).
    """
    pn, pz = ("tgrad_nz", "tgrad_z") if temporal else ("grad_nz", "grad_z")
    if purposes is not None:
        pn, pz = purposes
    coords, x, w = stratified_samples(coo_idx, coo_val, dims, p, q, seed, t, draw,
                                      PURPOSE[pn], PURPOSE[pz], cap)
    uc, yt = strat_grad_tensor(coords, x, w, s, A, loss, eps)
    G = [sparse_mttkrp(uc, yt, s, A, k) for k in range(len(A))]
    gs = sparse_temporal(uc, yt, A)
    F = sampled_loss(coords, x, w, s, A, loss, eps)
    return G, gs, F


# ----------------------------------------------------------------------------
# History penalty (Sec. 4.1 eq. gcp_stream_problem_2, Sec. 4.2 eq. spatial_gcp_grad)
# ----------------------------------------------------------------------------
def history_weights(hist_t, t, w, theta):
    """w_h = w theta^(t-h) (Sec. 4.1)."""
    return np.array([w * theta ** (t - h) for h in hist_t], np.float64)


def history_objective_bruteforce(s_hist, w_h, A, Abar):
    """1/2 sum_h w_h ||Mbar_h - M_h||_F^2 from explicit full tensors (tiny sizes)."""
    tot = 0.0
    for sh, wh in zip(s_hist, w_h):
        D = kruskal_full_bruteforce(sh, Abar) - kruskal_full_bruteforce(sh, A)
        tot += 0.5 * wh * float((D * D).sum())
    return tot


def hadamard_gram(U, V, skip=None):
    """*_{n != skip} U[n]' V[n]  (Hadamard product of R x R cross-Gram matrices)."""
    R = U[0].shape[1]
    out = np.ones((R, R))
    for n in range(len(U)):
        if n != skip:
            out *= np.asarray(U[n], np.float64).T @ np.asarray(V[n], np.float64)
    return out


def history_objective(s_hist, w_h, A, Abar):
    """1/2 sum_h w_h ||Mbar_h - M_h||^2 through <[[s;U]],[[s;V]]> = s'(*_n U_n'V_n)s."""
    Gbb = hadamard_gram(Abar, Abar)
    Gba = hadamard_gram(Abar, A)
    Gaa = hadamard_gram(A, A)
    tot = 0.0
    for sh, wh in zip(s_hist, w_h):
        sh = np.asarray(sh, np.float64)
        tot += 0.5 * wh * (sh @ Gbb @ sh - 2.0 * sh @ Gba @ sh + sh @ Gaa @ sh)
    return float(tot)


def history_gradient(A, Abar, s_hist, w_h, k, explicit_Z=False):
    """sum_h w_h (A^(k) diag(s_h) Z_k'Z_k diag(s_h) - Abar^(k) diag(s_h) Zbar_k'Z_k diag(s_h))
    (eq. spatial_gcp_grad).  Z_k'Z_k is formed from explicit Khatri-Rao products
    when explicit_Z, else by the identity Z_k'Z_k = *_{n != k} A^(n)'A^(n)."""
    if explicit_Z:
        ZZ = Zk(A, k).T @ Zk(A, k)
        ZbZ = Zk(Abar, k).T @ Zk(A, k)
    else:
        ZZ = hadamard_gram(A, A, skip=k)
        ZbZ = hadamard_gram(Abar, A, skip=k)
    Ak = np.asarray(A[k], np.float64)
    Abk = np.asarray(Abar[k], np.float64)
    G = np.zeros_like(Ak)
    for sh, wh in zip(s_hist, w_h):
        D = np.diag(np.asarray(sh, np.float64))
        G += wh * (Ak @ D @ ZZ @ D - Abk @ D @ ZbZ @ D)
    return G


def regularization_objective(A, s, lam, mu):
    """lambda/2 sum_k ||A^(k)||^2 + mu/2 ||s||^2 (eq. gcp_stream_t)."""
    val = 0.0
    if lam:
        val += 0.5 * lam * sum(float((np.asarray(a, np.float64) ** 2).sum()) for a in A)
    if mu:
        val += 0.5 * mu * float((np.asarray(s, np.float64) ** 2).sum())
    return val


def kruskal_full(s, A):
    """Full Kruskal tensor (alias of the explicit outer-product sum)."""
    return kruskal_full_bruteforce(s, A)


# ----------------------------------------------------------------------------
# Reconstruction losses and the K-tensor score (Sec. 6)
# ----------------------------------------------------------------------------
def coo_to_dense(coo_idx, coo_val, dims):
    """The full slice of a COO slice (small sizes only)."""
    X = np.zeros(dims)
    idx = np.asarray(coo_idx, np.int64).reshape(-1, len(dims))
    X[tuple(idx.T)] = np.asarray(coo_val, np.float64)
    return X


def exact_slice_loss(X, s, A, loss, eps=1e-10):
    """sum over every entry i of f(x_i, m_i) (a dense array X), and ||X||_F^2: the numerator and
    denominator of eq. local_loss evaluated exactly (the global loss of Sec. 6 uses this for every
    earlier slice with the final factors)."""
    X = np.asarray(X, np.float64)
    return dense_objective(X, s, A, loss, eps), float((X * X).sum())


def sampled_slice_loss(coo_idx, coo_val, dims, s, A, loss, p_obj, q_obj, seed, t, eps=1e-10, cap=64):
    """The sampled numerator of eq. local_loss for a sparse slice: Alg. 5's sample sum with the
    factor solver's objective samples (draw 0, time index t), no history or regularisation term;
    and ||X||_F^2 = sum of the squared nonzeros."""
    coords, x, w = stratified_samples(coo_idx, coo_val, dims, p_obj, q_obj, seed, t, 0, PURPOSE["obj_nz"],
                                      PURPOSE["obj_z"], cap)
    return sampled_loss(coords, x, w, s, A, loss, eps), float((np.asarray(coo_val, np.float64) ** 2).sum())


def congruence_matrix(A, B):
    """Q[r, c] = prod_k |cos(a_r^(k), b_c^(k))| between the columns of two K-tensors' factor
    matrices (Tomasi and Bro's congruence of rank-one components; weights play no part)."""
    R = np.shape(A[0])[1]
    Q = np.ones((R, R))
    for Ak, Bk in zip(A, B):
        Ak = np.asarray(Ak, np.float64)
        Bk = np.asarray(Bk, np.float64)
        na = np.linalg.norm(Ak, axis=0)
        nb = np.linalg.norm(Bk, axis=0)
        Q *= np.abs(Ak.T @ Bk) / np.outer(na, nb)
    return Q


def kruskal_score(A, B):
    """K-tensor score (Sec. 6.1): the mean congruence over matched components.  R <= 8: the best
    of all R! matchings; larger R: greedy (repeatedly the largest remaining entry of Q, ties to
    the smallest row-major index).  Returns (score, perm) with component r of A matched to
    component perm[r] of B."""
    import itertools
    Q = congruence_matrix(A, B)
    R = Q.shape[0]
    if R <= 8:
        best, bperm = -1.0, None
        for perm in itertools.permutations(range(R)):   # lexicographic order: ties keep the first
            v = sum(Q[r, perm[r]] for r in range(R))
            if v > best:
                best, bperm = v, perm
        return best / R, list(bperm)
    perm = [-1] * R
    rows, cols = set(range(R)), set(range(R))
    tot = 0.0
    for _ in range(R):
        bv, br, bc = -1.0, -1, -1
        for r in sorted(rows):
            for c in sorted(cols):
                if Q[r, c] > bv:
                    bv, br, bc = Q[r, c], r, c
        perm[br] = bc
        tot += bv
        rows.discard(br)
        cols.discard(bc)
    return tot / R, perm
