"""Seeded synthetic streams for streaming GCP (shared by the tests, the oracle and the bench).

This package only makes data: it holds none of the method's arithmetic (no
loss, gradient, sampling or solver code).  Planted tensors are multiplied out
here with numpy to synthesise observations, as the paper's synthetic
experiments do (arXiv 2110.14514, Sec. 6.1); the method itself never calls
this package.

Workloads (five seeded recipes, each with the shapes and distributions the
paper's experiments use):

  dense_gaussian_2way   20 x 30 slices, R = 4, N(0,1) factors, s_t ~ U[0.5, 1.5],
                        N(0, 0.1^2) noise, Gaussian loss
  dense_poisson_3way    100^3 slices, R = 16, U[0,1] factors and weights,
                        x ~ Poisson(m), Poisson loss
  sparse_binary_zipf    10000 x 5000 x 2000 slices with 1e6 unique nonzeros,
                        coordinates per mode ~ truncated Zipf(1.2) mapped
                        through a seeded permutation, values 1, R = 32,
                        Bernoulli-logit loss
  dense_gaussian_3way   256^3 slices, R = 64, N(0,1) factors, s_t ~ U[0.5, 1.5],
                        noise sd 1% of the RMS of the planted slice
  batched_streams       64 streams, I_k ~ U{32..160}, R ~ U{8, 16, ..., 64},
                        Gaussian (even stream) / Poisson (odd stream)

Seeding: every draw comes from ``numpy.random.default_rng([seed, stream, role, t])``
so that slice t of a stream is reproducible on its own.
"""
import numpy as np

__all__ = [
    "WORKLOADS", "workload", "truth", "dense_slice", "sparse_slice", "init_factors",
    "zipf_coords", "batched_stream_shapes",
]

_ROLE_TRUTH, _ROLE_SLICE, _ROLE_INIT, _ROLE_PERM, _ROLE_SHAPE = 0, 1, 2, 3, 4

WORKLOADS = {
    "dense_gaussian_2way": dict(seed=1, kind="dense", dims=(20, 30), rank=4, T=50, loss="gaussian",
                                H=10, factor_dist="normal", s_dist=(0.5, 1.5), noise=("abs", 0.1),
                                init_dist=("normal", 1.0), dtype="f64"),
    "dense_poisson_3way": dict(seed=2, kind="dense", dims=(100, 100, 100), rank=16, T=200, loss="poisson",
                               H=20, factor_dist="uniform", s_dist=(0.0, 1.0), noise=("poisson", None),
                               init_dist=("uniform", 1.0), dtype="f32"),
    "sparse_binary_zipf": dict(seed=3, kind="sparse", dims=(10000, 5000, 2000), rank=32, T=100,
                               loss="bernoulli_logit", nnz=1_000_000, zipf=1.2, p=100_000, q=100_000,
                               p_obj=100_000, q_obj=100_000, init_dist=("normal", 0.5), dtype="f32"),
    "dense_gaussian_3way": dict(seed=4, kind="dense", dims=(256, 256, 256), rank=64, T=50, loss="gaussian",
                                H=10, factor_dist="normal", s_dist=(0.5, 1.5), noise=("rel", 0.01),
                                init_dist=("normal", 1.0), dtype="f32"),
    "batched_streams": dict(seed=5, kind="batched", n_streams=64, dim_range=(32, 160),
                            rank_choices=(8, 16, 24, 32, 40, 48, 56, 64), T=100, dtype="f32"),
}


def workload(name):
    return dict(WORKLOADS[name])


def _rng(seed, stream, role, t=0):
    return np.random.default_rng([int(seed), int(stream), int(role), int(t)])


def _np_dtype(cfg):
    return np.float64 if cfg.get("dtype") == "f64" else np.float32


def truth(cfg, stream=0):
    """Planted factor matrices of a dense workload (float64)."""
    g = _rng(cfg["seed"], stream, _ROLE_TRUTH)
    if cfg["factor_dist"] == "normal":
        return [g.standard_normal((n, cfg["rank"])) for n in cfg["dims"]]
    return [g.random((n, cfg["rank"])) for n in cfg["dims"]]


def _planted(A, s):
    """sum_j s_j a_j^(1) o ... o a_j^(d), C order (data synthesis only)."""
    dims = [a.shape[0] for a in A]
    rest = A[1]
    for a in A[2:]:
        rest = (rest[:, None, :] * a[None, :, :]).reshape(-1, a.shape[1])
    return ((A[0] * s[None, :]) @ rest.T).reshape(dims)


def dense_slice(cfg, t, stream=0, A_true=None):
    """Slice t (t >= 1) of a dense workload: (X_t in the workload dtype, s_t float64)."""
    A = truth(cfg, stream) if A_true is None else A_true
    g = _rng(cfg["seed"], stream, _ROLE_SLICE, t)
    lo, hi = cfg["s_dist"]
    s = lo + (hi - lo) * g.random(cfg["rank"])
    M = _planted(A, s)
    kind, level = cfg["noise"]
    if kind == "abs":
        X = M + level * g.standard_normal(M.shape)
    elif kind == "rel":
        X = M + level * np.sqrt(np.mean(M * M)) * g.standard_normal(M.shape)
    elif kind == "poisson":
        X = g.poisson(np.maximum(M, 0.0)).astype(np.float64)
    else:
        raise ValueError(kind)
    return np.ascontiguousarray(X.astype(_np_dtype(cfg))), s


def zipf_coords(g, n, a, perm):
    """n draws from the Zipf(a) law truncated to {0..I-1} (inverse CDF), relabelled by perm."""
    I = perm.shape[0]
    pmf = np.arange(1, I + 1, dtype=np.float64) ** (-a)
    cdf = np.cumsum(pmf)
    cdf /= cdf[-1]
    r = np.searchsorted(cdf, g.random(n), side="right")
    return perm[np.minimum(r, I - 1)]


def sparse_slice(cfg, t, stream=0, nnz=None, dims=None):
    """Slice t of the sparse workload: COO (idx int32 (nnz, d), vals float32).

    Coordinates are drawn mode-independently from Zipf(a) and relabelled by a
    per-mode seeded permutation; draws repeat until exactly nnz distinct
    coordinates exist, kept in order of first occurrence.
    """
    dims = tuple(cfg["dims"] if dims is None else dims)
    nnz = cfg["nnz"] if nnz is None else nnz
    gp = _rng(cfg["seed"], stream, _ROLE_PERM)
    perms = [gp.permutation(n) for n in dims]
    g = _rng(cfg["seed"], stream, _ROLE_SLICE, t)
    coords = np.zeros((0, len(dims)), np.int64)
    batch = max(2 * nnz, 1024)
    while True:
        new = np.stack([zipf_coords(g, batch, cfg["zipf"], perms[k]) for k in range(len(dims))], axis=1)
        coords = np.concatenate([coords, new])
        key = np.zeros(coords.shape[0], np.uint64)
        for k, n in enumerate(dims):
            key = key * np.uint64(n) + coords[:, k].astype(np.uint64)
        _, first = np.unique(key, return_index=True)
        if first.size >= nnz:
            keep = np.sort(first)[:nnz]
            idx = np.ascontiguousarray(coords[keep].astype(np.int32))
            return idx, np.ones(nnz, np.float32)
        batch = nnz


def init_factors(cfg, stream=0, dims=None, rank=None):
    """Initial factor matrices for the solver, independent of the planted truth."""
    dims = cfg["dims"] if dims is None else dims
    rank = cfg["rank"] if rank is None else rank
    g = _rng(cfg["seed"], stream, _ROLE_INIT)
    kind, scale = cfg["init_dist"]
    dt = _np_dtype(cfg)
    if kind == "normal":
        return [np.ascontiguousarray((scale * g.standard_normal((n, rank))).astype(dt)) for n in dims]
    return [np.ascontiguousarray((scale * g.random((n, rank))).astype(dt)) for n in dims]


def batched_stream_shapes(cfg):
    """Per-stream (dims, rank, loss) of the batched workload."""
    out = []
    lo, hi = cfg["dim_range"]
    for s in range(cfg["n_streams"]):
        g = _rng(cfg["seed"], s, _ROLE_SHAPE)
        dims = tuple(int(x) for x in g.integers(lo, hi + 1, size=3))
        rank = int(g.choice(cfg["rank_choices"]))
        loss = "gaussian" if s % 2 == 0 else "poisson"
        out.append((dims, rank, loss))
    return out


def batched_stream_cfg(cfg, s):
    """Dense-workload recipe of stream s of the batched workload."""
    dims, rank, loss = batched_stream_shapes(cfg)[s]
    if loss == "gaussian":
        base = dict(factor_dist="normal", s_dist=(0.5, 1.5), noise=("rel", 0.01), init_dist=("normal", 1.0))
    else:
        base = dict(factor_dist="uniform", s_dist=(0.0, 1.0), noise=("poisson", None), init_dist=("uniform", 1.0))
    return dict(base, seed=cfg["seed"] * (1 << 32) + s, kind="dense", dims=dims, rank=rank, loss=loss,
                T=cfg["T"], H=10, dtype="f32")
