"""Python binding of libsgcp.so, the GB300 streaming-GCP library (arXiv 2110.14514).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  The C entry points are exported under their C names
(``sgcp_create``, ``sgcp_step``, ``sgcp_gradient``, ...) with ctypes
signatures; ``Context`` wraps one ``sgcp_ctx`` and takes torch tensors, whose
device pointers and CUDA stream it passes to the library.

There is no CPU fallback.  Importing this package loads the shared library
and raises ``ImportError`` if it has not been built
(``python paper_2110_14514_gb300/build.py``).
"""
import ctypes
import math
import os

from ctypes import POINTER, c_double, c_int32, c_int64, c_size_t, c_uint32, c_uint64, c_void_p, c_char_p

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsgcp.so")

# ----------------------------------------------------------------------------- constants (sgcp.h)
OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_SAMPLING_LIMIT, ERR_TIMEOUT, ERR_NUMERIC, ERR_STATE, ERR_UNSUPPORTED, ERR_DATA = range(10)
LOSS = {"gaussian": 0, "poisson": 1, "bernoulli_odds": 2, "bernoulli_logit": 3}
PREC_F32, PREC_F64, PREC_BF16_MTTKRP, PREC_F16_MTTKRP = 0, 1, 2, 3
TEMPORAL_ADAM, TEMPORAL_LSQ = 0, 1
OPT_ADAM, OPT_LBFGS = 0, 1
HISTORY_MODEL, HISTORY_SLICES = 0, 1
WANT_FACTORS, WANT_TEMPORAL, WANT_LOSS = 1, 2, 4
SAMPLES_FACTOR_GRAD, SAMPLES_FACTOR_OBJ, SAMPLES_TEMPORAL_GRAD, SAMPLES_TEMPORAL_OBJ = 0, 1, 2, 3


class sgcp_params(ctypes.Structure):
    _fields_ = [
        ("ndim", c_int32), ("rank", c_int32), ("dims", c_int64 * 4), ("loss", c_int32), ("precision", c_int32),
        ("lower_bound", c_double), ("log_eps", c_double), ("H", c_int32), ("temporal", c_int32),
        ("w", c_double), ("theta", c_double), ("lambda_", c_double), ("mu", c_double),
        ("p", c_int64), ("q", c_int64), ("p_obj", c_int64), ("q_obj", c_int64),
        ("tol_w", c_double), ("tol_f", c_double), ("kappa_w", c_int32), ("kappa_f", c_int32),
        ("tau_w", c_int32), ("tau_f", c_int32), ("alpha_w", c_double), ("alpha_f", c_double),
        ("beta1", c_double), ("beta2", c_double), ("adam_eps", c_double), ("alpha_decay", c_double),
        ("zero_attempt_cap", c_int32), ("optimizer", c_int32), ("lbfgs_mem", c_int32), ("lbfgs_iters", c_int32),
        ("sparse_cpl", c_int32), ("hot_rows", c_int32), ("history_kind", c_int32), ("reserved", c_int32),
        ("seed", c_uint64),
    ]


class sgcp_slice(ctypes.Structure):
    _fields_ = [("is_sparse", c_int32), ("on_host", c_int32), ("nnz", c_int64), ("idx", c_void_p),
                ("vals", c_void_p)]


class sgcp_grad_opts(ctypes.Structure):
    _fields_ = [("want", c_int32), ("sample_set", c_int32), ("t", c_int64), ("draw", c_uint32),
                ("accumulate", c_int32), ("y_scale", c_void_p)]


class sgcp_stats_t(ctypes.Structure):
    _fields_ = [("t", c_int64), ("iter", c_int64), ("F_w", c_double), ("F_f", c_double),
                ("epochs_w", c_int32), ("epochs_f", c_int32), ("accept_w", c_uint32), ("accept_f", c_uint32),
                ("alpha_w", c_double), ("alpha_f", c_double), ("hist_len", c_int32), ("error_bits", c_int32),
                ("kernels_launched", c_int64), ("evals_f", c_int32), ("pad", c_int32)]


class sgcp_warm_stats(ctypes.Structure):
    _fields_ = [("F", c_double), ("epochs", c_int32), ("accept", c_uint32)]


class sgcp_tune_entry(ctypes.Structure):
    _fields_ = [("bucket", c_int32 * 3), ("rank", c_int32), ("loss", c_int32), ("b1log", c_int32),
                ("n1", c_int32), ("n2", c_int32), ("us", ctypes.c_float)]


class sgcp_batch_opts(ctypes.Structure):
    _fields_ = [("autotune", c_int32), ("tune_reps", c_int32), ("table", POINTER(sgcp_tune_entry)),
                ("n_table", c_int32), ("grid_blocks", c_int32), ("spin_limit", c_int64)]


ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, c_size_t, c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_void_p)


class sgcp_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", c_void_p)]


_PTRS = POINTER(c_void_p)

# (name, restype, argtypes) of every entry point declared in include/sgcp.h
SIGNATURES = [
    ("sgcp_version", c_char_p, []),
    ("sgcp_status_string", c_char_p, [c_int32]),
    ("sgcp_params_default", c_int32, [POINTER(sgcp_params)]),
    ("sgcp_create", c_int32, [POINTER(sgcp_params), _PTRS, c_int32, POINTER(c_int64), c_void_p, c_int64,
                              POINTER(sgcp_allocator), c_void_p, POINTER(c_void_p)]),
    ("sgcp_destroy", None, [c_void_p]),
    ("sgcp_last_error", c_char_p, [c_void_p]),
    ("sgcp_ingest", c_int32, [c_void_p, POINTER(sgcp_slice)]),
    ("sgcp_gradient", c_int32, [c_void_p, POINTER(sgcp_slice), c_void_p, _PTRS, POINTER(sgcp_grad_opts), _PTRS,
                                c_void_p, c_void_p]),
    ("sgcp_sample_coords", c_int32, [c_void_p, POINTER(sgcp_slice), c_int32, c_int64, c_uint32, c_void_p,
                                     c_void_p]),
    ("sgcp_step", c_int32, [c_void_p, POINTER(sgcp_slice)]),
    ("sgcp_warm_start", c_int32, [c_void_p, c_int32, POINTER(sgcp_slice), c_void_p, c_void_p,
                                  POINTER(sgcp_warm_stats)]),
    ("sgcp_slice_loss", c_int32, [c_void_p, POINTER(sgcp_slice), c_void_p, _PTRS, c_int32, c_int64,
                                  POINTER(c_double)]),
    ("sgcp_kruskal_score", c_int32, [c_int32, c_int32, POINTER(c_int64), c_int32, _PTRS, _PTRS, POINTER(c_double),
                                     POINTER(c_int32), c_void_p]),
    ("sgcp_factors", c_int32, [c_void_p, _PTRS, c_void_p, POINTER(c_int64)]),
    ("sgcp_history", c_int32, [c_void_p, POINTER(c_int64), c_void_p, POINTER(c_int32)]),
    ("sgcp_check", c_int32, [c_void_p]),
    ("sgcp_stats", c_int32, [c_void_p, POINTER(sgcp_stats_t)]),
    ("sgcp_objectives_async", c_int32, [c_void_p, c_void_p]),
    ("sgcp_batch_objectives_async", c_int32, [c_void_p, c_void_p]),
    ("sgcp_state_size", c_int32, [c_void_p, POINTER(c_size_t)]),
    ("sgcp_state_export", c_int32, [c_void_p, c_void_p, c_size_t]),
    ("sgcp_state_import", c_int32, [c_void_p, c_void_p, c_size_t]),
    ("sgcp_gradient_sparse_noalloc", c_int32, [POINTER(sgcp_params), c_int64, c_void_p, c_void_p, c_void_p, _PTRS,
                                               POINTER(sgcp_grad_opts), _PTRS, c_void_p, c_void_p, c_void_p,
                                               c_void_p]),
    ("sgcp_batch_opts_default", c_int32, [POINTER(sgcp_batch_opts)]),
    ("sgcp_batch_create", c_int32, [c_int32, POINTER(sgcp_params), _PTRS, POINTER(sgcp_batch_opts),
                                    POINTER(sgcp_allocator), c_void_p, POINTER(c_void_p)]),
    ("sgcp_batch_destroy", None, [c_void_p]),
    ("sgcp_batch_last_error", c_char_p, [c_void_p]),
    ("sgcp_batch_step", c_int32, [c_void_p, _PTRS, c_int32]),
    ("sgcp_batch_factors", c_int32, [c_void_p, c_int32, _PTRS, c_void_p, POINTER(c_int64)]),
    ("sgcp_batch_stats", c_int32, [c_void_p, c_int32, POINTER(sgcp_stats_t)]),
    ("sgcp_batch_check", c_int32, [c_void_p]),
    ("sgcp_batch_tune_table", c_int32, [c_void_p, POINTER(sgcp_tune_entry), c_int32, POINTER(c_int32)]),
    ("sgcp_batch_unit_config", c_int32, [c_void_p, c_int32, POINTER(sgcp_tune_entry)]),
]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libsgcp.so is not built ({LIB_PATH}); run python paper_2110_14514_gb300/build.py")
    lib = ctypes.CDLL(LIB_PATH)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()
for _name, _res, _args in SIGNATURES:
    globals()[_name] = getattr(lib, _name)


class SgcpError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        name = lib.sgcp_status_string(status).decode()
        super().__init__(f"{name}: {msg}" if msg else name)


def _check(status, ctx=None, batch=None):
    if status != OK:
        if ctx:
            msg = lib.sgcp_last_error(ctx).decode()
        elif batch:
            msg = lib.sgcp_batch_last_error(batch).decode()
        else:
            msg = ""
        raise SgcpError(status, msg)


def params(dims, rank, loss="gaussian", **kw):
    """sgcp_params filled with the library defaults, then dims / rank / loss and any field in kw
    (``lam`` sets lambda)."""
    p = sgcp_params()
    _check(lib.sgcp_params_default(ctypes.byref(p)))
    p.ndim = len(dims)
    for k, n in enumerate(dims):
        p.dims[k] = int(n)
    p.rank = int(rank)
    p.loss = LOSS[loss] if isinstance(loss, str) else int(loss)
    for k, v in kw.items():
        if k == "lam":
            k = "lambda_"
        if k == "lower":
            k = "lower_bound"
        if v is None and k == "lower_bound":
            v = math.nan
        setattr(p, k, v)
    return p


def _ptr(t):
    return c_void_p(t.data_ptr()) if t is not None else c_void_p(0)


def _ptr_array(ts):
    arr = (c_void_p * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = t.data_ptr() if t is not None else 0
    return arr


def make_slice(X=None, idx=None, vals=None):
    """sgcp_slice for a dense tensor X or COO (idx int32 [nnz, d], vals); host tensors set on_host."""
    sl = sgcp_slice()
    if X is not None:
        sl.is_sparse = 0
        sl.on_host = 0 if X.is_cuda else 1
        sl.nnz = X.numel()
        sl.idx = None
        sl.vals = X.data_ptr()
        keep = (X,)
    else:
        sl.is_sparse = 1
        sl.on_host = 0 if vals.is_cuda else 1
        sl.nnz = vals.numel()
        sl.idx = idx.data_ptr() if idx.numel() else None
        sl.vals = vals.data_ptr() if vals.numel() else None
        keep = (idx, vals)
    return sl, keep


class Allocator:
    """A device-memory provider for the library (sgcp_allocator) built from two Python callables:
    alloc(nbytes) -> device address (int) or 0 / None when it cannot, and free(address).  The
    callables must stay valid while a context or batch created with this object exists (the
    object keeps them alive; keep the object)."""

    def __init__(self, alloc, free):
        def _alloc(nbytes, user):
            try:
                return alloc(int(nbytes)) or None
            except Exception:
                return None

        def _free(ptr, user):
            try:
                free(int(ptr))
            except Exception:
                pass
        self._alloc_cb = ALLOC_FN(_alloc)
        self._free_cb = FREE_FN(_free)
        self.c = sgcp_allocator(self._alloc_cb, self._free_cb, None)


def torch_allocator(stream):
    """torch's caching allocator as the provider of a context's or batch's device memory; blocks
    are allocated for `stream` (the stream the library queues its work on)."""
    import torch

    def alloc(nbytes):
        return torch.cuda.caching_allocator_alloc(nbytes, stream=stream)

    return Allocator(alloc, torch.cuda.caching_allocator_delete)


def _alloc_arg(allocator, stream):
    if allocator is None:
        return None, None
    if allocator == "torch":
        allocator = torch_allocator(stream)
    return allocator, ctypes.byref(allocator.c)


class Context:
    """One streaming-GCP context (sgcp_create ... sgcp_destroy) on the current CUDA device.
    allocator: None (the library calls cudaMalloc), "torch" (torch's caching allocator owns the
    context's device memory) or an Allocator."""

    def __init__(self, p, init_factors, hist_t=(), hist_s=None, t0=0, stream=None, allocator=None):
        import torch
        self.p = p
        self.ndim = p.ndim
        self.R = p.rank
        self.dims = [p.dims[k] for k in range(p.ndim)]
        self.dtype = torch.float64 if p.precision == PREC_F64 else torch.float32
        for a, n in zip(init_factors, self.dims):
            assert a.is_cuda and a.dtype == self.dtype and a.is_contiguous() and tuple(a.shape) == (n, self.R)
        # The library works on its own stream; every call orders it after the
        # caller's current stream and the caller's stream after it.
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self._torch = torch
        self._enter()
        ht = (c_int64 * max(len(hist_t), 1))(*[int(h) for h in hist_t])
        out = c_void_p()
        self.allocator, aref = _alloc_arg(allocator, self.stream)
        st = lib.sgcp_create(ctypes.byref(p), _ptr_array(init_factors), len(hist_t), ht,
                             _ptr(hist_s), int(t0), aref, c_void_p(self.stream.cuda_stream), ctypes.byref(out))
        _check(st)
        self.h = out
        self._keep = None
        self._leave()

    def _enter(self):
        self.stream.wait_stream(self._torch.cuda.current_stream())

    def _leave(self):
        self._torch.cuda.current_stream().wait_stream(self.stream)

    def close(self):
        if getattr(self, "h", None):
            lib.sgcp_destroy(self.h)
            self.h = None
        self._keep = None           # destroy waited for the stream: the last inputs may go

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _slice(self, X=None, idx=None, vals=None):
        sl, keep = make_slice(X, idx, vals)
        self._keep = keep
        return sl

    def ingest(self, X=None, idx=None, vals=None):
        sl = self._slice(X, idx, vals)
        self._enter()
        _check(lib.sgcp_ingest(self.h, ctypes.byref(sl)), self.h)
        self._leave()

    def step(self, X=None, idx=None, vals=None):
        sl = self._slice(X, idx, vals)
        self._enter()
        _check(lib.sgcp_step(self.h, ctypes.byref(sl)), self.h)
        self._leave()

    def warm_start(self, slices, S_init=None):
        """Static fit of the first n slices stacked along a new last mode (sgcp_warm_start).
        slices: dense tensors, or (idx, vals) pairs.  Returns (S as an n x R device tensor,
        {"F", "epochs", "accept"})."""
        import torch
        n = len(slices)
        arr = (sgcp_slice * n)()
        keep = []
        for h, x in enumerate(slices):
            sl, k = make_slice(X=x) if not isinstance(x, (tuple, list)) else make_slice(idx=x[0], vals=x[1])
            arr[h] = sl
            keep.append(k)
        S = torch.empty((n, self.R), dtype=self.dtype, device="cuda")
        st = sgcp_warm_stats()
        self._keep = keep
        self._enter()
        code = lib.sgcp_warm_start(self.h, n, arr, _ptr(S_init), _ptr(S), ctypes.byref(st))
        self._leave()
        _check(code, self.h)
        return S, {"F": st.F, "epochs": st.epochs, "accept": st.accept}

    def slice_loss(self, s, A, X=None, idx=None, vals=None, exact=False, t=1):
        """(sum_i f(x_i, m_i), ||X||_F^2) of a slice at M = [[s; A]] (sgcp_slice_loss); their ratio is
        the local / global reconstruction loss of Sec. 6."""
        out = (c_double * 2)()
        sl = self._slice(X, idx, vals)
        self._enter()
        code = lib.sgcp_slice_loss(self.h, ctypes.byref(sl), _ptr(s), _ptr_array(A), int(bool(exact)), int(t), out)
        self._leave()
        _check(code, self.h)
        return out[0], out[1]

    def gradient(self, s, A, X=None, idx=None, vals=None, want=WANT_FACTORS | WANT_TEMPORAL | WANT_LOSS,
                 sample_set=SAMPLES_FACTOR_GRAD, t=1, draw=0, G=None, gs=None, f=None, accumulate=False,
                 y_scale=None):
        """One fused gradient evaluation; returns (G list, gs, f) as device tensors."""
        import torch
        dev = s.device
        if want & WANT_FACTORS and G is None:
            G = [torch.empty((n, self.R), dtype=self.dtype, device=dev) for n in self.dims]
        if want & WANT_TEMPORAL and gs is None:
            gs = torch.empty(self.R, dtype=self.dtype, device=dev)
        if want & WANT_LOSS and f is None:
            f = torch.empty(1, dtype=torch.float64, device=dev)
        opts = sgcp_grad_opts(want=want, sample_set=sample_set, t=int(t), draw=int(draw),
                              accumulate=int(bool(accumulate)), y_scale=_ptr(y_scale))
        sl = self._slice(X, idx, vals)
        self._enter()
        st = lib.sgcp_gradient(self.h, ctypes.byref(sl), _ptr(s), _ptr_array(A), ctypes.byref(opts),
                               _ptr_array(G) if G is not None else None, _ptr(gs), _ptr(f))
        self._leave()
        _check(st, self.h)
        return G, gs, f

    def sample_coords(self, idx, vals, sample_set, t, draw, n):
        import torch
        coords = torch.empty((n, self.ndim), dtype=torch.int32, device=vals.device)
        att = torch.empty(n, dtype=torch.int32, device=vals.device)
        sl = self._slice(None, idx, vals)
        self._enter()
        _check(lib.sgcp_sample_coords(self.h, ctypes.byref(sl), sample_set, int(t), int(draw), _ptr(coords),
                                      _ptr(att)), self.h)
        self._leave()
        return coords, att

    def factors(self):
        import torch
        A = [torch.empty((n, self.R), dtype=self.dtype, device="cuda") for n in self.dims]
        s = torch.empty(self.R, dtype=self.dtype, device="cuda")
        t = c_int64()
        self._enter()
        _check(lib.sgcp_factors(self.h, _ptr_array(A), _ptr(s), ctypes.byref(t)), self.h)
        self._leave()
        return A, s, t.value

    def history(self):
        import torch
        H = max(self.p.H, 1)
        h = (c_int64 * H)()
        s = torch.empty((H, self.R), dtype=self.dtype, device="cuda")
        n = c_int32()
        self._enter()
        _check(lib.sgcp_history(self.h, h, _ptr(s), ctypes.byref(n)), self.h)
        self._leave()
        return [h[i] for i in range(n.value)], s[: n.value]

    def check(self):
        _check(lib.sgcp_check(self.h), self.h)

    def stats(self):
        st = sgcp_stats_t()
        code = lib.sgcp_stats(self.h, ctypes.byref(st))
        _check(code, self.h)
        return {f: getattr(st, f) for f, _ in sgcp_stats_t._fields_}

    def objectives_async(self, out):
        """Queue the copy of the last slice's (F_w, F_f) into out (a pinned host float64 tensor of
        2 elements) on the context stream; valid after the stream reaches it (sgcp_objectives_async)."""
        assert out.dtype == self._torch.float64 and out.numel() >= 2 and not out.is_cuda and out.is_contiguous()
        _check(lib.sgcp_objectives_async(self.h, c_void_p(out.data_ptr())), self.h)

    def state_export(self):
        n = c_size_t()
        _check(lib.sgcp_state_size(self.h, ctypes.byref(n)), self.h)
        buf = ctypes.create_string_buffer(n.value)
        _check(lib.sgcp_state_export(self.h, buf, n), self.h)
        return buf.raw

    def state_import(self, data):
        buf = ctypes.create_string_buffer(data, len(data))
        _check(lib.sgcp_state_import(self.h, buf, len(data)), self.h)


def kruskal_score(A, B, stream=None):
    """K-tensor score of Sec. 6.1 between two lists of device factor matrices (same shapes, float32
    or float64): (score, perm) with component r of A matched to component perm[r] of B."""
    import torch
    n = len(A)
    R = A[0].shape[1]
    dims = (c_int64 * n)(*[a.shape[0] for a in A])
    prec = PREC_F64 if A[0].dtype == torch.float64 else PREC_F32
    score = c_double()
    perm = (c_int32 * R)()
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(lib.sgcp_kruskal_score(n, R, dims, prec, _ptr_array(A), _ptr_array(B), ctypes.byref(score), perm,
                                  c_void_p(st.cuda_stream)))
    return score.value, list(perm)


def _entry_dict(e):
    return {"bucket": tuple(e.bucket), "rank": e.rank, "loss": e.loss, "b1log": e.b1log, "n1": e.n1, "n2": e.n2,
            "us": e.us}


class Batch:
    """Many independent streams advanced together (sgcp_batch_create ... sgcp_batch_destroy): one
    persistent kernel per time step runs every stream's Alg. 1 loop body."""

    def __init__(self, plist, init_factors, autotune=False, tune_reps=3, table=None, grid_blocks=0,
                 spin_limit=0, stream=None, allocator=None):
        import torch
        self._torch = torch
        self.n = len(plist)
        self.plist = list(plist)
        self.dims = [[p.dims[k] for k in range(3)] for p in plist]
        self.R = [p.rank for p in plist]
        for s, (p, A) in enumerate(zip(plist, init_factors)):
            assert len(A) == 3
            for a, n in zip(A, self.dims[s]):
                assert a.is_cuda and a.dtype == torch.float32 and a.is_contiguous() and tuple(a.shape) == (n, p.rank)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        arr = (sgcp_params * self.n)(*plist)
        flat = [a for A in init_factors for a in A]
        opts = sgcp_batch_opts()
        _check(lib.sgcp_batch_opts_default(ctypes.byref(opts)))
        opts.autotune = int(bool(autotune))
        opts.tune_reps = int(tune_reps)
        opts.grid_blocks = int(grid_blocks)
        opts.spin_limit = int(spin_limit)
        self._table = None
        if table:
            self._table = (sgcp_tune_entry * len(table))()
            for i, e in enumerate(table):
                t = self._table[i]
                for k in range(3):
                    t.bucket[k] = e["bucket"][k]
                t.rank, t.loss, t.b1log, t.n1, t.n2, t.us = e["rank"], e["loss"], e["b1log"], e["n1"], e["n2"], e["us"]
            opts.table = self._table
            opts.n_table = len(table)
        self.stream.wait_stream(torch.cuda.current_stream())
        out = c_void_p()
        self.allocator, aref = _alloc_arg(allocator, self.stream)
        _check(lib.sgcp_batch_create(self.n, arr, _ptr_array(flat), ctypes.byref(opts), aref,
                                     c_void_p(self.stream.cuda_stream), ctypes.byref(out)))
        self.h = out
        self._keep = None
        torch.cuda.current_stream().wait_stream(self.stream)

    def close(self):
        if getattr(self, "h", None):
            lib.sgcp_batch_destroy(self.h)
            self.h = None
        self._keep = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def step(self, X):
        """X: one dense float32 slice per stream, all device tensors or all host (CPU) tensors."""
        assert len(X) == self.n
        on_host = not X[0].is_cuda
        for x in X:
            assert x.dtype == self._torch.float32 and x.is_contiguous() and x.is_cuda != on_host
        self._keep = X
        self.stream.wait_stream(self._torch.cuda.current_stream())
        st = lib.sgcp_batch_step(self.h, _ptr_array(X), int(on_host))
        self._torch.cuda.current_stream().wait_stream(self.stream)
        _check(st, batch=self.h)

    def factors(self, s):
        torch = self._torch
        A = [torch.empty((n, self.R[s]), dtype=torch.float32, device="cuda") for n in self.dims[s]]
        sv = torch.empty(self.R[s], dtype=torch.float32, device="cuda")
        t = c_int64()
        self.stream.wait_stream(torch.cuda.current_stream())
        _check(lib.sgcp_batch_factors(self.h, s, _ptr_array(A), _ptr(sv), ctypes.byref(t)), batch=self.h)
        torch.cuda.current_stream().wait_stream(self.stream)
        return A, sv, t.value

    def stats(self, s):
        st = sgcp_stats_t()
        _check(lib.sgcp_batch_stats(self.h, s, ctypes.byref(st)), batch=self.h)
        return {f: getattr(st, f) for f, _ in sgcp_stats_t._fields_}

    def objectives_async(self, out):
        """Queue the read-back of every stream's (F_w, F_f) into out (a pinned host float64 tensor
        of 2 x n elements) on the batch stream (sgcp_batch_objectives_async)."""
        t = self._torch
        assert out.dtype == t.float64 and out.numel() >= 2 * self.n and not out.is_cuda and out.is_contiguous()
        _check(lib.sgcp_batch_objectives_async(self.h, c_void_p(out.data_ptr())), batch=self.h)

    def check(self):
        _check(lib.sgcp_batch_check(self.h), batch=self.h)

    def tune_table(self):
        n = c_int32()
        _check(lib.sgcp_batch_tune_table(self.h, None, 0, ctypes.byref(n)), batch=self.h)
        arr = (sgcp_tune_entry * max(n.value, 1))()
        _check(lib.sgcp_batch_tune_table(self.h, arr, n.value, ctypes.byref(n)), batch=self.h)
        return [_entry_dict(arr[i]) for i in range(n.value)]

    def unit_config(self, s):
        e = sgcp_tune_entry()
        _check(lib.sgcp_batch_unit_config(self.h, s, ctypes.byref(e)), batch=self.h)
        return _entry_dict(e)
