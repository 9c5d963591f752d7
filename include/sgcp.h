/*
 * sgcp.h -- C ABI of the GB300 streaming-GCP library (libsgcp.so).
 *
 * Streaming Generalized CP decomposition (Phipps, Johnson, Kolda, arXiv
 * 2110.14514).  As each tensor slice X_t (a d-way tensor, d = 2..4) arrives,
 * the library fits its temporal weights s_t with the factor matrices held
 * fixed (Alg. 3, or the Gaussian least-squares solve of Sec. 5), then updates
 * the factor matrices A^(1..d) against the streaming objective of Sec. 4.2
 * (eq. gcp_stream_objective): the GCP loss of the new slice, the model-based
 * history penalty 1/2 sum_h w_h ||Mbar_h - M_h||^2 over a reservoir-sampled
 * window of earlier steps, and lambda/mu regularisation (Alg. 4), with ADAM
 * steps that are checkpointed and rolled back per epoch (Alg. 2).  Sparse
 * slices use stratified sampling of nonzeros and zeros (Alg. 5, Alg. 6).
 *
 * Conventions shared by every entry point:
 *  - Every function returns an sgcp_status and never throws or aborts.
 *  - "device" pointers are CUDA global-memory pointers on the context's
 *    device (for instance the data pointers of torch tensors); "host"
 *    pointers are ordinary CPU memory.  The caller owns every pointer it
 *    passes and must keep device inputs alive until the work queued on the
 *    context's stream has completed.  The library owns its own state, which
 *    it allocates at sgcp_create and frees at sgcp_destroy.
 *  - Floating-point arrays use the context's element type: double when
 *    params.precision == SGCP_PREC_F64, float otherwise.
 *  - Factor matrices A^(k) are row-major I_k x R (row i = R contiguous
 *    values), s is a vector of R values, dense slices are stored in C order
 *    (last index fastest), sparse slices are COO with 0-based int32
 *    coordinates, one row of ndim coordinates per nonzero.
 *  - Work is queued asynchronously on the stream given to sgcp_create.
 *    Argument errors are reported synchronously.  Errors detected on the
 *    device (bad coordinates, exhausted zero sampling, non-finite values)
 *    are latched into a device error word; sgcp_check / sgcp_stats read it
 *    (synchronising the stream) and from then on the context answers
 *    SGCP_ERR_STATE until it is destroyed.
 *  - One context must be used by one host thread at a time.
 *  - Inside a slice update the gradient and factor-update kernels of a solver
 *    chain are launched with programmatic stream serialization, each starting
 *    its independent set-up while the kernel before it finishes.  A library
 *    built with SGCP_BUILD_SERIAL=1 in the environment launches every kernel
 *    with full serialization instead (same arithmetic and results; the build
 *    kernel profilers replay).
 *
 * Limits: 2 <= ndim <= 4; rank R a multiple of 4 with 4 <= R <= 128; dense
 * slices need ndim <= 3; I_k * R < 2^31 for every mode; the product of the
 * dimensions fits in 63 bits.
 */
#ifndef SGCP_H
#define SGCP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SGCP_OK = 0,
    SGCP_ERR_ARG = 1,            /* invalid argument (reported synchronously) */
    SGCP_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    SGCP_ERR_OOM = 3,            /* device allocation failed */
    SGCP_ERR_SAMPLING_LIMIT = 4, /* a zero-sample slot found no zero within zero_attempt_cap tries */
    SGCP_ERR_TIMEOUT = 5,        /* a bounded device wait gave up */
    SGCP_ERR_NUMERIC = 6,        /* non-finite objective value */
    SGCP_ERR_STATE = 7,          /* the context latched an earlier error */
    SGCP_ERR_UNSUPPORTED = 8,    /* valid request outside the implemented limits */
    SGCP_ERR_DATA = 9            /* slice data invalid: coordinate out of range or duplicate */
} sgcp_status;

/* GCP losses f(x, m) (Sec. 2.2, eq. GCP_problem; log m evaluated as log(m + log_eps)). */
typedef enum {
    SGCP_LOSS_GAUSSIAN = 0,        /* (x - m)^2 */
    SGCP_LOSS_POISSON = 1,         /* m - x log m */
    SGCP_LOSS_BERNOULLI_ODDS = 2,  /* log(m + 1) - x log m */
    SGCP_LOSS_BERNOULLI_LOGIT = 3  /* log(1 + e^m) - x m */
} sgcp_loss;

typedef enum {
    SGCP_PREC_F32 = 0,          /* all arithmetic in float (reductions of losses in double) */
    SGCP_PREC_F64 = 1,          /* all arithmetic in double (dense slices only) */
    SGCP_PREC_BF16_MTTKRP = 2,  /* dense MTTKRP operands in bf16 on tensor cores, fp32 accumulate */
    SGCP_PREC_F16_MTTKRP = 3    /* dense MTTKRP operands in fp16 on tensor cores, fp32 accumulate */
} sgcp_precision;

typedef enum {
    SGCP_TEMPORAL_ADAM = 0,     /* Alg. 3 */
    SGCP_TEMPORAL_LSQ = 1       /* Gaussian least-squares solve (Sec. 5) */
} sgcp_temporal;

/* History term of the factor solve (Sec. 4.1). */
typedef enum {
    SGCP_HISTORY_MODEL = 0,     /* 1/2 sum_h w_h ||Mbar_h - M_h||^2, no slice kept (eq. gcp_stream_problem_2) */
    SGCP_HISTORY_SLICES = 1     /* sum_h w_h sum_i f(x_ih, m_ih) over the window's stored slices X_h with
                                   M_h = [[s_h; A]] (eq. gcp_stream_problem_1): the context keeps up to H
                                   slices on the device; ADAM factor solver only, no checkpoint */
} sgcp_history_kind;

typedef enum {
    SGCP_OPT_ADAM = 0,          /* Alg. 4 */
    SGCP_OPT_LBFGS = 1          /* projected L-BFGS on the exact objective (dense slices; not in the paper) */
} sgcp_optimizer;

/* OnlineGCP arguments (Table 1) and solver settings (Table 2).  Fill with
 * sgcp_params_default, then set the problem fields (ndim, dims, rank, loss). */
typedef struct {
    int32_t ndim;             /* d, number of slice modes (2..4) */
    int32_t rank;             /* R */
    int64_t dims[4];          /* I_1..I_d */
    int32_t loss;             /* sgcp_loss */
    int32_t precision;        /* sgcp_precision */
    double lower_bound;       /* l; NaN selects the loss default (0 for Poisson/odds, -inf otherwise) */
    double log_eps;           /* epsilon of log(m + eps) */
    int32_t H;                /* maximum history window size */
    int32_t temporal;         /* sgcp_temporal */
    double w, theta;          /* history weights w_h = w theta^(t-h) */
    double lambda, mu;        /* factor / temporal-weight regularisation */
    int64_t p, q;             /* gradient samples: nonzeros, zeros (sparse slices) */
    int64_t p_obj, q_obj;     /* objective samples: nonzeros, zeros (sparse slices) */
    double tol_w, tol_f;      /* epoch loop continues while the estimate exceeds tol */
    int32_t kappa_w, kappa_f; /* maximum epochs */
    int32_t tau_w, tau_f;     /* iterations per epoch */
    double alpha_w, alpha_f;  /* ADAM learning rates */
    double beta1, beta2, adam_eps;
    double alpha_decay;       /* learning-rate factor applied on a rejected epoch */
    int32_t zero_attempt_cap; /* attempts per zero-sample slot */
    int32_t optimizer;        /* sgcp_optimizer */
    int32_t lbfgs_mem;        /* L-BFGS memory */
    int32_t lbfgs_iters;      /* L-BFGS iterations per slice */
    int32_t sparse_cpl;       /* tuning: factor columns per lane in the sparse kernel (4, 8, 16; 0 = auto) */
    int32_t hot_rows;         /* tuning: rows per mode accumulated in shared memory by the sparse kernel
                                 (0..64; -1 = 4); results do not depend on it */
    int32_t history_kind;     /* SGCP_HISTORY_MODEL (default) or SGCP_HISTORY_SLICES */
    int32_t reserved;         /* must be 0 */
    uint64_t seed;            /* Philox4x32-10 key for every random draw */
} sgcp_params;

/* One slice.  Sparse: nnz COO entries (idx [nnz][ndim] int32, vals [nnz]).
 * Dense: vals holds the full slice in C order, idx is NULL.
 * on_host = 1 means idx / vals are host pointers; the call queues their copy to
 * the device on a copy stream of the context, ordered before every use of the
 * slice and after the work of the step before last, so that it can overlap the
 * previous step.  From pinned (page-locked) host memory the copy is
 * asynchronous: the host buffers must stay unchanged until the context stream
 * has passed the call (sgcp_check, sgcp_stats or a synchronisation of that
 * stream); pageable host memory may be reused once the call returns. */
typedef struct {
    int32_t is_sparse;
    int32_t on_host;
    int64_t nnz;
    const int32_t* idx;
    const void* vals;
} sgcp_slice;

/* Bits of sgcp_grad_opts.want */
#define SGCP_WANT_FACTORS 1   /* G^(k) = Y~_(k) Z_k diag(s), k = 1..d   (eq. gcp_grad_A) */
#define SGCP_WANT_TEMPORAL 2  /* g_s = Z' vec(Y~)                       (eq. gcp_grad_lambda) */
#define SGCP_WANT_LOSS 4      /* F~ = sum over samples of weight * f(x, m) (Alg. 5 sample sum) */

/* Sample sets: which Philox purpose pair a sparse draw uses (Alg. 5 / Alg. 6). */
#define SGCP_SAMPLES_FACTOR_GRAD 0
#define SGCP_SAMPLES_FACTOR_OBJ 1
#define SGCP_SAMPLES_TEMPORAL_GRAD 2
#define SGCP_SAMPLES_TEMPORAL_OBJ 3

typedef struct {
    int32_t want;             /* SGCP_WANT_* bits */
    int32_t sample_set;       /* SGCP_SAMPLES_*; the GRAD sets draw p + q samples, the OBJ sets p_obj + q_obj */
    int64_t t;                /* time index placed in the sample counter */
    uint32_t draw;            /* draw index placed in the sample counter */
    int32_t accumulate;       /* 0: outputs are overwritten; 1: results are added to them */
    const void* y_scale;      /* device scalar (element type) multiplying every y and f; NULL = 1 */
} sgcp_grad_opts;

typedef struct {
    int64_t t;                    /* slices processed */
    int64_t iter;                 /* factor-solver iteration counter i of Alg. 1 / Alg. 4 */
    double F_w, F_f;              /* final objective estimates of the last slice's two solvers */
    int32_t epochs_w, epochs_f;   /* epochs run in the last slice */
    uint32_t accept_w, accept_f;  /* bit e set when epoch e of the last slice was accepted */
    double alpha_w, alpha_f;      /* learning rates after the last slice */
    int32_t hist_len;             /* current history window size */
    int32_t error_bits;           /* device error word (0 = none) */
    int64_t kernels_launched;     /* kernels queued by this context so far (graph nodes included) */
    int32_t evals_f;              /* L-BFGS factor solver: objective evaluations of the last slice
                                     (the first point plus every line-search trial); ADAM: 0 */
    int32_t pad;
} sgcp_stats_t;
typedef sgcp_stats_t sgcp_step_stats;   /* the same record under its per-step name */

/* Device-memory provider for the state a context or a batch owns (the variables of Alg. 1 and
 * Table 1: factor matrices, Abar, ADAM moments and checkpoints, history window, Gram sums, the
 * sparse-slice hash and hot-row tables, host-slice staging, L-BFGS work vectors).  With it a
 * caller lets another memory manager -- for instance torch's caching allocator -- own that memory.
 *   alloc(bytes, user)  returns `bytes` of device memory on the current device, aligned to at
 *                       least 256 bytes, or NULL when it cannot (the library call then returns
 *                       SGCP_ERR_OOM; memory that is not 256-byte aligned is handed back and the
 *                       call returns SGCP_ERR_ARG);
 *   free(ptr, user)     releases a pointer that alloc returned.
 * Both are called on the host thread that calls the library: during sgcp_create /
 * sgcp_batch_create, at the first use of a lazily sized buffer (the hash and staging buffers of a
 * larger slice than before, the L-BFGS vectors, the batch's host-slice staging), and during
 * destroy.  Before it frees a buffer that queued work may still use, the library synchronises its
 * stream.  Every pointer obtained is freed by the time sgcp_destroy / sgcp_batch_destroy returns,
 * and a create call that fails frees what it obtained before returning. */
typedef struct {
    void* (*alloc)(size_t bytes, void* user);
    void (*free)(void* ptr, void* user);
    void* user;
} sgcp_allocator;

typedef struct sgcp_ctx sgcp_ctx;

/* Version string of the library (library plumbing: no passage of the paper). */
const char* sgcp_version(void);

/* Human-readable name of a status code (library plumbing: no passage of the paper). */
const char* sgcp_status_string(sgcp_status status);

/* Defaults of Table 2 of the paper (beta1 = 0.9, beta2 = 0.999, eps = 1e-8,
 * tau = 100, theta = 1, lambda = mu = 0) plus kappa_w = kappa_f = 5,
 * alpha_w = 0.1, alpha_f = 1e-3, tol = -inf, zero_attempt_cap = 64,
 * log_eps = 1e-10, alpha_decay = 0.1.  Returns SGCP_ERR_ARG if p is NULL. */
sgcp_status sgcp_params_default(sgcp_params* p);

/* Create a streaming context (Alg. 1, before its loop).
 *  params        problem and solver settings (copied).
 *  init_factors  device, ndim pointers to I_k x R initial factor matrices (copied).
 *  n_hist        size of the initial history window (0..H), hist_t (host, n_hist
 *                time indices, each < the first slice's t) and hist_s (device,
 *                n_hist x R temporal weights) describe it (Table 1).
 *  t0            time index of the last warm-start slice; the first sgcp_step is t0 + 1.
 *  allocator     host, copied: provider of every device buffer the context owns, or NULL for
 *                cudaMalloc / cudaFree (see sgcp_allocator).
 *  cuda_stream   cudaStream_t to queue work on (NULL = a stream the context creates).
 *  out           receives the context.
 * Errors: SGCP_ERR_ARG (bad parameters, an allocator without alloc or free),
 * SGCP_ERR_UNSUPPORTED (outside the limits above), SGCP_ERR_OOM, SGCP_ERR_CUDA. */
sgcp_status sgcp_create(const sgcp_params* params, const void* const* init_factors,
                        int32_t n_hist, const int64_t* hist_t, const void* hist_s,
                        int64_t t0, const sgcp_allocator* allocator, void* cuda_stream, sgcp_ctx** out);

/* Destroy a context and free its device state (synchronises its stream).  The end
 * of the stream of Alg. 1; library plumbing with no passage of its own.  NULL is a no-op. */
void sgcp_destroy(sgcp_ctx* ctx);

/* Message describing the most recent error of ctx ("" if none; library plumbing).
 * The string is owned by the context and valid until its next call or destruction. */
const char* sgcp_last_error(const sgcp_ctx* ctx);

/* Load a slice into the context: copies host data if on_host, checks
 * coordinates, builds the nonzero-membership hash used to reject zero-sample
 * candidates (Sec. 4.3) and the per-mode hot-row tables.  sgcp_gradient and
 * sgcp_step call this themselves when given a slice other than the one
 * loaded last (compared by pointers and nnz); call it explicitly after
 * changing the contents behind the same pointers. */
sgcp_status sgcp_ingest(sgcp_ctx* ctx, const sgcp_slice* X);

/* One stochastic (sparse) or exact (dense) GCP gradient evaluation, the
 * fused model -> loss derivative -> MTTKRP path (Sec. 2.2 eqs. gcp_grad_A and
 * gcp_grad_lambda; Alg. 6 sampling for sparse slices):
 *   G_out[k] (device, I_k x R)  <- Y~_(k) Z_k diag(s)        if SGCP_WANT_FACTORS
 *   gs_out   (device, R)        <- Z' vec(Y~)                if SGCP_WANT_TEMPORAL
 *   f_out    (device, 1 double) <- sum of weight * f(x, m)   if SGCP_WANT_LOSS
 * s (device, R) and A (device, ndim pointers, I_k x R) are the point of
 * evaluation.  History and regularisation terms are not included.  Outputs
 * not requested may be NULL.  s, A[k] and G_out[k] must be 16-byte aligned
 * (they are read or accumulated with 16-byte vector accesses; any cudaMalloc'd
 * or torch-allocated buffer is), else SGCP_ERR_ARG.  Asynchronous on the
 * context stream. */
sgcp_status sgcp_gradient(sgcp_ctx* ctx, const sgcp_slice* X, const void* s, const void* const* A,
                          const sgcp_grad_opts* opts, void* const* G_out, void* gs_out, double* f_out);

/* Materialise the coordinates of one sparse sample draw, the stratified
 * sample of Alg. 6 (GRAD sets) or of Alg. 5 (OBJ sets), Sec. 4.3: nonzeros
 * drawn uniformly, zeros by rejection against the nonzero hash (the same draw
 * sgcp_gradient makes with these arguments): coords_out (device int32,
 * [n][ndim]) with n = p + q (GRAD sets) or p_obj + q_obj (OBJ sets),
 * nonzero samples first; attempt_out (device int32 [n] or NULL) receives the
 * accepted attempt of each zero sample and -1 for nonzero samples. */
sgcp_status sgcp_sample_coords(sgcp_ctx* ctx, const sgcp_slice* X, int32_t sample_set, int64_t t,
                               uint32_t draw, int32_t* coords_out, int32_t* attempt_out);

/* The sparse gradient of sgcp_gradient (Sec. 2.2 eqs. gcp_grad_A and
 * gcp_grad_lambda over the stratified sample of Alg. 6) without a context
 * and without any device allocation.  The paper has no counterpart of this
 * calling form: it exists
 * for callers that cannot let a library allocate device memory -- for
 * instance a serving process that reserves its whole GPU memory budget at
 * start-up, or a latency-critical loop where a cudaMalloc, which may
 * synchronise the device, is not acceptable.
 *
 * It computes the same outputs as sgcp_gradient for a sparse slice (same
 * Philox sample draw, same weights), from: params (ndim, dims, rank, loss,
 * log_eps, p, q, p_obj, q_obj, zero_attempt_cap, sparse_cpl and seed are
 * read; precision must not be SGCP_PREC_F64), the COO slice (device: idx
 * [nnz][ndim] int32, vals [nnz] float), s (device, R floats), A (host array
 * of ndim device pointers to I_k x R float matrices), opts, and the outputs
 * G_out / gs_out / f_out as in sgcp_gradient (s, A[k], G_out[k] 16-byte
 * aligned, else SGCP_ERR_ARG).  err_out (device int32 or
 * NULL) is set to 0 and then receives the device error bits of this call
 * (coordinate out of range or duplicate: 1 or 2; zero sampling exhausted: 4).
 * A sample that lands on an out-of-range COO entry is dropped before any
 * factor or gradient row is touched, with or without err_out.
 * Work is queued on cuda_stream (NULL = legacy default stream).
 *
 * Its only scratch is a fixed 4 MiB device array (2^19 hash slots) inside
 * the library, which every GPU that loads the library holds until the
 * process exits.  Hence nnz is limited to 262144 (SGCP_ERR_UNSUPPORTED
 * beyond).  The first call on each device looks up that array's device
 * address (with the device current) and keeps it for the life of the
 * process; make this first call before any CUDA stream capture, and do not
 * use the entry point on a device across a cudaDeviceReset.  All calls share the array and each clears the part it
 * uses, so calls whose GPU work overlaps (other streams or host threads)
 * race on it and must be serialised by the caller.  No hot-row shared-memory
 * tables are used, so the summation order differs from sgcp_gradient's
 * within float rounding. */
sgcp_status sgcp_gradient_sparse_noalloc(const sgcp_params* params, int64_t nnz, const int32_t* idx,
                                         const float* vals, const float* s, const float* const* A,
                                         const sgcp_grad_opts* opts, float* const* G_out, float* gs_out,
                                         double* f_out, int32_t* err_out, void* cuda_stream);

/* Result of a warm start: the final estimate of the stacked objective, the epochs run, and bit e
 * set when epoch e was accepted. */
typedef struct {
    double F;
    int32_t epochs;
    uint32_t accept;
} sgcp_warm_stats;

/* Warm start (Sec. 4.4: the initial factor matrices come from a static fit of an initial set of
 * slices; Sec. 6: every experiment starts that way and lets those slices form the first history
 * window).  Fits the first n slices X[0..n-1] (host array of slices, each dense or each sparse,
 * device or host data as in sgcp_step) stacked as a (d+1)-way tensor whose last mode indexes the
 * slices, that mode's factor matrix S (n x R) holding the slices' temporal weights: GCP-SGD with
 * the factor solver's settings (kappa_f epochs of tau_f ADAM iterations at alpha_f, rollback of
 * rejected epochs, tol_f, lambda on every matrix of the stack including S), starting from the
 * context's current factors and S_init (device, n x R; NULL = all ones).  Dense slices use the
 * exact gradient and objective; sparse slices are sampled per slice (p + q gradient samples and
 * p_obj + q_obj objective samples each, slice h at time index h + 1).
 * Afterwards the context stands at t = n: its factor matrices are the fit, the history window
 * holds S_h of the slices that the reservoir rule of Alg. 1 keeps as h = 1..n enter in order,
 * s is S_n, and the next sgcp_step processes slice n + 1.  S_out (device, n x R, may be NULL)
 * receives S; stats_out (host, may be NULL) the result.
 * Needs a context that has processed no slice and was created without a history window.
 * Synchronises the context stream (the call returns when the fit is done). */
sgcp_status sgcp_warm_start(sgcp_ctx* ctx, int32_t n, const sgcp_slice* X, const void* S_init, void* S_out,
                            sgcp_warm_stats* stats_out);

/* Reconstruction loss of a slice at the model M = [[s; A]] (Sec. 6, eq. local_loss): out (host,
 * 2 doubles) receives sum_i f(x_i, m_i) and ||X||_F^2; their ratio is the local loss of a slice
 * at the factors of its own time step, and -- with the last step's factors -- the slice's term of
 * the global loss.  exact = 0: dense slices are summed over every entry, sparse slices estimated
 * with the objective sample set (p_obj + q_obj stratified samples at time index t, draw 0; Alg. 5
 * without the history and regularisation terms).  exact = 1: every entry, zeros included (for a
 * sparse slice the model is evaluated over the whole index space, which needs ndim <= 3).  s and
 * A as in sgcp_gradient.  Synchronises the context stream. */
sgcp_status sgcp_slice_loss(sgcp_ctx* ctx, const sgcp_slice* X, const void* s, const void* const* A, int32_t exact,
                            int64_t t, double* out);

/* K-tensor score (Sec. 6.1): the congruence between the rank-one components of two K-tensors with
 * nmodes factor matrices each (device, A[k] and B[k] both I_k x rank, row-major, element type
 * float for SGCP_PREC_F32 or double for SGCP_PREC_F64; the temporal mode may be one of them):
 * Q[r][c] = prod_k |cos(a_r^(k), b_c^(k))|, and the score = the mean of Q over the best matching
 * of components -- all rank! matchings for rank <= 8, greedy (largest remaining entry first)
 * above.  score_out (host) receives it, perm_out (host, rank int32, may be NULL) the matching
 * (component r of A to component perm_out[r] of B); 1 means the same components up to order and
 * scale.  1 <= nmodes <= 8, 1 <= rank <= 128.  Uses a small stream-ordered scratch allocation and
 * synchronises cuda_stream (NULL = the legacy default stream). */
sgcp_status sgcp_kruskal_score(int32_t nmodes, int32_t rank, const int64_t* dims, int32_t precision,
                               const void* const* A, const void* const* B, double* score_out, int32_t* perm_out,
                               void* cuda_stream);

/* Process the next slice: one pass of the loop body of Alg. 1 (temporal
 * solve, factor solve, reservoir history update, Abar <- A).  Asynchronous;
 * the whole solver sequence runs as CUDA graphs on the context stream. */
sgcp_status sgcp_step(sgcp_ctx* ctx, const sgcp_slice* X_t);

/* Copy the current factor matrices A^(k) (device, ndim pointers) and the last
 * temporal weights s_t (device, R) out of the context, i.e. the model Alg. 1
 * holds after its last slice; either may be NULL.
 * t_out (host, may be NULL) receives the index of the last processed slice.
 * Asynchronous on the context stream. */
sgcp_status sgcp_factors(sgcp_ctx* ctx, void* const* A_out, void* s_out, int64_t* t_out);

/* Copy the history window of Sec. 4.1 (the reservoir-sampled time indices h
 * and their temporal weights s_h): h_out (host, H int64 time indices) and s_out
 * (device, H x R weights, may be NULL); *n_out receives |window|.  h_out and
 * n_out are filled at once from the context's host-side window bookkeeping;
 * the s_out copy is asynchronous on the context stream. */
sgcp_status sgcp_history(sgcp_ctx* ctx, int64_t* h_out, void* s_out, int32_t* n_out);

/* Synchronise the context stream and return its latched device error status
 * (library plumbing: the device error word described above). */
sgcp_status sgcp_check(sgcp_ctx* ctx);

/* Synchronise and report solver statistics of the last slice: the objective
 * estimates of Alg. 3 and Alg. 4 (EstimateObjective, Alg. 5), the epochs each
 * ran and which were accepted, and the ADAM learning rates after the decays of
 * Alg. 3 / Alg. 4 (sgcp_stats_t above). */
sgcp_status sgcp_stats(sgcp_ctx* ctx, sgcp_stats_t* out);

/* Queue on the context stream, behind the work queued so far, a device-to-host
 * copy of the two objective estimates of the last processed slice: out[0] =
 * the temporal solver's F (EstimateObjective of Alg. 3 at its accepted point),
 * out[1] = the factor solver's (Alg. 4), the values sgcp_stats reports as F_w
 * and F_f.  out: host memory for 2 doubles, owned by the caller; with pinned
 * (page-locked) memory the call returns at once and the values are valid once
 * the context stream has passed this point (cudaStreamSynchronize on it, or
 * sgcp_check); with pageable memory the copy completes before the call
 * returns.  Lets a caller read every step's result without draining the GPU
 * between steps.  No device error check: sgcp_check reports latched errors. */
sgcp_status sgcp_objectives_async(sgcp_ctx* ctx, double* out);

/* Checkpoint (library plumbing; the state is that of Alg. 1 and Table 1): the
 * state that makes the stream resumable (t, i, Abar, s,
 * history window, factor-solver ADAM moments, learning rate).  sgcp_state_size
 * gives the byte size; export writes it to a host buffer, import restores it
 * into a context created with the same params.  Both synchronise. */
sgcp_status sgcp_state_size(const sgcp_ctx* ctx, size_t* size);
sgcp_status sgcp_state_export(sgcp_ctx* ctx, void* host_buf, size_t size);
sgcp_status sgcp_state_import(sgcp_ctx* ctx, const void* host_buf, size_t size);

/* ------------------------------------------------------------------------
 * Batched streams.  Many independent streams, each its own OnlineGCP problem
 * (its own dims, rank, loss and solver parameters), advanced together: one
 * sgcp_batch_step call runs the loop body of Alg. 1 (Alg. 3 temporal ADAM
 * epochs, Alg. 4 factor ADAM epochs with the history penalty, Alg. 2
 * checkpoints, Abar <- A, reservoir update) for every stream in ONE
 * persistent kernel launch, captured in a CUDA graph.  Blocks take work
 * units (tile boxes of a slice gradient, Gram-matrix row chunks, factor-update
 * row chunks) from per-stream phase counters, so streams of very different
 * size advance independently and the GPU stays full.  Each stream computes
 * what sgcp_step computes for it, up to the order of float additions.
 *
 * Limits per stream: dense 3-way slices, precision SGCP_PREC_F32, temporal
 * solver SGCP_TEMPORAL_ADAM, optimizer SGCP_OPT_ADAM, rank R a multiple of 4
 * with 4 <= R <= 64, kappa_w, kappa_f <= 32.
 *
 * Unit tile shapes come from an autotuner: for each key (shape bucket
 * ceil(I_k / 32) per mode, R, loss) it times candidate shapes of the slice
 * gradient unit and keeps the fastest; the table can be read back and passed
 * to later batches.
 * ------------------------------------------------------------------------ */
typedef struct sgcp_batch sgcp_batch;

typedef struct {
    int32_t bucket[3];   /* ceil(I_k / 32), k = 1..3 */
    int32_t rank;
    int32_t loss;        /* sgcp_loss */
    int32_t b1log;       /* tile of 2^b1log i1 rows x 2^(6 - b1log) i2 rows x 32 i3 columns, 2 <= b1log <= 4 */
    int32_t n1, n2;      /* tiles per unit along i1 and i2: 2^b1log n1 <= 32, 2^(6 - b1log) n2 <= 32 */
    float us;            /* measured time of one slice-gradient pass in microseconds (0 = not timed) */
} sgcp_tune_entry;

typedef struct {
    int32_t autotune;              /* 1: time candidates for every key missing from the table */
    int32_t tune_reps;             /* timed launches per candidate (best kept); default 3 */
    const sgcp_tune_entry* table;  /* host array of known entries, or NULL */
    int32_t n_table;
    int32_t grid_blocks;           /* persistent blocks; 0 = every block that fits on the device */
    int64_t spin_limit;            /* empty polls before a block gives up (SGCP_ERR_TIMEOUT); 0 = default 2^22 */
} sgcp_batch_opts;

/* Defaults of sgcp_batch_opts (library plumbing): autotune off, tune_reps 3,
 * no table, grid_blocks 0 (every resident block), spin_limit 0 (2^22).
 * Returns SGCP_ERR_ARG if opts is NULL. */
sgcp_status sgcp_batch_opts_default(sgcp_batch_opts* opts);

/* Create a batch of n_streams independent streams, each as sgcp_create would
 * (Alg. 1 before its loop).  params: host array of n_streams parameter sets.  init_factors: host array
 * of 3 * n_streams device pointers (stream s, mode k at [3 s + k]), each an
 * I_k x R float matrix copied into the batch.  opts may be NULL (defaults).
 * allocator and cuda_stream as in sgcp_create.  Streams start at t = 0 with empty history. */
sgcp_status sgcp_batch_create(int32_t n_streams, const sgcp_params* params, const void* const* init_factors,
                              const sgcp_batch_opts* opts, const sgcp_allocator* allocator, void* cuda_stream,
                              sgcp_batch** out);

/* Destroy a batch and free its device state (synchronises its stream; library
 * plumbing).  NULL is a no-op. */
void sgcp_batch_destroy(sgcp_batch* batch);

/* Message describing the most recent error of the batch ("" if none; library plumbing). */
const char* sgcp_batch_last_error(const sgcp_batch* batch);

/* Advance every stream by one slice: the loop body of Alg. 1 for each stream
 * (see above).  X: host array of n_streams pointers to
 * dense float slices in C order (I_1 x I_2 x I_3 of that stream); device
 * pointers when x_on_host = 0, host pointers when x_on_host = 1 (the call then
 * queues their copies into one of two library-owned staging buffers, used in
 * turn, on a copy stream of the batch, so that they overlap the step before;
 * the batch stream waits for them).  The caller keeps device inputs alive,
 * and pinned host inputs unchanged, until the step has completed; pageable
 * host inputs may be reused once the call returns.
 * Asynchronous on the batch stream. */
sgcp_status sgcp_batch_step(sgcp_batch* batch, const void* const* X, int32_t x_on_host);

/* Stream s: copy the model Alg. 1 holds after its last slice, its factor
 * matrices (3 device pointers, entries may be NULL)
 * and temporal weights (device, R floats, may be NULL); t_out (host) receives
 * its last slice index.  Asynchronous on the batch stream. */
sgcp_status sgcp_batch_factors(sgcp_batch* batch, int32_t s, void* const* A_out, void* s_out, int64_t* t_out);

/* Synchronise; statistics of stream s after its last slice (as sgcp_stats: the
 * Alg. 3 / Alg. 4 objective estimates, epochs and learning rates). */
sgcp_status sgcp_batch_stats(sgcp_batch* batch, int32_t s, sgcp_stats_t* out);

/* Queue on the batch stream, behind the work queued so far, the read-back of
 * every stream's two objective estimates after its last slice (the F_w and F_f
 * of sgcp_batch_stats; EstimateObjective of Alg. 3 and 4): out[2 s] and
 * out[2 s + 1] for stream s.  out: host memory for 2 x (number of streams)
 * doubles, owned by the caller; with pinned memory the call returns at once
 * and the values are valid once the batch stream has passed this point
 * (sgcp_batch_check or a synchronisation of the stream).  One gather kernel
 * and one copy; the gather buffer is allocated at the first call. */
sgcp_status sgcp_batch_objectives_async(sgcp_batch* batch, double* out);

/* Synchronise and return the latched device error status of the batch
 * (library plumbing). */
sgcp_status sgcp_batch_check(sgcp_batch* batch);

/* The tuning table of the batch (library plumbing: tile shapes of the
 * gradient unit, no passage of the paper; known plus newly timed entries): up to cap
 * entries to out (host); *n_out receives the table size. */
sgcp_status sgcp_batch_tune_table(const sgcp_batch* batch, sgcp_tune_entry* out, int32_t cap, int32_t* n_out);

/* The unit tile shape stream s runs with (its table entry; library plumbing). */
sgcp_status sgcp_batch_unit_config(const sgcp_batch* batch, int32_t s, sgcp_tune_entry* out);

#ifdef __cplusplus
}
#endif

#endif /* SGCP_H */
