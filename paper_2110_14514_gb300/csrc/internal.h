// Internal launcher interfaces between the kernel files and the C ABI layer.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "solver_dev.cuh"

namespace sgcp {

// Launches kern<<<grid, block, smem, st>>>(args...) with programmatic stream serialization: the
// kernel may start while the previous kernel in the stream runs, so it must call grid_dep_wait()
// before it touches anything that kernel writes or reads.
template <typename... P, typename... Args>
inline cudaError_t launch_after_prev(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                     Args&&... args) {
#ifdef SGCP_NO_GRID_DEP
    kern<<<grid, block, smem, st>>>(static_cast<Args&&>(args)...);
    return cudaGetLastError();
#else
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<Args&&>(args)...);
#endif
}

// Arguments of the fused sparse sample -> model -> y -> MTTKRP kernel.
struct SparseGradArgs {
    const SliceDesc* slice;          // device descriptor (graph path) or nullptr
    SliceDesc inline_slice;          // used when slice == nullptr
    int ndim;
    int R;
    int64_t dims[4];
    const float* A[4];
    const float* s;
    float* G[4];                     // SGCP_WANT_FACTORS outputs (accumulated into)
    float* gs;                       // SGCP_WANT_TEMPORAL output (accumulated into)
    double* f;                       // SGCP_WANT_LOSS output (accumulated into)
    const unsigned long long* hkeys; // nonzero-membership hash (open addressing)
    int hlog2;                       // log2 of the table size
    const int32_t* hot[4];           // per-mode row -> hot slot (-1 = not hot)
    const int32_t* hot_rows;         // [ndim][kMaxHot] slot -> row
    int nhot;                        // slots per mode (0 disables privatisation)
    uint32_t key0, key1;             // Philox key
    uint32_t draw;
    uint32_t pur_nz, pur_z;
    int64_t p, q;                    // requested sample counts
    int all_nnz;                     // 1: visit every nonzero once with weight 1, no zeros
    int cap;                         // attempts per zero slot
    int want;                        // SGCP_WANT_* bits
    int loss;
    float eps;
    const float* y_scale;            // device scalar or nullptr
    int* err;                        // device error word
    const int32_t* skip;             // device flag: nonzero -> kernel does nothing
    int32_t* coords_out;             // sample-coordinate dump mode (nullptr otherwise)
    int32_t* attempt_out;
    int tstep_on;                    // fuse the temporal ADAM step into the last block
    TemporalStep<float> tstep;
    int cpl;                         // columns per lane (4, 8, 16; 0 = default for R)
    int f_minus_zero;                // loss: add f(x, m) - f(0, m) per sample (the nonzeros' part of an exact loss)
    int overlap;                     // host: launch with launch_after_prev (a kernel of a solve's chain)
    float* zero_buf;                 // cleared after grid_dep_wait (the next factor update's Gram sums) or nullptr
    int zero_n;
    // Deferred ADAM step on s (Alg. 3): with pend_on every block forms, after grid_dep_wait, the s
    // it uses from the state (s, u, v) in pend (rate = pend.rate) and the previous gradient sum
    // pend_g (pend_apply = 0: the state unchanged); block 0 writes that state to pend_out.  So the
    // step of one temporal-gradient kernel runs at the start of the next, with no last-block
    // election at the end of the first.
    int pend_on, pend_apply;
    TemporalStep<float> pend;        // s, u, v in; st unused
    const float* pend_g;
    float *pend_s_out, *pend_u_out, *pend_v_out;
};

// Arguments of the dense fused gradient kernels (3-way tiled and the 2-way path).
template <typename T>
struct DenseGradArgs {
    const SliceDesc* slice;  // device descriptor or nullptr; vals = T[prod dims], C order
    SliceDesc inline_slice;  // used when slice == nullptr
    int ndim;
    int R;
    int64_t dims[3];
    const T* A[3];
    const T* s;
    T* G[3];
    T* gs;
    double* f;
    int want;
    int loss;
    T eps;
    const T* y_scale;
    const int32_t* skip;
    int tstep_on;            // fuse the temporal ADAM step into the last block
    TemporalStep<T> tstep;
    const void* xmap;        // tensor-core path: device CUtensorMap of the slice (nullptr = plain loads)
};
// (the CUDA-core dense kernels read a slice whose vals pointer is nullptr as the all-zero slice)

struct IngestArgs {
    SliceDesc slice;
    int ndim;
    int64_t dims[4];
    unsigned long long* hkeys;
    int hlog2;
    int32_t* counts;        // concatenated per-mode row counts (sum I_k)
    int32_t* hot;           // concatenated per-mode row -> slot (sum I_k), preset to -1
    int32_t* hot_rows;      // [ndim][kMaxHot]
    int64_t row_off[4];
    int64_t sub_stride;     // histogram every sub_stride-th nonzero
    int nhot;
    int* err;
};

// Launchers (return cudaGetLastError()).
cudaError_t launch_ingest(const IngestArgs& a, int64_t nnz_host, cudaStream_t st, int64_t* launches);
cudaError_t launch_sparse_grad(const SparseGradArgs& a, int64_t total_samples, cudaStream_t st, int64_t* launches);
cudaError_t launch_sample_coords(const SparseGradArgs& a, int64_t total_samples, cudaStream_t st, int64_t* launches);
// Hash-only ingest into a caller-provided table of 2^hlog2 slots (cleared to all ones).
cudaError_t launch_hash_build(const SliceDesc& sd, int ndim, const int64_t* dims, unsigned long long* keys, int hlog2,
                              int* err, cudaStream_t st);
template <typename T>
cudaError_t launch_dense_grad(const DenseGradArgs<T>& a, cudaStream_t st, int64_t* launches);
// Tensor-core (tcgen05) dense gradient, 3-way slices, R % 16 == 0 and R <= 64;
// bf16 selects BF16 MTTKRP operands, otherwise FP16.
cudaError_t launch_dense_grad_tc(const DenseGradArgs<float>& a, bool bf16, int* err, cudaStream_t st,
                                 int64_t* launches);
// Encode the TMA tensor map of a dense I1 x I2 x I3 float slice for the tensor-core kernel (boxes of
// 32 i3 x 16 i2 x 8 i1, 128-byte swizzle) into a 128-byte host buffer; false when the slice does
// not qualify (I3 % 4 != 0, a misaligned base) or the driver offers no encoder.
bool encode_x_map(void* map128, const float* X, int64_t I1, int64_t I2, int64_t I3);
// Copy a 128-byte tensor map into device memory (128-byte aligned) on a stream.
cudaError_t launch_write_map(void* dst_dev, const void* map128, cudaStream_t st, int64_t* launches);

// ---------------------------------------------------------------------------
// Solver kernels (k_solver.cu)
// ---------------------------------------------------------------------------

template <typename T>
struct GramArgs {
    int ndim;
    int R;
    int64_t dims[4];
    int64_t row_off[4];       // row offsets of each mode in the concatenated factor buffer
    const T* A;               // concatenated factors, rows of R
    const T* Abar;
    int npairs;
    int sel_u[6], sel_v[6];
    T* part;                  // per-block partial sums [npairs][ndim][nblk][R][R]
    int nblk;                 // blocks per mode (grid.x)
    int64_t rows_per_block;   // multiple of the staging depth
    double* out;              // [npairs][ndim][R][R] (written by launch_gram's reduce step)
    const int32_t* skip;
};

// Gram partial-sum geometry for a problem: blocks per mode and rows per block.
void gram_geometry(int64_t max_dim, int* nblk, int64_t* rows_per_block);

template <typename T>
struct FactorUpdateArgs {
    int ndim;
    int R;
    int64_t nrows;            // sum I_k
    int64_t row_off[4];
    T* A;
    const T* Abar;
    T* G;
    T* u;
    T* v;
    const T* B;               // [ndim][R][R]  (Gamma_k * S_H) or nullptr
    const T* C;               // [ndim][R][R]  ((Gamma_k - Gammabar_k) * S_H) or nullptr
    const int32_t* hist_len;  // device: history terms apply when *hist_len > 0
    double lam;
    double beta1, beta2, eps, lower;
    const double* rate;       // bias-corrected learning rate of this iteration (see k_epoch_begin)
    const int32_t* skip;
    int grad_only;            // 1: store the full gradient g in G and leave A, u, v untouched
    // Optional (FP32, R <= 32), buffers of [2][ndim][R][R] floats (A'A, D'A):
    //   gprev: Gram sums of the factors this update starts from (written by the previous update);
    //          when set, B_k and C_k are formed from them and SH instead of read from B, C;
    //   gacc:  zero on entry; receives the Grams of the rows this update writes;
    //   gzero: cleared by the last block (ticket tk) once every block has read gprev (or nullptr
    //          when the kernel between two updates clears it).
    const float* gprev;
    float* gacc;
    float* gzero;
    const double* SH;
    SolverState* tk;
    int overlap;              // host: launch with launch_after_prev when the FP32 row kernel applies
};

template <typename T>
cudaError_t launch_gram(const GramArgs<T>& a, int64_t nrows, cudaStream_t st, int64_t* launches);
// B_k = Gamma_k * S_H, C_k = (Gamma_k - Gammabar_k) * S_H from grams [pair][ndim][R][R]: P_n = A'A at
// pair 0, E_n = D'A at pair e_pair.
template <typename T>
cudaError_t launch_hist_coeffs(int ndim, int R, const double* grams, int e_pair, const double* SH,
                               const int32_t* hist_len, T* B, T* C, const int32_t* skip, cudaStream_t st,
                               int64_t* launches);
template <typename T>
cudaError_t launch_factor_update(const FactorUpdateArgs<T>& a, cudaStream_t st, int64_t* launches);


// Solver bookkeeping.
cudaError_t launch_solver_init(SolverState* st, double alpha, int reset_counter, cudaStream_t stream,
                               int64_t* launches);
// Alg. 3/4 loop test and the epoch's per-iteration learning rates rates[j], j < tau.
// zero (nzero floats, optional) is cleared as well: a buffer the epoch's first kernel sums into.
cudaError_t launch_epoch_begin(SolverState* st, double tol, double* rates, int tau, double beta1, double beta2,
                               cudaStream_t stream, int64_t* launches, float* zero = nullptr, int nzero = 0);
template <typename T>
cudaError_t launch_epoch_end(SolverState* st, int64_t n, T* a, T* u, T* v, T* a_o, T* u_o, T* v_o, int tau,
                             double decay, double beta1, double beta2, cudaStream_t stream, int64_t* launches);
template <typename T>
cudaError_t launch_adam_reset(int64_t n, const T* a, T* u, T* v, T* a_o, T* u_o, T* v_o, int zero_a, T* a_zero,
                              cudaStream_t stream, int64_t* launches);

// Objective finishing terms.
// Temporal: F_new += mu/2 ||s||^2; if set_cur, F_cur = F_new.
template <typename T>
cudaError_t launch_obj_finish_w(SolverState* st, const T* s, int R, double mu, int set_cur, int* err,
                                const int32_t* skip, cudaStream_t stream, int64_t* launches);
// Factor: F_new += 1/2 <S_H, telescoped history Gram sum> + lambda/2 sum ||A||^2.
// grams: [6][ndim][R][R] for pairs (A,A), (Abar,Abar), (Abar,A), (D,D), (D,A), (Abar,D).
cudaError_t launch_obj_finish_f(SolverState* st, int ndim, int R, const double* grams, const double* SH,
                                const int32_t* hist_len, double lam, int set_cur, int* err, const int32_t* skip,
                                cudaStream_t stream, int64_t* launches);

// S_H = sum_h w theta^(t-h) s_h s_h' over the window (double R x R).
template <typename T>
cudaError_t launch_history_SH(int R, const T* s_hist, const int64_t* h_dev, const int32_t* hist_len,
                              const SliceDesc* slice, double w, double theta, double* SH, cudaStream_t stream,
                              int64_t* launches);

// Least-squares temporal solve: (Gamma + mu/2 I) s = rhs, s <- max(s, l), Gamma = *_n P_n.
template <typename T>
cudaError_t launch_lsq_solve(int ndim, int R, const double* P, const T* rhs, double mu, double lower, T* s,
                             double* work, int* err, cudaStream_t stream, int64_t* launches);

// Write a slice descriptor into device memory (by-value kernel argument, so
// no host buffer has to outlive the call).
cudaError_t launch_write_desc(SliceDesc* dst, SliceDesc val, cudaStream_t stream, int64_t* launches);
// History slot update after step t: slot <- (t, s_t), window length <- len.
template <typename T>
cudaError_t launch_hist_update(int R, T* s_hist, int64_t* h_dev, int32_t* hist_len, int slot, int64_t t, int len,
                               const T* s, cudaStream_t stream, int64_t* launches);

// ---------------------------------------------------------------------------
// Projected L-BFGS factor solver, driven on the device (k_solver.cu).  The
// iteration's scalars live in LbfgsState; one slice's solve is captured in the
// step graph with the line search as a WHILE conditional node whose body the
// Armijo test ends (no host round trip).
// ---------------------------------------------------------------------------
constexpr int kLbfgsSlots = 65;   // lbfgs_mem <= 64 live pairs plus one candidate slot

struct LbfgsState {
    double F;        // objective at the current iterate x
    double step;     // trial step of the current line search
    double gamma;    // s'y / y'y of the newest stored pair (initial Hessian scaling)
    int32_t npairs;  // stored pairs (order[0..npairs), oldest first)
    int32_t trial;   // trials made in the current line search
    int32_t done;    // set when a line search found no acceptable step: later iterations do nothing
    int32_t accepted;
    int32_t iters;   // accepted iterations of this solve
    int32_t evals;   // objective evaluations of this solve
    int32_t order[kLbfgsSlots];
    double rho[kLbfgsSlots];
};

template <typename T>
struct LbfgsArgs {
    LbfgsState* ls;
    SolverState* sf;    // F_new holds the objective of the last evaluation
    T* A;               // the context's factors (the evaluation point)
    const T* G;         // full gradient at A (written by the evaluation)
    T* x;               // current iterate
    T* g;               // gradient at x
    T* pd;              // search direction H g
    T* const* S;        // device table of kLbfgsSlots pair vectors s
    T* const* Y;        // device table of kLbfgsSlots pair vectors y
    int64_t n;          // sum I_k * R
    int m;              // memory (live pairs kept)
    double lower;       // projection bound l
};

// After the first evaluation: x <- A, g <- G, F <- F(A), empty memory.
template <typename T>
cudaError_t launch_lbfgs_begin(const LbfgsArgs<T>& a, cudaStream_t st, int64_t* launches);
// pd <- H g (two-loop recursion); step <- 1 for the line search.  Nothing once the solve stopped.
template <typename T>
cudaError_t launch_lbfgs_direction(const LbfgsArgs<T>& a, cudaStream_t st, int64_t* launches);
// Trial point A <- max(x - step pd, l).
template <typename T>
cudaError_t launch_lbfgs_trial(const LbfgsArgs<T>& a, cudaStream_t st, int64_t* launches);
// Armijo test of the evaluated trial point: on rejection halves the step and sets the line
// search's WHILE handle to 1 (another trial, at most 30), else to 0.
template <typename T>
cudaError_t launch_lbfgs_armijo(const LbfgsArgs<T>& a, cudaGraphConditionalHandle h, cudaStream_t st,
                                int64_t* launches);
// After the line search: store the pair, move to the trial point; or restore x and stop.
template <typename T>
cudaError_t launch_lbfgs_update(const LbfgsArgs<T>& a, cudaStream_t st, int64_t* launches);
// Report the solve like an epoch summary: F_cur <- F, epoch <- iterations.
cudaError_t launch_lbfgs_finish(LbfgsState* ls, SolverState* sf, cudaStream_t st, int64_t* launches);

// Warm start (stacked static fit): F_new += lambda/2 ||W||^2 over n elements; F_cur <- F_new if set_cur.
template <typename T>
cudaError_t launch_reg_objective(SolverState* st, const T* W, int64_t n, double lam, int set_cur, int* err,
                                 const int32_t* skip, cudaStream_t stream, int64_t* launches);

// ---------------------------------------------------------------------------
// Evaluation metrics (k_score.cu): reconstruction losses and the K-tensor score of Sec. 6
// ---------------------------------------------------------------------------
// *out += sum_i x_i^2 over n elements.
template <typename T>
cudaError_t launch_sum_squares(const T* x, int64_t n, double* out, cudaStream_t st, int64_t* launches);
// Congruence of two K-tensors (nm modes, I_k x R factor matrices A[k], B[k], element T): per-mode
// cross-Grams C = [nm][R][R], column norms^2 na, nb = [nm][R] (scratch), then score and perm.
template <typename T>
cudaError_t launch_congruence(int nm, int R, const int64_t* dims, const T* const* A, const T* const* B,
                              double* C, double* na, double* nb, double* score, int32_t* perm, cudaStream_t st);

// Stored-slice history: per-step slot weights / draw bases / skip flags, and the skip flags after
// each epoch test (inactive slot or finished solver).
template <typename T>
cudaError_t launch_hist_slots_begin(SliceDesc* desc, T* wts, int32_t* skip, const int32_t* hist_len,
                                    const int64_t* h_dev, const SliceDesc* cur, double w, double theta, int H,
                                    uint32_t per_step, cudaStream_t st, int64_t* launches);
cudaError_t launch_hist_slots_skip(int32_t* skip, const int32_t* hist_len, const int32_t* done, int H,
                                   cudaStream_t st, int64_t* launches);

// Small helpers.
template <typename T>
cudaError_t launch_copy(T* dst, const T* src, int64_t n, cudaStream_t stream, int64_t* launches);

}  // namespace sgcp

namespace sgcp {

// ---------------------------------------------------------------------------
// Batched streams (k_batch.cu): many independent OnlineGCP streams with dense
// 3-way FP32 slices, advanced by one persistent kernel per time step.
// ---------------------------------------------------------------------------
constexpr int kBatchMaxR = 64;      // largest rank of a batched stream
constexpr int kBatchThreads = 256;
constexpr int kBatchGramRows = 64;  // rows of one Gram-chunk unit
constexpr int kBatchUpdRows = 32;   // rows of one factor-update unit

// Per-stream description: read-only while a step runs.
struct BatchStream {
    int R, loss;
    int P, PF0;                    // phases of one step; first factor phase
    int dims[3], row_off[3], nrows, N;
    int b1log, n1, n2;             // unit tile: 2^b1log i1 rows x 2^(5-b1log) i2 rows, n1 x n2 tiles per unit
    int nb1, nb2, nb3, n_box;      // units of the slice gradient
    int gch[3], n_gram;            // 64-row Gram chunks per mode
    int uch[3], n_upd;             // 32-row factor-update chunks per mode
    int kappa_w, tau_w, kappa_f, tau_f;
    float eps, lower;
    double tol_w, tol_f, alpha_w, alpha_f, beta1, beta2, adam_eps, decay, w, theta, lam, mu;
    float *A, *Abar, *G, *u, *v, *u_o, *v_o, *a_o;     // N each (modes concatenated)
    float *s, *s_u, *s_v, *s_uo, *s_vo, *s_ao, *gs;    // R each
    float* s_hist;                 // [H][R]
    int64_t* h_dev;                // [H]
    int32_t* hist_len;
    double* SH;                    // [R][R]
    double* grams;                 // [6][3][R][R]
    float* gpart;                  // [n_gram][6][R][R] Gram-chunk partial sums
    float *Bc, *Cc;                // [3][R][R] history coefficients
    SolverState *st_w, *st_f;
    double *rates_w, *rates_f;     // [tau_w], [tau_f]
};

// Per-stream inputs of one step (written before each launch).
struct BatchStepEntry {
    const float* X;                // dense slice, C order
    int64_t t;                     // time index of the slice
    int32_t slot, len;             // history slot to overwrite after the step (-1 = none), new window length
    int32_t hist_on;               // window non-empty during this step
    int32_t pad;
};

// Per-stream scheduling words.
struct BatchCtl {
    unsigned long long claim;      // (phase << 32) | next unclaimed unit
    int32_t done;                  // units of the current phase completed
    int32_t pad;
};

struct BatchArgs {
    const BatchStream* S;
    const BatchStepEntry* E;
    BatchCtl* ctl;
    const int32_t* order;          // streams in scheduling priority order
    int nS;
    int* finished;                 // streams that completed the step
    int* err;
    long long spin_limit;          // empty polls before a block gives up (ERRB_TIMEOUT)
};

size_t batch_smem_bytes();
int batch_blocks_per_sm();
cudaError_t launch_batch_begin(BatchStepEntry* dE, const BatchStepEntry* host_entries, int n, BatchCtl* ctl, int nS,
                               int* finished, cudaStream_t st, int64_t* launches);
cudaError_t launch_batch_step(const BatchArgs& a, int grid, cudaStream_t st, int64_t* launches);
// Autotuner timing launch: blocks x (factor-gradient unit blockIdx % n_box) of one stream description.
cudaError_t launch_batch_units(const BatchStream* S_dev, const BatchStepEntry* E_dev, int n_box, int blocks,
                               cudaStream_t st);

}  // namespace sgcp
