// C ABI of the batched-streams mode: many independent OnlineGCP streams
// (dense 3-way FP32 slices of uneven shape, rank and loss) advanced by one
// persistent kernel per time step (k_batch.cu), captured in a CUDA graph;
// per-stream device state carved from one allocation; the unit-shape
// autotuner.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "dense_tile.cuh"
#include "internal.h"
#include "sgcp.h"

using namespace sgcp;

struct sgcp_batch {
    int nS = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<sgcp_params> P;
    std::vector<BatchStream> hS;
    BatchStream* dS = nullptr;
    BatchStepEntry* dE = nullptr;
    BatchCtl* ctl = nullptr;
    int32_t* dorder = nullptr;
    int* finished = nullptr;
    int* err = nullptr;
    void* arena = nullptr;
    // host-slice staging: two buffers used in turn, one region per stream in each, filled on
    // copy_stream so that the copies of one step's slices overlap the step before it
    float* xstage[2] = {nullptr, nullptr};
    std::vector<int64_t> xoff;
    int64_t xstage_floats = 0;
    int xnext = 0;                         // buffer of the next staged step
    bool xused[2] = {false, false};        // buffer holds slices that queued work may read
    cudaStream_t copy_stream = nullptr;    // created with the first staged step
    cudaEvent_t ev_xused[2] = {nullptr, nullptr};   // end of the work queued while a buffer was current
    cudaEvent_t ev_xstaged = nullptr;
    double* fout = nullptr;                // [nS][2] objective estimates gathered for the host
    std::vector<std::vector<int64_t>> hist_t;
    std::vector<int64_t> t;
    std::vector<BatchStepEntry> hE;
    cudaGraphExec_t graph = nullptr;
    int grid = 0;
    long long spin_limit = 1LL << 22;
    std::vector<sgcp_tune_entry> table;
    std::vector<int> cfg;                  // table index of each stream's unit shape
    std::string last_error;
    sgcp_status sticky = SGCP_OK;
    int64_t launches = 0;
    sgcp_allocator ualloc{};               // caller's device-memory provider (used when custom_alloc)
    bool custom_alloc = false;
};

namespace {

sgcp_status bfail(sgcp_batch* b, sgcp_status st, const std::string& msg) {
    if (b) b->last_error = msg;
    return st;
}

sgcp_status bcuda(sgcp_batch* b, cudaError_t e, const char* what) {
    if (b) {
        b->last_error = std::string(what) + ": " + cudaGetErrorString(e);
        b->sticky = SGCP_ERR_CUDA;
    }
    return e == cudaErrorMemoryAllocation ? SGCP_ERR_OOM : SGCP_ERR_CUDA;
}

// Device allocation of batch state: through the caller's allocator when one was given at
// sgcp_batch_create (NULL on failure or misalignment), else cudaMalloc.
template <typename P>
bool balloc(sgcp_batch* b, P** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b->custom_alloc) {
        void* q = b->ualloc.alloc(bytes, b->ualloc.user);
        if (q && (reinterpret_cast<uintptr_t>(q) & 255) != 0) {
            b->ualloc.free(q, b->ualloc.user);
            q = nullptr;
        }
        *p = (P*)q;
        return q != nullptr;
    }
    void* q = nullptr;
    if (cudaMalloc(&q, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    *p = (P*)q;
    return true;
}

// Release a pointer from balloc; a caller's allocator may hand the memory out again at once, so
// the batch stream's queued work is waited for first (cudaFree waits by itself).
void bfree(sgcp_batch* b, void* p) {
    if (!p) return;
    if (b->custom_alloc) {
        if (b->stream) cudaStreamSynchronize(b->stream);
        b->ualloc.free(p, b->ualloc.user);
    } else {
        cudaFree(p);
    }
}

#define BCK(call, what)                                      \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return bcuda(b, e_, what);    \
    } while (0)

int ceil_div(int a, int b) { return (a + b - 1) / b; }

// Unit geometry of a stream for tile shape (b1log, n1, n2).
void set_geometry(BatchStream& S, int b1log, int n1, int n2) {
    S.b1log = b1log;
    S.n1 = n1;
    S.n2 = n2;
    const int S1 = (1 << b1log) * n1, S2 = (64 >> b1log) * n2;
    S.nb1 = ceil_div(S.dims[0], S1);
    S.nb2 = ceil_div(S.dims[1], S2);
    S.nb3 = ceil_div(S.dims[2], 32);
    S.n_box = S.nb1 * S.nb2 * S.nb3;
}

bool same_key(const sgcp_tune_entry& e, const BatchStream& S) {
    for (int k = 0; k < 3; ++k)
        if (e.bucket[k] != ceil_div(S.dims[k], 32)) return false;
    return e.rank == S.R && e.loss == S.loss;
}

bool valid_shape(int b1log, int n1, int n2) {
    return b1log >= 2 && b1log <= 4 && n1 >= 1 && n2 >= 1 && (1 << b1log) * n1 <= kBoxMaxS &&
           (64 >> b1log) * n2 <= kBoxMaxS;
}

// Default shape without timing: 8 x 8 tiles, boxes up to 32 x 32 rows.
sgcp_tune_entry default_entry(const BatchStream& S) {
    sgcp_tune_entry e{};
    for (int k = 0; k < 3; ++k) e.bucket[k] = ceil_div(S.dims[k], 32);
    e.rank = S.R;
    e.loss = S.loss;
    e.b1log = 3;
    e.n1 = std::min(4, ceil_div(S.dims[0], 8));
    e.n2 = std::min(4, ceil_div(S.dims[1], 8));
    e.us = 0.f;
    return e;
}

// Carve aligned pieces out of one allocation.
struct Carver {
    char* base;
    size_t off = 0;
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

// Lay out (or size, when base == nullptr) one stream's device state.
void carve_stream(Carver& cv, BatchStream& S, int H, int R) {
    const size_t N = (size_t)S.N, RR = (size_t)R * R;
    const int Hs = H > 0 ? H : 1;
    float** vecN[] = {&S.A, &S.Abar, &S.G, &S.u, &S.v, &S.u_o, &S.v_o, &S.a_o};
    for (float** p : vecN) *p = cv.take<float>(N);
    float** vecR[] = {&S.s, &S.s_u, &S.s_v, &S.s_uo, &S.s_vo, &S.s_ao, &S.gs};
    for (float** p : vecR) *p = cv.take<float>(R);
    S.s_hist = cv.take<float>((size_t)Hs * R);
    S.h_dev = cv.take<int64_t>(Hs);
    S.hist_len = cv.take<int32_t>(1);
    S.SH = cv.take<double>(RR);
    S.grams = cv.take<double>(18 * RR);
    S.gpart = cv.take<float>((size_t)S.n_gram * 6 * RR);
    S.Bc = cv.take<float>(3 * RR);
    S.Cc = cv.take<float>(3 * RR);
    S.st_w = cv.take<SolverState>(1);
    S.st_f = cv.take<SolverState>(1);
    S.rates_w = cv.take<double>(S.tau_w > 0 ? S.tau_w : 1);
    S.rates_f = cv.take<double>(S.tau_f > 0 ? S.tau_f : 1);
}

sgcp_status check_params(const sgcp_params& p, int s, std::string& why) {
    char buf[160];
    auto bad = [&](const char* m) {
        snprintf(buf, sizeof(buf), "stream %d: %s", s, m);
        why = buf;
    };
    if (p.ndim != 3) return bad("batched streams take 3-way slices"), SGCP_ERR_UNSUPPORTED;
    if (p.reserved != 0) return bad("reserved field not 0"), SGCP_ERR_ARG;
    if (p.history_kind != SGCP_HISTORY_MODEL)
        return bad("batched streams use the model-based history penalty"), SGCP_ERR_UNSUPPORTED;
    if (p.precision != SGCP_PREC_F32) return bad("batched streams run in FP32"), SGCP_ERR_UNSUPPORTED;
    if (p.temporal != SGCP_TEMPORAL_ADAM || p.optimizer != SGCP_OPT_ADAM)
        return bad("batched streams use the ADAM temporal and factor solvers"), SGCP_ERR_UNSUPPORTED;
    if (p.rank < 4 || p.rank > kBatchMaxR || p.rank % 4 != 0) return bad("rank must be 4..64, a multiple of 4"),
                                                                      SGCP_ERR_UNSUPPORTED;
    if (p.loss < 0 || p.loss > 3) return bad("bad loss"), SGCP_ERR_ARG;
    for (int k = 0; k < 3; ++k) {
        if (p.dims[k] < 1 || p.dims[k] > 0x7fffffff) return bad("bad dimension"), SGCP_ERR_ARG;
        if ((double)p.dims[k] * p.rank >= 2147483648.0) return bad("I_k * R too large"), SGCP_ERR_UNSUPPORTED;
    }
    if ((double)p.dims[0] * p.dims[1] * p.dims[2] > 9.0e18) return bad("slice too large"), SGCP_ERR_UNSUPPORTED;
    if (p.H < 0 || p.kappa_w < 0 || p.kappa_f < 0 || p.tau_w < 0 || p.tau_f < 0 || p.kappa_w > 32 ||
        p.kappa_f > 32)
        return bad("bad solver schedule"), SGCP_ERR_ARG;
    const double phases = 3.0 + p.kappa_w * (p.tau_w + 1.0) + p.kappa_f * (2.0 * p.tau_f + 1.0);
    if (phases > 1.0e9) return bad("too many solver iterations per step"), SGCP_ERR_UNSUPPORTED;
    return SGCP_OK;
}

sgcp_status batch_ready(sgcp_batch* b) {
    if (!b) return SGCP_ERR_ARG;
    if (b->sticky != SGCP_OK) return SGCP_ERR_STATE;
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return bcuda(b, e, "cudaSetDevice");
    return SGCP_OK;
}

sgcp_status bstatus_from_err(int bits) {
    if (bits & ERRB_TIMEOUT) return SGCP_ERR_TIMEOUT;
    if (bits & (ERRB_NUMERIC | ERRB_SOLVE)) return SGCP_ERR_NUMERIC;
    if (bits) return SGCP_ERR_STATE;
    return SGCP_OK;
}

// Time one candidate shape for stream s: a launch of the factor-gradient
// units, repeated so that the launch fills the device several times over;
// returns microseconds per slice-gradient pass (or a negative value on error).
float time_candidate(sgcp_batch* b, int s, const sgcp_tune_entry& c, int reps, BatchStream* dtune,
                     BatchStepEntry* dEt, float* gscratch, float* xones, cudaEvent_t e0, cudaEvent_t e1) {
    BatchStream S = b->hS[s];
    set_geometry(S, c.b1log, c.n1, c.n2);
    S.G = gscratch;
    S.s = xones;   // s = 1 and X = 1 keep every gradient value, and so every atomic, in the timing
    BatchStepEntry E{};
    E.X = xones;
    if (cudaMemcpyAsync(dtune, &S, sizeof(S), cudaMemcpyHostToDevice, b->stream) != cudaSuccess) return -1.f;
    if (cudaMemcpyAsync(dEt, &E, sizeof(E), cudaMemcpyHostToDevice, b->stream) != cudaSuccess) return -1.f;
    const int target = 4 * b->grid;
    const int passes = std::max(1, ceil_div(target, S.n_box));
    const int blocks = passes * S.n_box;
    if (launch_batch_units(dtune, dEt, S.n_box, blocks, b->stream) != cudaSuccess) return -1.f;   // warm-up
    float best = -1.f;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0, b->stream);
        if (launch_batch_units(dtune, dEt, S.n_box, blocks, b->stream) != cudaSuccess) return -1.f;
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const float us = 1000.f * ms / passes;
        if (best < 0.f || us < best) best = us;
    }
    return best;
}

sgcp_status autotune(sgcp_batch* b, int reps) {
    // scratch: a slice of ones as large as the largest stream's, a gradient buffer, descriptors
    int64_t maxX = 0, maxN = 0;
    for (const BatchStream& S : b->hS) {
        maxX = std::max(maxX, (int64_t)S.dims[0] * S.dims[1] * S.dims[2]);
        maxN = std::max(maxN, (int64_t)S.N);
    }
    float *xones = nullptr, *gscratch = nullptr;
    BatchStream* dtune = nullptr;
    BatchStepEntry* dEt = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    sgcp_status st = SGCP_OK;
    auto cleanup = [&]() {
        bfree(b, xones);
        bfree(b, gscratch);
        bfree(b, dtune);
        bfree(b, dEt);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if (!balloc(b, &xones, std::max<int64_t>(maxX, kBatchMaxR) * sizeof(float)) ||
        !balloc(b, &gscratch, maxN * sizeof(float)) || !balloc(b, &dtune, sizeof(BatchStream)) ||
        !balloc(b, &dEt, sizeof(BatchStepEntry)) || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return bfail(b, SGCP_ERR_OOM, "autotune: scratch allocation failed");
    }
    {
        const std::vector<float> ones((size_t)std::max<int64_t>(maxX, kBatchMaxR), 1.0f);
        if (cudaMemcpy(xones, ones.data(), ones.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
            cleanup();
            return bfail(b, SGCP_ERR_CUDA, "autotune: scratch fill failed");
        }
    }
    for (int s = 0; s < b->nS && st == SGCP_OK; ++s) {
        const BatchStream& S = b->hS[s];
        bool known = false;
        for (const sgcp_tune_entry& e : b->table)
            if (same_key(e, S)) known = true;
        if (known) continue;
        sgcp_tune_entry best = default_entry(S);
        best.us = -1.f;
        for (int b1log = 2; b1log <= 4; ++b1log)
            for (int S1 : {8, 16, 32})
                for (int S2 : {8, 16, 32}) {
                    const int n1 = S1 >> b1log, n2 = (S2 << b1log) >> 6;
                    if (n1 < 1 || n2 < 1 || !valid_shape(b1log, n1, n2)) continue;
                    if (S1 > 2 * ((S.dims[0] + 7) / 8 * 8) || S2 > 2 * ((S.dims[1] + 7) / 8 * 8)) continue;
                    sgcp_tune_entry c = best;
                    c.b1log = b1log;
                    c.n1 = n1;
                    c.n2 = n2;
                    const float us = time_candidate(b, s, c, reps, dtune, dEt, gscratch, xones, e0, e1);
                    if (us < 0.f) {
                        st = bfail(b, SGCP_ERR_CUDA, "autotune: timing launch failed");
                        break;
                    }
                    if (best.us < 0.f || us < best.us) {
                        best = c;
                        best.us = us;
                    }
                }
        if (st == SGCP_OK) b->table.push_back(best);
    }
    cudaError_t e = cudaStreamSynchronize(b->stream);
    cleanup();
    if (st != SGCP_OK) return st;
    if (e != cudaSuccess) return bcuda(b, e, "autotune");
    return SGCP_OK;
}

sgcp_status build_graph(sgcp_batch* b) {
    BatchArgs a{};
    a.S = b->dS;
    a.E = b->dE;
    a.ctl = b->ctl;
    a.order = b->dorder;
    a.nS = b->nS;
    a.finished = b->finished;
    a.err = b->err;
    a.spin_limit = b->spin_limit;
    cudaGraph_t g = nullptr;
    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed), "begin capture");
    cudaError_t e1 = launch_batch_step(a, b->grid, b->stream, nullptr);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e1 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bcuda(b, e1, "capture batch step");
    }
    if (e2 != cudaSuccess) return bcuda(b, e2, "end capture");
    cudaError_t e3 = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) return bcuda(b, e3, "instantiate graph");
    return SGCP_OK;
}

}  // namespace

extern "C" {

sgcp_status sgcp_batch_opts_default(sgcp_batch_opts* o) {
    if (!o) return SGCP_ERR_ARG;
    std::memset(o, 0, sizeof(*o));
    o->autotune = 0;
    o->tune_reps = 3;
    o->table = nullptr;
    o->n_table = 0;
    o->grid_blocks = 0;
    o->spin_limit = 0;
    return SGCP_OK;
}

sgcp_status sgcp_batch_create(int32_t n_streams, const sgcp_params* params, const void* const* init_factors,
                              const sgcp_batch_opts* opts, const sgcp_allocator* allocator, void* cuda_stream,
                              sgcp_batch** out) {
    if (!out) return SGCP_ERR_ARG;
    *out = nullptr;
    if (allocator && (!allocator->alloc || !allocator->free)) return SGCP_ERR_ARG;
    if (n_streams < 1 || n_streams > 65536 || !params || !init_factors) return SGCP_ERR_ARG;
    sgcp_batch_opts o;
    sgcp_batch_opts_default(&o);
    if (opts) o = *opts;
    if (o.tune_reps < 1 || o.grid_blocks < 0 || o.spin_limit < 0 || o.n_table < 0 || (o.n_table > 0 && !o.table))
        return SGCP_ERR_ARG;
    for (int i = 0; i < o.n_table; ++i)
        if (!valid_shape(o.table[i].b1log, o.table[i].n1, o.table[i].n2)) return SGCP_ERR_ARG;
    std::string why;
    for (int s = 0; s < n_streams; ++s) {
        if (sgcp_status st = check_params(params[s], s, why)) return st;
        for (int k = 0; k < 3; ++k)
            if (!init_factors[3 * s + k]) return SGCP_ERR_ARG;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return SGCP_ERR_CUDA;
    }
    sgcp_batch* b = new (std::nothrow) sgcp_batch();
    if (!b) return SGCP_ERR_OOM;
    b->nS = n_streams;
    b->device = dev;
    if (allocator) {
        b->ualloc = *allocator;
        b->custom_alloc = true;
    }
    b->P.assign(params, params + n_streams);
    if (o.spin_limit > 0) b->spin_limit = o.spin_limit;
    for (int i = 0; i < o.n_table; ++i) b->table.push_back(o.table[i]);
    auto bail = [&](sgcp_status st) {
        sgcp_batch_destroy(b);
        return st;
    };
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return SGCP_ERR_CUDA;
        }
        b->own_stream = true;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    b->grid = o.grid_blocks > 0 ? o.grid_blocks : std::max(1, sms) * batch_blocks_per_sm();

    // per-stream descriptions
    b->hS.resize(n_streams);
    b->hist_t.resize(n_streams);
    b->t.assign(n_streams, 0);
    b->hE.resize(n_streams);
    for (int s = 0; s < n_streams; ++s) {
        const sgcp_params& p = params[s];
        BatchStream& S = b->hS[s];
        std::memset(&S, 0, sizeof(S));
        S.R = p.rank;
        S.loss = p.loss;
        S.nrows = 0;
        for (int k = 0; k < 3; ++k) {
            S.dims[k] = (int)p.dims[k];
            S.row_off[k] = S.nrows;
            S.nrows += S.dims[k];
            S.gch[k] = ceil_div(S.dims[k], kBatchGramRows);
            S.uch[k] = ceil_div(S.dims[k], kBatchUpdRows);
        }
        S.N = S.nrows * S.R;
        S.n_gram = S.gch[0] + S.gch[1] + S.gch[2];
        S.n_upd = S.uch[0] + S.uch[1] + S.uch[2];
        S.kappa_w = p.kappa_w;
        S.tau_w = p.tau_w;
        S.kappa_f = p.kappa_f;
        S.tau_f = p.tau_f;
        S.PF0 = 2 + p.kappa_w * (p.tau_w + 1);
        S.P = S.PF0 + 1 + p.kappa_f * (2 * p.tau_f + 1);
        S.eps = (float)p.log_eps;
        double lower = p.lower_bound;
        if (std::isnan(lower))
            lower = (p.loss == SGCP_LOSS_POISSON || p.loss == SGCP_LOSS_BERNOULLI_ODDS) ? 0.0 : -INFINITY;
        S.lower = (float)lower;
        S.tol_w = p.tol_w;
        S.tol_f = p.tol_f;
        S.alpha_w = p.alpha_w;
        S.alpha_f = p.alpha_f;
        S.beta1 = p.beta1;
        S.beta2 = p.beta2;
        S.adam_eps = p.adam_eps;
        S.decay = p.alpha_decay;
        S.w = p.w;
        S.theta = p.theta;
        S.lam = p.lambda;
        S.mu = p.mu;
        const sgcp_tune_entry d = default_entry(S);
        set_geometry(S, d.b1log, d.n1, d.n2);
    }
    // one allocation for all streams' state
    Carver sizer{nullptr};
    for (int s = 0; s < n_streams; ++s) carve_stream(sizer, b->hS[s], params[s].H, b->hS[s].R);
    const size_t arena_bytes = sizer.off + 256;
    if (!balloc(b, &b->arena, arena_bytes)) return bail(bfail(b, SGCP_ERR_OOM, "batch state allocation failed"));
    Carver cv{(char*)b->arena};
    for (int s = 0; s < n_streams; ++s) carve_stream(cv, b->hS[s], params[s].H, b->hS[s].R);
    if (!balloc(b, &b->dS, n_streams * sizeof(BatchStream)) || !balloc(b, &b->dE, n_streams * sizeof(BatchStepEntry)) ||
        !balloc(b, &b->ctl, n_streams * sizeof(BatchCtl)) || !balloc(b, &b->dorder, n_streams * sizeof(int32_t)) ||
        !balloc(b, &b->finished, sizeof(int)) || !balloc(b, &b->err, sizeof(int)))
        return bail(bfail(b, SGCP_ERR_OOM, "batch control allocation failed"));
    cudaStream_t st = b->stream;
    cudaError_t e = cudaMemsetAsync(b->arena, 0, arena_bytes, st);
    SolverState st0{};
    st0.b1pow = 1.0;
    st0.b2pow = 1.0;
    for (int s = 0; s < n_streams && e == cudaSuccess; ++s) {
        BatchStream& S = b->hS[s];
        for (int k = 0; k < 3 && e == cudaSuccess; ++k)
            e = cudaMemcpyAsync(S.A + (size_t)S.row_off[k] * S.R, init_factors[3 * s + k],
                                (size_t)S.dims[k] * S.R * sizeof(float), cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(S.Abar, S.A, (size_t)S.N * sizeof(float), cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(S.a_o, S.A, (size_t)S.N * sizeof(float), cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(S.st_w, &st0, sizeof(st0), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(S.st_f, &st0, sizeof(st0), cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(b->err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // host-side st0 dies here
    if (e != cudaSuccess) return bail(bcuda(b, e, "batch init"));

    // unit shapes: table entries, then autotuning (needs the factors in place), else defaults
    if (o.autotune)
        if (sgcp_status ts = autotune(b, o.tune_reps)) return bail(ts);
    b->cfg.assign(n_streams, -1);
    for (int s = 0; s < n_streams; ++s) {
        BatchStream& S = b->hS[s];
        int idx = -1;
        for (size_t i = 0; i < b->table.size(); ++i)
            if (same_key(b->table[i], S)) idx = (int)i;
        if (idx < 0) {
            b->table.push_back(default_entry(S));
            idx = (int)b->table.size() - 1;
        }
        b->cfg[s] = idx;
        set_geometry(S, b->table[idx].b1log, b->table[idx].n1, b->table[idx].n2);
    }
    // scheduling priority: streams with the most work per phase first
    std::vector<int32_t> order(n_streams);
    for (int s = 0; s < n_streams; ++s) order[s] = s;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        const BatchStream &Sa = b->hS[a], &Sc = b->hS[c];
        const double wa = (double)Sa.dims[0] * Sa.dims[1] * Sa.dims[2] * Sa.R;
        const double wc = (double)Sc.dims[0] * Sc.dims[1] * Sc.dims[2] * Sc.R;
        return wa > wc;
    });
    e = cudaMemcpy(b->dS, b->hS.data(), n_streams * sizeof(BatchStream), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->dorder, order.data(), n_streams * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bail(bcuda(b, e, "batch descriptors"));
    *out = b;
    return SGCP_OK;
}

void sgcp_batch_destroy(sgcp_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->copy_stream) cudaStreamSynchronize(b->copy_stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    void* ptrs[] = {b->arena, b->dS, b->dE, b->ctl, b->dorder, b->finished, b->err, b->xstage[0], b->xstage[1],
                    b->fout};
    for (void* p : ptrs) bfree(b, p);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    if (b->copy_stream) cudaStreamDestroy(b->copy_stream);
    if (b->ev_xstaged) cudaEventDestroy(b->ev_xstaged);
    for (int i = 0; i < 2; ++i)
        if (b->ev_xused[i]) cudaEventDestroy(b->ev_xused[i]);
    delete b;
}

const char* sgcp_batch_last_error(const sgcp_batch* b) { return b ? b->last_error.c_str() : "null batch"; }

sgcp_status sgcp_batch_step(sgcp_batch* b, const void* const* X, int32_t x_on_host) {
    if (sgcp_status st = batch_ready(b)) return st;
    if (!X) return bfail(b, SGCP_ERR_ARG, "batch step: X is NULL");
    for (int s = 0; s < b->nS; ++s)
        if (!X[s]) return bfail(b, SGCP_ERR_ARG, "batch step: a slice pointer is NULL");
    int xb = -1;   // staging buffer of this step (host slices)
    if (x_on_host) {
        if (b->xoff.empty()) {
            int64_t tot = 0;
            b->xoff.resize(b->nS);
            for (int s = 0; s < b->nS; ++s) {
                b->xoff[s] = tot;
                const BatchStream& S = b->hS[s];
                tot += ((int64_t)S.dims[0] * S.dims[1] * S.dims[2] + 63) / 64 * 64;
            }
            b->xstage_floats = tot;
        }
        if (!b->copy_stream) {
            BCK(cudaStreamCreateWithFlags(&b->copy_stream, cudaStreamNonBlocking), "copy stream");
            BCK(cudaEventCreateWithFlags(&b->ev_xstaged, cudaEventDisableTiming), "staging event");
            BCK(cudaEventCreateWithFlags(&b->ev_xused[0], cudaEventDisableTiming), "staging event");
            BCK(cudaEventCreateWithFlags(&b->ev_xused[1], cudaEventDisableTiming), "staging event");
        }
        // Buffer xb is refilled; the other buffer was current for all the work queued since the
        // last staged step, whose end is marked here.  xb was last read by the work before that
        // mark two staged steps ago: the copy stream waits for it, the batch stream for the copies.
        xb = b->xnext;
        if (!b->xstage[xb] && !balloc(b, &b->xstage[xb], b->xstage_floats * sizeof(float)))
            return bfail(b, SGCP_ERR_OOM, "slice staging allocation failed");
        if (b->xused[xb ^ 1]) BCK(cudaEventRecord(b->ev_xused[xb ^ 1], b->stream), "staging event");
        if (b->xused[xb]) BCK(cudaStreamWaitEvent(b->copy_stream, b->ev_xused[xb], 0), "staging wait");
    }
    for (int s = 0; s < b->nS; ++s) {
        const BatchStream& S = b->hS[s];
        BatchStepEntry& E = b->hE[s];
        const float* x = (const float*)X[s];
        if (x_on_host) {
            float* dst = b->xstage[xb] + b->xoff[s];
            BCK(cudaMemcpyAsync(dst, X[s], (size_t)S.dims[0] * S.dims[1] * S.dims[2] * sizeof(float),
                                cudaMemcpyHostToDevice, b->copy_stream),
                "copy slice");
            x = dst;
        }
        const int64_t t = b->t[s] + 1;
        const int H = b->P[s].H;
        std::vector<int64_t>& ht = b->hist_t[s];
        E.X = x;
        E.t = t;
        E.hist_on = ht.empty() ? 0 : 1;
        E.slot = -1;
        E.len = (int32_t)ht.size();
        if (H > 0) {
            if ((int)ht.size() < H) {
                E.slot = (int32_t)ht.size();
                E.len = E.slot + 1;
            } else {
                const uint32_t j = reservoir_index(b->P[s].seed, t);
                if ((int64_t)j <= H) E.slot = (int32_t)j - 1;
            }
        }
    }
    if (x_on_host) {
        BCK(cudaEventRecord(b->ev_xstaged, b->copy_stream), "staging event");
        BCK(cudaStreamWaitEvent(b->stream, b->ev_xstaged, 0), "staging wait");
        b->xused[xb] = true;
        b->xnext = xb ^ 1;
    }
    BCK(launch_batch_begin(b->dE, b->hE.data(), b->nS, b->ctl, b->nS, b->finished, b->stream, &b->launches),
        "batch begin");
    if (!b->graph)
        if (sgcp_status st = build_graph(b)) return st;
    BCK(cudaGraphLaunch(b->graph, b->stream), "graph launch");
    b->launches += 1;
    for (int s = 0; s < b->nS; ++s) {   // host copy of the window, as the tails will leave it
        const BatchStepEntry& E = b->hE[s];
        std::vector<int64_t>& ht = b->hist_t[s];
        if (E.slot >= 0) {
            if (E.slot == (int)ht.size()) ht.push_back(E.t);
            else ht[E.slot] = E.t;
        }
        b->t[s] = E.t;
    }
    return SGCP_OK;
}

sgcp_status sgcp_batch_factors(sgcp_batch* b, int32_t s, void* const* A_out, void* s_out, int64_t* t_out) {
    if (!b || s < 0 || s >= b->nS) return SGCP_ERR_ARG;
    cudaSetDevice(b->device);
    const BatchStream& S = b->hS[s];
    if (A_out)
        for (int k = 0; k < 3; ++k) {
            if (!A_out[k]) continue;
            BCK(cudaMemcpyAsync(A_out[k], S.A + (size_t)S.row_off[k] * S.R, (size_t)S.dims[k] * S.R * sizeof(float),
                                cudaMemcpyDeviceToDevice, b->stream),
                "copy factors");
        }
    if (s_out) BCK(cudaMemcpyAsync(s_out, S.s, S.R * sizeof(float), cudaMemcpyDeviceToDevice, b->stream), "copy s");
    if (t_out) *t_out = b->t[s];
    return SGCP_OK;
}

sgcp_status sgcp_batch_check(sgcp_batch* b) {
    if (!b) return SGCP_ERR_ARG;
    if (b->sticky != SGCP_OK) return SGCP_ERR_STATE;
    cudaSetDevice(b->device);
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "synchronize");
    int bits = 0;
    e = cudaMemcpy(&bits, b->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bcuda(b, e, "read error word");
    if (bits) {
        b->sticky = bstatus_from_err(bits);
        char buf[96];
        snprintf(buf, sizeof(buf), "device error bits 0x%x", bits);
        b->last_error = buf;
        return b->sticky;
    }
    return SGCP_OK;
}

namespace {
// F_w, F_f of every stream (the accepted objective estimates of its temporal and factor solvers)
// into out[2 s], out[2 s + 1]: one thread per stream reads the stream's two solver states.
__global__ void k_batch_objectives(const BatchStream* __restrict__ dS, int nS, double* out) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nS; s += gridDim.x * blockDim.x) {
        out[2 * s] = dS[s].st_w->F_cur;
        out[2 * s + 1] = dS[s].st_f->F_cur;
    }
}
}  // namespace

sgcp_status sgcp_batch_objectives_async(sgcp_batch* b, double* out) {
    if (!out) return SGCP_ERR_ARG;
    if (sgcp_status st = batch_ready(b)) return st;
    const size_t bytes = (size_t)b->nS * 2 * sizeof(double);
    if (!b->fout && !balloc(b, &b->fout, bytes)) return bfail(b, SGCP_ERR_OOM, "objective buffer allocation failed");
    k_batch_objectives<<<(b->nS + 127) / 128, 128, 0, b->stream>>>(b->dS, b->nS, b->fout);
    BCK(cudaGetLastError(), "objective gather");
    BCK(cudaMemcpyAsync(out, b->fout, bytes, cudaMemcpyDeviceToHost, b->stream), "objective read-back");
    b->launches += 1;
    return SGCP_OK;
}

sgcp_status sgcp_batch_stats(sgcp_batch* b, int32_t s, sgcp_stats_t* out) {
    if (!b || !out || s < 0 || s >= b->nS) return SGCP_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
    sgcp_status st = sgcp_batch_check(b);
    const BatchStream& S = b->hS[s];
    SolverState w{}, f{};
    int bits = 0;
    cudaMemcpy(&w, S.st_w, sizeof(w), cudaMemcpyDeviceToHost);
    cudaMemcpy(&f, S.st_f, sizeof(f), cudaMemcpyDeviceToHost);
    cudaMemcpy(&bits, b->err, sizeof(int), cudaMemcpyDeviceToHost);
    out->t = b->t[s];
    out->iter = f.i;
    out->F_w = w.F_cur;
    out->F_f = f.F_cur;
    out->epochs_w = w.epoch;
    out->epochs_f = f.epoch;
    out->accept_w = w.accept;
    out->accept_f = f.accept;
    out->alpha_w = w.alpha;
    out->alpha_f = f.alpha;
    out->hist_len = (int32_t)b->hist_t[s].size();
    out->error_bits = bits;
    out->kernels_launched = b->launches;
    return st;
}

sgcp_status sgcp_batch_tune_table(const sgcp_batch* b, sgcp_tune_entry* out, int32_t cap, int32_t* n_out) {
    if (!b || cap < 0 || (cap > 0 && !out)) return SGCP_ERR_ARG;
    const int n = (int)b->table.size();
    if (n_out) *n_out = n;
    for (int i = 0; i < n && i < cap; ++i) out[i] = b->table[i];
    return SGCP_OK;
}

sgcp_status sgcp_batch_unit_config(const sgcp_batch* b, int32_t s, sgcp_tune_entry* out) {
    if (!b || !out || s < 0 || s >= b->nS) return SGCP_ERR_ARG;
    *out = b->table[b->cfg[s]];
    return SGCP_OK;
}

}  // extern "C"
