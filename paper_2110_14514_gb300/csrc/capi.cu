// C ABI of the streaming-GCP library: context state, slice loading, the
// direct gradient entry point, and the OnlineGCP step (Alg. 1 loop body of
// arXiv 2110.14514) enqueued as one captured CUDA graph per slice kind.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <initializer_list>
#include <new>
#include <string>
#include <vector>

#include "internal.h"
#include "sgcp.h"

using namespace sgcp;

struct sgcp_ctx {
    sgcp_params P;
    int ndim = 0, R = 0;
    int64_t dims[4] = {0, 0, 0, 0};
    int64_t row_off[4] = {0, 0, 0, 0};
    int64_t nrows = 0, N = 0;
    bool f64 = false;
    size_t esz = 4;
    double lower = 0.0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    std::string last_error;
    sgcp_status sticky = SGCP_OK;
    int64_t launches = 0;
    std::vector<void*> allocs;
    sgcp_allocator ualloc{};     // caller's device-memory provider (used when custom_alloc)
    bool custom_alloc = false;

    // factor-solver state (N elements each, element type T)
    void *A = nullptr, *Abar = nullptr, *G = nullptr, *u = nullptr, *v = nullptr, *u_o = nullptr, *v_o = nullptr,
         *a_o = nullptr;
    // temporal-solver state (R each)
    void *s = nullptr, *s_u = nullptr, *s_v = nullptr, *s_uo = nullptr, *s_vo = nullptr, *s_ao = nullptr,
         *gs = nullptr;
    // sparse temporal solve with the step deferred to the next kernel: a second (s, u, v) and
    // three gradient sums in rotation
    void *s2 = nullptr, *gs3 = nullptr;
    // history window
    void* s_hist = nullptr;
    int64_t* h_dev = nullptr;
    int32_t* hist_len_dev = nullptr;
    std::vector<int64_t> hist_t;
    double* SH = nullptr;
    double* grams = nullptr;     // [6][ndim][R][R]
    void* gpart = nullptr;       // Gram partial sums [6][ndim][gram_nblk][R][R], element type T
    int gram_nblk = 1;
    int64_t gram_rpb = 256;
    cudaStream_t side = nullptr; // second capture stream: Gram work runs beside the gradient kernel
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    float* gacc = nullptr;       // 2 x [2][ndim][R][R] Gram sums of the factor updates (FP32, R <= 32, H > 0)
    void* Bc = nullptr;          // [ndim][R][R], element type T
    void* Cc = nullptr;
    double* lsq_work = nullptr;  // R*R + R
    SolverState* st_w = nullptr;
    SolverState* st_f = nullptr;
    double* rates_w = nullptr;   // per-epoch learning rates of the temporal / factor ADAM iterations
    double* rates_f = nullptr;
    int* err = nullptr;
    SliceDesc* slice_dev = nullptr;
    double* metric = nullptr;    // [2]: loss sum and ||X||^2 of sgcp_slice_loss
    // stored-slice history (SGCP_HISTORY_SLICES): the window's slices themselves, one slot each
    bool stored_hist = false;
    int hist_sparse = -1;                  // kind of the stored slices (-1 while none is stored)
    std::vector<void*> hs_idx, hs_vals;
    std::vector<size_t> hs_idx_cap, hs_vals_cap, hs_keys_cap;
    std::vector<void*> hs_keys;
    SliceDesc* hist_desc = nullptr;        // [H] device descriptors of the slots
    void* hist_w = nullptr;                // [H] slot weights w theta^(t - h), element type
    int32_t* hist_skip = nullptr;          // [H] 1: slot inactive or solver finished
    int32_t* zero_i = nullptr;             // a device 0: the model-based terms see an empty window

    // sparse-slice structures
    unsigned long long* hkeys = nullptr;
    int hlog2 = 0;
    int32_t *counts = nullptr, *hot = nullptr, *hot_rows = nullptr;
    int nhot = kMaxHot;

    // staging of host slices
    // staging of host (and realigned) slices: two buffer pairs used in turn, filled on copy_stream
    // so that the copy of one step's slice overlaps the work of the step before it
    void* stage_idx[2] = {nullptr, nullptr};
    size_t stage_idx_bytes[2] = {0, 0};
    void* stage_vals[2] = {nullptr, nullptr};
    size_t stage_vals_bytes[2] = {0, 0};
    int stage_next = 0;                       // buffer pair of the next staged slice
    bool stage_used[2] = {false, false};      // pair holds a slice that queued work may read
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_stage_used[2] = {nullptr, nullptr};   // end of the work queued while a pair was current
    cudaEvent_t ev_staged = nullptr;          // the latest staging copies are complete

    // slice currently loaded
    bool loaded = false;
    int loaded_sparse = 0;
    const void* loaded_user_idx = nullptr;
    const void* loaded_user_vals = nullptr;
    int64_t loaded_nnz = -1;
    SliceDesc cur{};

    int64_t t = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};   // [dense, sparse]
    // L-BFGS solver (optimizer SGCP_OPT_LBFGS): iterate, gradient, direction, m + 1 pair slots,
    // their device pointer tables and the device-resident iteration state
    void *lb_x = nullptr, *lb_g = nullptr, *lb_p = nullptr;
    void** lb_tab = nullptr;       // [2][kLbfgsSlots]: S slots, then Y slots
    LbfgsState* lb_state = nullptr;
    cudaStream_t lb_stream = nullptr;   // captures the bodies of the line-search WHILE nodes
    int64_t graph_kernels[2] = {0, 0};
    // tensor-core contexts: TMA tensor map of the current dense slice (device, 128 bytes)
    bool tc = false;
    void* xmap = nullptr;
    bool xmap_ok = false;
    bool xmap_written = false;           // xmap holds xmap_last
    unsigned char xmap_last[128] = {};
};

namespace {

sgcp_status fail(sgcp_ctx* c, sgcp_status st, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        c->last_error = buf;
    }
    return st;
}

sgcp_status cuda_fail(sgcp_ctx* c, cudaError_t e, const char* what) {
    if (c) {
        c->last_error = std::string(what) + ": " + cudaGetErrorString(e);
        c->sticky = SGCP_ERR_CUDA;
    }
    return e == cudaErrorMemoryAllocation ? SGCP_ERR_OOM : SGCP_ERR_CUDA;
}

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

// Device allocation of context state: through the caller's allocator when one was given at
// sgcp_create, else cudaMalloc.  Every pointer is recorded so that sgcp_destroy releases it.
sgcp_status dalloc(sgcp_ctx* c, void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (c->custom_alloc) {
        *p = c->ualloc.alloc(bytes, c->ualloc.user);
        if (!*p) {
            c->last_error = "allocator returned NULL";
            return SGCP_ERR_OOM;
        }
        if ((reinterpret_cast<uintptr_t>(*p) & 255) != 0) {
            c->ualloc.free(*p, c->ualloc.user);
            *p = nullptr;
            c->last_error = "allocator returned memory that is not 256-byte aligned";
            return SGCP_ERR_ARG;
        }
        c->allocs.push_back(*p);
        return SGCP_OK;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        c->last_error = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? SGCP_ERR_OOM : SGCP_ERR_CUDA;
    }
    c->allocs.push_back(*p);
    return SGCP_OK;
}

// Release one pointer obtained from dalloc.  cudaFree waits for the device; a caller's allocator
// may hand the memory out again at once, so the context's queued work is waited for first.
void release(sgcp_ctx* c, void* p) {
    if (c->custom_alloc) {
        if (c->stream) cudaStreamSynchronize(c->stream);
        c->ualloc.free(p, c->ualloc.user);
    } else {
        cudaFree(p);
    }
}

template <typename P>
sgcp_status dalloc_t(sgcp_ctx* c, P** p, size_t bytes) {
    void* q = nullptr;
    sgcp_status st = dalloc(c, &q, bytes);
    *p = (P*)q;
    return st;
}

void dfree(sgcp_ctx* c, void* p) {
    if (!p) return;
    for (size_t i = 0; i < c->allocs.size(); ++i)
        if (c->allocs[i] == p) {
            c->allocs.erase(c->allocs.begin() + (long)i);
            break;
        }
    release(c, p);
}

int64_t omega_of(const sgcp_ctx* c) {
    int64_t w = 1;
    for (int k = 0; k < c->ndim; ++k) w *= c->dims[k];
    return w;
}

void* offs(void* base, int64_t elems, size_t esz) { return (char*)base + (size_t)elems * esz; }

uint32_t purpose_nz(int set) {
    switch (set) {
        case SGCP_SAMPLES_FACTOR_GRAD: return PUR_GRAD_NZ;
        case SGCP_SAMPLES_FACTOR_OBJ: return PUR_OBJ_NZ;
        case SGCP_SAMPLES_TEMPORAL_GRAD: return PUR_TGRAD_NZ;
        default: return PUR_TOBJ_NZ;
    }
}

uint32_t purpose_z(int set) { return purpose_nz(set) + 1; }

// Load X: stage host data, ingest sparse slices when they changed, fill c->cur.
sgcp_status load_slice(sgcp_ctx* c, const sgcp_slice* X, int64_t t, bool force_ingest) {
    if (!X) return fail(c, SGCP_ERR_ARG, "slice is NULL");
    const bool sparse = X->is_sparse != 0;
    const int64_t omega = omega_of(c);
    const int64_t nnz = sparse ? X->nnz : omega;
    if (sparse) {
        if (c->f64) return fail(c, SGCP_ERR_UNSUPPORTED, "sparse slices need a float context");
        if (nnz < 0 || nnz > omega || nnz >= (int64_t)1 << 31)
            return fail(c, SGCP_ERR_ARG, "sparse slice nnz %lld out of range", (long long)nnz);
        if (nnz > 0 && (!X->idx || !X->vals)) return fail(c, SGCP_ERR_ARG, "sparse slice without idx/vals");
    } else {
        if (!X->vals) return fail(c, SGCP_ERR_ARG, "dense slice without vals");
        if (c->ndim > 3) return fail(c, SGCP_ERR_UNSUPPORTED, "dense slices support ndim <= 3");
    }
    const void* idx_d = X->idx;
    const void* vals_d = X->vals;
    // the tensor-core kernel loads dense tiles by TMA, which needs a 16-byte aligned slice
    const bool restage = !X->on_host && !sparse && c->tc && (reinterpret_cast<uintptr_t>(X->vals) & 15) != 0;
    if (X->on_host || restage) {
        const size_t ib = sparse ? (size_t)nnz * c->ndim * sizeof(int32_t) : 0;
        const size_t vb = (size_t)nnz * (sparse ? sizeof(float) : c->esz);
        // Pair b is refilled; the other pair was current for all the work queued since the last
        // staged slice, whose end is marked here.  Pair b was last read by the work before that
        // mark two staged slices ago: the copy stream waits for it, the context stream waits for
        // the copies.
        if (!c->copy_stream) {   // created with the first staged slice: contexts fed device slices never hold it
            CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking), "copy stream");
            CK(cudaEventCreateWithFlags(&c->ev_staged, cudaEventDisableTiming), "staging event");
            CK(cudaEventCreateWithFlags(&c->ev_stage_used[0], cudaEventDisableTiming), "staging event");
            CK(cudaEventCreateWithFlags(&c->ev_stage_used[1], cudaEventDisableTiming), "staging event");
        }
        const int b = c->stage_next;
        if (c->stage_used[b ^ 1]) CK(cudaEventRecord(c->ev_stage_used[b ^ 1], c->stream), "staging event");
        if (ib > c->stage_idx_bytes[b]) {
            dfree(c, c->stage_idx[b]);
            c->stage_idx[b] = nullptr;
            c->stage_idx_bytes[b] = 0;
            sgcp_status st = dalloc(c, &c->stage_idx[b], ib);
            if (st) return st;
            c->stage_idx_bytes[b] = ib;
        }
        if (vb > c->stage_vals_bytes[b]) {
            dfree(c, c->stage_vals[b]);
            c->stage_vals[b] = nullptr;
            c->stage_vals_bytes[b] = 0;
            sgcp_status st = dalloc(c, &c->stage_vals[b], vb);
            if (st) return st;
            c->stage_vals_bytes[b] = vb;
        }
        if (c->stage_used[b]) CK(cudaStreamWaitEvent(c->copy_stream, c->ev_stage_used[b], 0), "staging wait");
        const cudaMemcpyKind kind = X->on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
        if (!X->on_host) {   // a realigned device slice: work queued on the context stream may still write it
            CK(cudaEventRecord(c->ev_staged, c->stream), "staging order");
            CK(cudaStreamWaitEvent(c->copy_stream, c->ev_staged, 0), "staging order");
        }
        if (ib) CK(cudaMemcpyAsync(c->stage_idx[b], X->idx, ib, kind, c->copy_stream), "copy slice idx");
        if (vb) CK(cudaMemcpyAsync(c->stage_vals[b], X->vals, vb, kind, c->copy_stream), "copy slice vals");
        CK(cudaEventRecord(c->ev_staged, c->copy_stream), "staging event");
        CK(cudaStreamWaitEvent(c->stream, c->ev_staged, 0), "staging wait");
        c->stage_used[b] = true;
        c->stage_next = b ^ 1;
        idx_d = c->stage_idx[b];
        vals_d = c->stage_vals[b];
        force_ingest = true;
    }
    c->cur.idx = (const int32_t*)idx_d;
    c->cur.vals = vals_d;
    c->cur.nnz = nnz;
    c->cur.t = t;
    const bool same = c->loaded && c->loaded_sparse == (int)sparse && c->loaded_user_idx == X->idx &&
                      c->loaded_user_vals == X->vals && c->loaded_nnz == nnz;
    if (sparse && (force_ingest || !same)) {
        int hl = 10;
        while (((int64_t)1 << hl) < 2 * nnz) ++hl;
        if (hl > c->hlog2) {
            dfree(c, c->hkeys);
            c->hkeys = nullptr;
            sgcp_status st = dalloc_t(c, &c->hkeys, ((size_t)1 << hl) * sizeof(unsigned long long));
            if (st) return st;
            c->hlog2 = hl;
        }
        CK(cudaMemsetAsync(c->hkeys, 0xFF, ((size_t)1 << c->hlog2) * sizeof(unsigned long long), c->stream),
           "clear hash");
        CK(cudaMemsetAsync(c->counts, 0, (size_t)c->nrows * sizeof(int32_t), c->stream), "clear counts");
        CK(cudaMemsetAsync(c->hot, 0xFF, (size_t)c->nrows * sizeof(int32_t), c->stream), "clear hot");
        CK(cudaMemsetAsync(c->hot_rows, 0xFF, (size_t)c->ndim * kMaxHot * sizeof(int32_t), c->stream),
           "clear hot rows");
        IngestArgs ia{};
        ia.slice = c->cur;
        ia.ndim = c->ndim;
        for (int k = 0; k < 4; ++k) {
            ia.dims[k] = c->dims[k];
            ia.row_off[k] = c->row_off[k];
        }
        ia.hkeys = c->hkeys;
        ia.hlog2 = c->hlog2;
        ia.counts = c->counts;
        ia.hot = c->hot;
        ia.hot_rows = c->hot_rows;
        ia.sub_stride = nnz > 131072 ? nnz / 131072 : 1;
        ia.nhot = c->nhot;
        ia.err = c->err;
        if (nnz > 0) CK(launch_ingest(ia, nnz, c->stream, &c->launches), "ingest");
    }
    // The step graph reads the slice through its device descriptor, so the descriptor carries the
    // hash as well: a larger slice reallocates the table, and the graph (captured once) must not
    // keep the old table's address and size.
    c->cur.hkeys = sparse ? c->hkeys : nullptr;
    c->cur.hlog2 = sparse ? c->hlog2 : 0;
    c->cur.draw_base = 0;
    c->loaded = true;
    c->loaded_sparse = (int)sparse;
    c->loaded_user_idx = X->idx;
    c->loaded_user_vals = X->vals;
    c->loaded_nnz = nnz;
    return SGCP_OK;
}

// Tensor-core contexts: encode the TMA tensor map of the dense slice in c->cur and write it to
// c->xmap on the context stream (the step graph and direct launches read it from there).  With
// the slice staged to 16-byte alignment, whether it encodes depends only on I3 and the driver, so
// it is the same for every slice of a context.  The map encodes only the slice's address and
// shape, so a map equal to the one already written is not written again.
sgcp_status prepare_xmap(sgcp_ctx* c) {
    if (!c->tc) return SGCP_OK;
    unsigned char map[128] = {};
    c->xmap_ok = encode_x_map(map, (const float*)c->cur.vals, c->dims[0], c->dims[1], c->dims[2]);
    if (!c->xmap_ok || (c->xmap_written && std::memcmp(map, c->xmap_last, sizeof(map)) == 0)) return SGCP_OK;
    c->xmap_written = false;
    CK(launch_write_map(c->xmap, map, c->stream, &c->launches), "tensor map");
    std::memcpy(c->xmap_last, map, sizeof(map));
    c->xmap_written = true;
    return SGCP_OK;
}

SparseGradArgs sparse_args(sgcp_ctx* c, const SliceDesc* slice_dev, int set, uint32_t draw, int want,
                           const void* s, const void* const* A, void* const* G, void* gs, double* f, int loss,
                           const void* y_scale, const int32_t* skip) {
    SparseGradArgs a{};
    a.slice = slice_dev;
    a.inline_slice = c->cur;
    a.ndim = c->ndim;
    a.R = c->R;
    for (int k = 0; k < 4; ++k) a.dims[k] = c->dims[k];
    for (int k = 0; k < c->ndim; ++k) {
        a.A[k] = (const float*)A[k];
        a.G[k] = G ? (float*)G[k] : nullptr;
        a.hot[k] = c->hot + c->row_off[k];
    }
    a.s = (const float*)s;
    a.gs = (float*)gs;
    a.f = f;
    a.hkeys = c->hkeys;
    a.hlog2 = c->hlog2;
    a.hot_rows = c->hot_rows;
    a.nhot = c->nhot;
    a.key0 = (uint32_t)(c->P.seed & 0xFFFFFFFFu);
    a.key1 = (uint32_t)(c->P.seed >> 32);
    a.draw = draw;
    a.pur_nz = purpose_nz(set);
    a.pur_z = purpose_z(set);
    const bool obj = (set == SGCP_SAMPLES_FACTOR_OBJ || set == SGCP_SAMPLES_TEMPORAL_OBJ);
    a.p = obj ? c->P.p_obj : c->P.p;
    a.q = obj ? c->P.q_obj : c->P.q;
    a.all_nnz = 0;
    a.cap = c->P.zero_attempt_cap;
    a.want = want;
    a.loss = loss;
    a.eps = (float)c->P.log_eps;
    a.y_scale = (const float*)y_scale;
    a.err = c->err;
    a.skip = skip;
    a.cpl = c->P.sparse_cpl;
    return a;
}

template <typename T>
DenseGradArgs<T> dense_args(sgcp_ctx* c, const SliceDesc* slice_dev, int want, const void* s, const void* const* A,
                            void* const* G, void* gs, double* f, int loss, const void* y_scale, const int32_t* skip) {
    DenseGradArgs<T> a{};
    a.slice = slice_dev;
    a.inline_slice = c->cur;
    a.ndim = c->ndim;
    a.R = c->R;
    for (int k = 0; k < 3; ++k) a.dims[k] = c->dims[k];
    for (int k = 0; k < c->ndim; ++k) {
        a.A[k] = (const T*)A[k];
        a.G[k] = G ? (T*)G[k] : nullptr;
    }
    a.s = (const T*)s;
    a.gs = (T*)gs;
    a.f = f;
    a.want = want;
    a.loss = loss;
    a.eps = (T)c->P.log_eps;
    a.y_scale = (const T*)y_scale;
    a.skip = skip;
    a.xmap = (c->tc && c->xmap_ok) ? c->xmap : nullptr;
    return a;
}

// Gradient launch used by both the direct entry point and the step graph.
// Temporal-solver ADAM step fused into a temporal-gradient launch (nullptr = none).
struct TStepSpec {
    void *s, *u, *v;
    SolverState* st;
    const double* rate;
};

// A deferred ADAM step on s (sparse kernels): state in (s, u, v), previous gradient sum g,
// state out (written by one block); apply = 0 copies the state unchanged.
struct PendSpec {
    int apply;
    void *s, *u, *v;
    const double* rate;
    const void* g;
    void *s_out, *u_out, *v_out;
};

template <typename T>
TemporalStep<T> make_tstep(sgcp_ctx* c, const TStepSpec* ts) {
    TemporalStep<T> t{};
    t.s = (T*)ts->s;
    t.u = (T*)ts->u;
    t.v = (T*)ts->v;
    t.st = ts->st;
    t.rate = ts->rate;
    t.mu = c->P.mu;
    t.beta1 = c->P.beta1;
    t.beta2 = c->P.beta2;
    t.eps = c->P.adam_eps;
    t.lower = c->lower;
    return t;
}

sgcp_status enqueue_gradient(sgcp_ctx* c, bool sparse, const SliceDesc* slice_dev, int set, uint32_t draw, int want,
                             const void* s, const void* const* A, void* const* G, void* gs, double* f, int loss,
                             const void* y_scale, const int32_t* skip, int all_nnz = 0,
                             const TStepSpec* tstep = nullptr, bool overlap = false, float* zero_buf = nullptr,
                             int zero_n = 0, const PendSpec* pend = nullptr) {
    if (sparse) {
        SparseGradArgs a = sparse_args(c, slice_dev, set, draw, want, s, A, G, gs, f, loss, y_scale, skip);
        a.all_nnz = all_nnz;
        a.overlap = overlap ? 1 : 0;
        a.zero_buf = zero_buf;
        a.zero_n = zero_buf ? zero_n : 0;
        if (pend) {
            const TStepSpec in{pend->s, pend->u, pend->v, nullptr, pend->rate};
            a.pend_on = 1;
            a.pend_apply = pend->apply;
            a.pend = make_tstep<float>(c, &in);
            a.pend_g = (const float*)pend->g;
            a.pend_s_out = (float*)pend->s_out;
            a.pend_u_out = (float*)pend->u_out;
            a.pend_v_out = (float*)pend->v_out;
        }
        if (tstep) {
            a.tstep_on = 1;
            a.tstep = make_tstep<float>(c, tstep);
        }
        int64_t total;
        if (all_nnz) total = (int64_t)1 << 40;   // grid-stride over nnz (unknown when captured): full grid
        else {
            const bool obj = (set == SGCP_SAMPLES_FACTOR_OBJ || set == SGCP_SAMPLES_TEMPORAL_OBJ);
            total = obj ? c->P.p_obj + c->P.q_obj : c->P.p + c->P.q;
        }
        CK(launch_sparse_grad(a, total, c->stream, &c->launches), "sparse gradient");
    } else if (c->f64) {
        DenseGradArgs<double> a = dense_args<double>(c, slice_dev, want, s, A, G, gs, f, loss, y_scale, skip);
        if (tstep) {
            a.tstep_on = 1;
            a.tstep = make_tstep<double>(c, tstep);
        }
        CK(launch_dense_grad<double>(a, c->stream, &c->launches), "dense gradient");
    } else {
        DenseGradArgs<float> a = dense_args<float>(c, slice_dev, want, s, A, G, gs, f, loss, y_scale, skip);
        if (tstep) {
            a.tstep_on = 1;
            a.tstep = make_tstep<float>(c, tstep);
        }
        if (c->P.precision == SGCP_PREC_BF16_MTTKRP || c->P.precision == SGCP_PREC_F16_MTTKRP)
            CK(launch_dense_grad_tc(a, c->P.precision == SGCP_PREC_BF16_MTTKRP, c->err, c->stream, &c->launches),
               "dense tensor-core gradient");
        else
            CK(launch_dense_grad<float>(a, c->stream, &c->launches), "dense gradient");
    }
    return SGCP_OK;
}

// ---------------------------------------------------------------------------
// One OnlineGCP step (Alg. 1 body minus the host-side reservoir choice),
// enqueued on c->stream; captured into a graph by build_graph.
// ---------------------------------------------------------------------------
// Stored-slice history: the fused kernel on the slice kept in window slot j, at (A, s_h), every y
// and f scaled by the slot weight w_h; skipped while the slot is inactive or the solver is done.
// Its samples use their own purposes, the slot's time index and the step's draw base.
template <typename T>
sgcp_status enqueue_stored(sgcp_ctx* c, bool sparse, int j, bool obj, uint32_t draw, int want, const void* const* A,
                           void* const* G, double* f) {
    const SliceDesc* sd = c->hist_desc + j;
    const void* sh = offs(c->s_hist, (int64_t)j * c->R, c->esz);
    const void* wj = offs(c->hist_w, j, c->esz);
    const int32_t* sk = c->hist_skip + j;
    if (sparse) {
        SparseGradArgs a = sparse_args(c, sd, SGCP_SAMPLES_FACTOR_GRAD, draw, want, sh, A, G, nullptr, f, c->P.loss,
                                       wj, sk);
        a.pur_nz = obj ? PUR_HOBJ_NZ : PUR_HGRAD_NZ;
        a.pur_z = a.pur_nz + 1;
        a.p = obj ? c->P.p_obj : c->P.p;
        a.q = obj ? c->P.q_obj : c->P.q;
        a.nhot = 0;
        CK(launch_sparse_grad(a, a.p + a.q, c->stream, &c->launches), "stored-slice gradient");
    } else if (c->f64) {
        DenseGradArgs<double> a = dense_args<double>(c, sd, want, sh, A, G, nullptr, f, c->P.loss, wj, sk);
        a.xmap = nullptr;
        CK(launch_dense_grad<double>(a, c->stream, &c->launches), "stored-slice gradient");
    } else {
        DenseGradArgs<float> a = dense_args<float>(c, sd, want, sh, A, G, nullptr, f, c->P.loss, wj, sk);
        a.xmap = nullptr;
        if (c->tc)
            CK(launch_dense_grad_tc(a, c->P.precision == SGCP_PREC_BF16_MTTKRP, c->err, c->stream, &c->launches),
               "stored-slice gradient");
        else
            CK(launch_dense_grad<float>(a, c->stream, &c->launches), "stored-slice gradient");
    }
    return SGCP_OK;
}

// Grow a slot buffer to at least `bytes` (contents not kept).
sgcp_status slot_buffer(sgcp_ctx* c, void** p, size_t* cap, size_t bytes) {
    if (bytes <= *cap && *p) return SGCP_OK;
    dfree(c, *p);
    *p = nullptr;
    *cap = 0;
    if (sgcp_status st = dalloc(c, p, bytes)) return st;
    *cap = bytes;
    return SGCP_OK;
}

// Keep slice src (time index t) in window slot `slot`: a copy of its data, its own nonzero hash
// (sparse), and its device descriptor.  Queued on the context stream after the work that reads it.
sgcp_status store_slice(sgcp_ctx* c, int slot, bool sparse, const SliceDesc& src, int64_t t) {
    SliceDesc d{};
    d.nnz = src.nnz;
    d.t = t;
    const size_t vb = (size_t)src.nnz * (sparse ? sizeof(float) : c->esz);
    if (sgcp_status st = slot_buffer(c, &c->hs_vals[slot], &c->hs_vals_cap[slot], vb)) return st;
    if (vb) CK(cudaMemcpyAsync(c->hs_vals[slot], src.vals, vb, cudaMemcpyDeviceToDevice, c->stream), "store slice");
    d.vals = c->hs_vals[slot];
    if (sparse) {
        const size_t ib = (size_t)src.nnz * c->ndim * sizeof(int32_t);
        if (sgcp_status st = slot_buffer(c, &c->hs_idx[slot], &c->hs_idx_cap[slot], ib)) return st;
        if (ib) CK(cudaMemcpyAsync(c->hs_idx[slot], src.idx, ib, cudaMemcpyDeviceToDevice, c->stream), "store slice");
        d.idx = (const int32_t*)c->hs_idx[slot];
        int hl = 10;
        while (((int64_t)1 << hl) < 2 * src.nnz) ++hl;
        const size_t kb = ((size_t)1 << hl) * sizeof(unsigned long long);
        if (sgcp_status st = slot_buffer(c, &c->hs_keys[slot], &c->hs_keys_cap[slot], kb)) return st;
        CK(cudaMemsetAsync(c->hs_keys[slot], 0xFF, kb, c->stream), "clear slot hash");
        if (src.nnz > 0) {
            CK(launch_hash_build(d, c->ndim, c->dims, (unsigned long long*)c->hs_keys[slot], hl, c->err, c->stream),
               "slot hash");
            c->launches += 1;
        }
        d.hkeys = (const unsigned long long*)c->hs_keys[slot];
        d.hlog2 = hl;
    }
    CK(launch_write_desc(c->hist_desc + slot, d, c->stream, &c->launches), "slot descriptor");
    c->hist_sparse = sparse ? 1 : 0;
    return SGCP_OK;
}

template <typename T>
sgcp_status enqueue_lbfgs(sgcp_ctx* c);

template <typename T>
sgcp_status enqueue_step(sgcp_ctx* c, bool sparse, bool with_factor) {
    const int R = c->R, d = c->ndim;
    const sgcp_params& P = c->P;
    const size_t esz = sizeof(T);
    const void* Aptr[4];
    void* Gptr[4];
    for (int k = 0; k < d; ++k) {
        Aptr[k] = offs(c->A, c->row_off[k] * R, esz);
        Gptr[k] = offs(c->G, c->row_off[k] * R, esz);
    }
    GramArgs<T> ga{};
    ga.ndim = d;
    ga.R = R;
    for (int k = 0; k < 4; ++k) {
        ga.dims[k] = c->dims[k];
        ga.row_off[k] = c->row_off[k];
    }
    ga.A = (const T*)c->A;
    ga.Abar = (const T*)c->Abar;
    ga.part = (T*)c->gpart;
    ga.nblk = c->gram_nblk;
    ga.rows_per_block = c->gram_rpb;
    ga.out = c->grams;
    const int loss = P.loss;
    // fork / join of the side stream inside the capture
    auto fork = [&]() -> cudaError_t {
        cudaError_t e = cudaEventRecord(c->ev_fork, c->stream);
        return e == cudaSuccess ? cudaStreamWaitEvent(c->side, c->ev_fork, 0) : e;
    };
    auto join = [&]() -> cudaError_t {
        cudaError_t e = cudaEventRecord(c->ev_join, c->side);
        return e == cudaSuccess ? cudaStreamWaitEvent(c->stream, c->ev_join, 0) : e;
    };

    CK(launch_history_SH<T>(R, (const T*)c->s_hist, c->h_dev, c->hist_len_dev, c->slice_dev, P.w, P.theta, c->SH,
                            c->stream, &c->launches),
       "S_H");
    const bool stored = c->stored_hist;
    if (stored)
        CK(launch_hist_slots_begin<T>(c->hist_desc, (T*)c->hist_w, c->hist_skip, c->hist_len_dev, c->h_dev,
                                      c->slice_dev, P.w, P.theta, P.H, (uint32_t)((int64_t)P.kappa_f * P.tau_f),
                                      c->stream, &c->launches),
           "history slots");

    // ---------------- temporal weights (Alg. 3, or the least-squares solve) ----------------
    if (P.temporal == SGCP_TEMPORAL_LSQ) {
        ga.npairs = 1;
        ga.sel_u[0] = SEL_A;
        ga.sel_v[0] = SEL_A;
        ga.skip = nullptr;
        CK(launch_gram<T>(ga, c->nrows, c->stream, &c->launches), "gram");
        CK(cudaMemsetAsync(c->gs, 0, R * esz, c->stream), "clear gs");
        sgcp_status st = enqueue_gradient(c, sparse, c->slice_dev, SGCP_SAMPLES_TEMPORAL_GRAD, 0, SGCP_WANT_TEMPORAL,
                                          c->s, Aptr, nullptr, c->gs, nullptr, LOSS_IDENTITY_X, nullptr, nullptr, 1);
        if (st) return st;
        CK(launch_lsq_solve<T>(d, R, c->grams, (const T*)c->gs, P.mu, c->lower, (T*)c->s, c->lsq_work, c->err,
                               c->stream, &c->launches),
           "lsq solve");
    } else {
        SolverState* sw = c->st_w;
        const int32_t* skip = &sw->done;
        CK(launch_adam_reset<T>(R, (const T*)c->s, (T*)c->s_u, (T*)c->s_v, (T*)c->s_ao, (T*)c->s_uo, (T*)c->s_vo, 1,
                                (T*)c->s, c->stream, &c->launches),
           "adam init");
        CK(launch_solver_init(sw, P.alpha_w, 1, c->stream, &c->launches), "solver init");
        CK(cudaMemsetAsync(c->gs, 0, R * esz, c->stream), "clear gs");
        TStepSpec tsw{c->s, c->s_u, c->s_v, sw, c->rates_w};
        sgcp_status st = enqueue_gradient(c, sparse, c->slice_dev, SGCP_SAMPLES_TEMPORAL_OBJ, 0, SGCP_WANT_LOSS, c->s,
                                          Aptr, nullptr, nullptr, &sw->F_new, loss, nullptr, nullptr);
        if (st) return st;
        CK(launch_obj_finish_w<T>(sw, (const T*)c->s, R, P.mu, 1, c->err, nullptr, c->stream, &c->launches), "obj");
        // Sparse slices: the ADAM step on s of gradient kernel it runs at the start of kernel it + 1
        // (every block forms the new s itself), and the epoch's objective kernel applies the last
        // one.  The state after `it` steps lives in SP[(it + tau) % 2], so the state after tau steps
        // is in SP[0] = (s, s_u, s_v); gradient sums rotate over three buffers G3[it % 3], each
        // cleared by the kernel before the one that sums into it (the epoch's first by k_epoch_begin).
        const bool defer = sparse;
        const int tau = P.tau_w;
        float* G3 = (float*)c->gs3;
        void* SP[2][3] = {{c->s, c->s_u, c->s_v}, {c->s2, offs(c->s2, R, esz), offs(c->s2, 2 * R, esz)}};
        auto g3 = [&](int i) { return G3 + (size_t)(i % 3) * R; };
        for (int e = 0; e < P.kappa_w; ++e) {
            CK(launch_epoch_begin(sw, P.tol_w, c->rates_w, P.tau_w, P.beta1, P.beta2, c->stream, &c->launches,
                                  defer ? g3(0) : nullptr, R),
               "epoch begin");
            for (int it = 0; it < P.tau_w; ++it) {
                tsw.rate = c->rates_w + it;
                // a chain of gradient kernels: each one's sampling overlaps the one before
                if (defer) {
                    PendSpec ps{};
                    const PendSpec* pp = nullptr;
                    const int cur = (it + tau) & 1;
                    if (it == 0 && cur == 1) {   // odd tau: the epoch's start state copied into SP[1]
                        ps = PendSpec{0, SP[0][0], SP[0][1], SP[0][2], nullptr, nullptr, SP[1][0], SP[1][1], SP[1][2]};
                        pp = &ps;
                    } else if (it > 0) {
                        const int prev = cur ^ 1;
                        ps = PendSpec{1,       SP[prev][0], SP[prev][1], SP[prev][2], c->rates_w + it - 1,
                                      g3(it - 1), SP[cur][0], SP[cur][1], SP[cur][2]};
                        pp = &ps;
                    }
                    st = enqueue_gradient(c, sparse, c->slice_dev, SGCP_SAMPLES_TEMPORAL_GRAD,
                                          (uint32_t)(e * P.tau_w + it), SGCP_WANT_TEMPORAL, c->s, Aptr, nullptr, g3(it),
                                          nullptr, loss, nullptr, skip, 0, nullptr, true,
                                          it + 1 < tau ? g3(it + 1) : nullptr, R, pp);
                } else {
                    st = enqueue_gradient(c, sparse, c->slice_dev, SGCP_SAMPLES_TEMPORAL_GRAD,
                                          (uint32_t)(e * P.tau_w + it), SGCP_WANT_TEMPORAL, c->s, Aptr, nullptr, c->gs,
                                          nullptr, loss, nullptr, skip, 0, &tsw, true);
                }
                if (st) return st;
            }
            if (defer) {   // the epoch's last step (from SP[1]) lands in SP[0] as the objective is estimated
                const PendSpec ps{1,         SP[1][0], SP[1][1], SP[1][2], c->rates_w + tau - 1,
                                  g3(tau - 1), SP[0][0], SP[0][1], SP[0][2]};
                st = enqueue_gradient(c, sparse, c->slice_dev, SGCP_SAMPLES_TEMPORAL_OBJ, 0, SGCP_WANT_LOSS, c->s,
                                      Aptr, nullptr, nullptr, &sw->F_new, loss, nullptr, skip, 0, nullptr, true,
                                      nullptr, 0, &ps);
            } else {
                st = enqueue_gradient(c, sparse, c->slice_dev, SGCP_SAMPLES_TEMPORAL_OBJ, 0, SGCP_WANT_LOSS, c->s, Aptr,
                                      nullptr, nullptr, &sw->F_new, loss, nullptr, skip);
            }
            if (st) return st;
            CK(launch_obj_finish_w<T>(sw, (const T*)c->s, R, P.mu, 0, c->err, skip, c->stream, &c->launches), "obj");
            CK(launch_epoch_end<T>(sw, R, (T*)c->s, (T*)c->s_u, (T*)c->s_v, (T*)c->s_ao, (T*)c->s_uo, (T*)c->s_vo,
                                   P.tau_w, P.alpha_decay, P.beta1, P.beta2, c->stream, &c->launches),
               "epoch end");
        }
    }

    if (!with_factor) return SGCP_OK;
    if (P.optimizer == SGCP_OPT_LBFGS) {
        // ---------------- factor matrices: projected L-BFGS (dense slices) ----------------
        if (sgcp_status st = enqueue_lbfgs<T>(c)) return st;
        CK(cudaMemcpyAsync(c->Abar, c->A, (size_t)c->N * esz, cudaMemcpyDeviceToDevice, c->stream), "Abar <- A");
        return SGCP_OK;
    }
    // ---------------- factor matrices (Alg. 4) ----------------
    SolverState* sf = c->st_f;
    const int32_t* skip = &sf->done;
    const bool hist_possible = P.H > 0 && !stored;   // the model-based history terms
    CK(launch_solver_init(sf, P.alpha_f, 0, c->stream, &c->launches), "solver init");
    auto objective_f = [&](int set_cur, const int32_t* sk) -> sgcp_status {
        CK(fork(), "fork");
        sgcp_status st2 = enqueue_gradient(c, sparse, c->slice_dev, SGCP_SAMPLES_FACTOR_OBJ, 0, SGCP_WANT_LOSS, c->s,
                                           Aptr, nullptr, nullptr, &sf->F_new, loss, nullptr, sk);
        if (st2) return st2;
        if (stored) {
            // sum_h w_h sum_i f(x_ih, m_ih) over the stored slices, then lambda/2 ||A||^2 from A'A
            for (int j = 0; j < P.H; ++j)
                if ((st2 = enqueue_stored<T>(c, sparse, j, true, 0, SGCP_WANT_LOSS, Aptr, nullptr, &sf->F_new)))
                    return st2;
            GramArgs<T> g1 = ga;
            g1.npairs = 1;
            g1.sel_u[0] = SEL_A;
            g1.sel_v[0] = SEL_A;
            g1.skip = sk;
            CK(launch_gram<T>(g1, c->nrows, c->side, &c->launches), "gram");
            CK(join(), "join");
            CK(launch_obj_finish_f(sf, d, R, c->grams, c->SH, c->zero_i, P.lambda, set_cur, c->err, sk, c->stream,
                                   &c->launches),
               "obj f");
            return SGCP_OK;
        }
        GramArgs<T> g6 = ga;
        g6.npairs = 6;
        const int su[6] = {SEL_A, SEL_ABAR, SEL_ABAR, SEL_D, SEL_D, SEL_ABAR};
        const int sv[6] = {SEL_A, SEL_ABAR, SEL_A, SEL_D, SEL_A, SEL_D};
        for (int i = 0; i < 6; ++i) {
            g6.sel_u[i] = su[i];
            g6.sel_v[i] = sv[i];
        }
        g6.skip = sk;
        CK(launch_gram<T>(g6, c->nrows, c->side, &c->launches), "gram6");
        CK(join(), "join");
        CK(launch_obj_finish_f(sf, d, R, c->grams, c->SH, c->hist_len_dev, P.lambda, set_cur, c->err, sk, c->stream,
                               &c->launches),
           "obj f");
        return SGCP_OK;
    };
    sgcp_status st = objective_f(1, nullptr);
    if (st) return st;
    FactorUpdateArgs<T> fu{};
    fu.ndim = d;
    fu.R = R;
    fu.nrows = c->nrows;
    for (int k = 0; k < 4; ++k) fu.row_off[k] = c->row_off[k];
    fu.A = (T*)c->A;
    fu.Abar = (const T*)c->Abar;
    fu.G = (T*)c->G;
    fu.u = (T*)c->u;
    fu.v = (T*)c->v;
    fu.B = hist_possible ? (const T*)c->Bc : nullptr;
    fu.C = hist_possible ? (const T*)c->Cc : nullptr;
    fu.hist_len = c->hist_len_dev;
    fu.lam = P.lambda;
    fu.beta1 = P.beta1;
    fu.beta2 = P.beta2;
    fu.eps = P.adam_eps;
    fu.lower = c->lower;
    fu.skip = skip;
    // With gacc each update also sums the Grams of the factors it writes (two alternating buffers)
    // and the next update forms its B_k, C_k from them, so the Gram / history-coefficient chain
    // beside the gradient runs only for an epoch's first iteration (whose A may have been rolled
    // back).  The update of iteration it accumulates into buffer it % 2 (except the epoch's last
    // update, whose sums no update would read), which is zero when it starts: cleared by the
    // sparse gradient kernel of the same iteration, or (dense) by the last block of the update
    // that read it.
    const bool fused = hist_possible && c->gacc != nullptr;
    const size_t gsz = 2 * (size_t)d * R * R;
    if (fused) {
        fu.SH = c->SH;
        fu.tk = sf;
        CK(cudaMemsetAsync(c->gacc, 0, 2 * gsz * sizeof(float), c->stream), "clear Gram sums");
    }
    for (int e = 0; e < P.kappa_f; ++e) {
        CK(launch_epoch_begin(sf, P.tol_f, c->rates_f, P.tau_f, P.beta1, P.beta2, c->stream, &c->launches),
           "epoch begin");
        if (stored)
            CK(launch_hist_slots_skip(c->hist_skip, c->hist_len_dev, &sf->done, P.H, c->stream, &c->launches),
               "history slots");
        for (int it = 0; it < P.tau_f; ++it) {
            fu.rate = c->rates_f + it;
            float* gclear = nullptr;   // sparse: the gradient kernel clears the buffer this update sums into
            if (fused) {
                float* prev = c->gacc + gsz * ((it + 1) & 1);   // written by the update of it - 1
                fu.gprev = it > 0 ? prev : nullptr;
                fu.gacc = it + 1 < P.tau_f ? c->gacc + gsz * (it & 1) : nullptr;
                // the buffer update it - 1 read is cleared before update it adds into it: by the
                // gradient kernel between the two (sparse), else by update it - 1's last block
                fu.gzero = (it > 0 && !sparse) ? prev : nullptr;
                if (sparse) gclear = fu.gacc;
            }
            const bool chain = hist_possible && (!fused || it == 0);
            if (chain) CK(fork(), "fork");
            // gradient and update overlap their neighbours in the chain (the update only when no
            // side-stream join precedes it)
            st = enqueue_gradient(c, sparse, c->slice_dev, SGCP_SAMPLES_FACTOR_GRAD, (uint32_t)(e * P.tau_f + it),
                                  SGCP_WANT_FACTORS, c->s, Aptr, Gptr, nullptr, nullptr, loss, nullptr, skip, 0,
                                  nullptr, true, gclear, (int)gsz);
            if (st) return st;
            for (int j = 0; stored && j < P.H; ++j)   // + sum_h w_h Y_h(k) Z_k diag(s_h)
                if ((st = enqueue_stored<T>(c, sparse, j, false, (uint32_t)(e * P.tau_f + it), SGCP_WANT_FACTORS, Aptr,
                                            Gptr, nullptr)))
                    return st;
            if (chain) {
                // history coefficients from the current A, beside the gradient kernel
                GramArgs<T> g2 = ga;
                g2.npairs = 2;
                g2.sel_u[0] = SEL_A;
                g2.sel_v[0] = SEL_A;
                g2.sel_u[1] = SEL_D;
                g2.sel_v[1] = SEL_A;
                g2.skip = skip;
                CK(launch_gram<T>(g2, c->nrows, c->side, &c->launches), "gram2");
                CK(launch_hist_coeffs<T>(d, R, c->grams, 1, c->SH, c->hist_len_dev, (T*)c->Bc, (T*)c->Cc, skip,
                                         c->side, &c->launches),
                   "hist coeffs");
                CK(join(), "join");
            }
            fu.overlap = chain ? 0 : 1;
            CK(launch_factor_update<T>(fu, c->stream, &c->launches), "factor update");
        }
        st = objective_f(0, skip);
        if (st) return st;
        CK(launch_epoch_end<T>(sf, c->N, (T*)c->A, (T*)c->u, (T*)c->v, (T*)c->a_o, (T*)c->u_o, (T*)c->v_o, P.tau_f,
                               P.alpha_decay, P.beta1, P.beta2, c->stream, &c->launches),
           "epoch end");
    }
    CK(cudaMemcpyAsync(c->Abar, c->A, (size_t)c->N * esz, cudaMemcpyDeviceToDevice, c->stream), "Abar <- A");
    return SGCP_OK;
}

// ---------------------------------------------------------------------------
// Projected L-BFGS on the factor matrices of a dense slice (the paper's
// conclusions ask for solvers other than SGD; this one follows Nocedal &
// Wright, "Numerical Optimization", Alg. 7.4, with a backtracking Armijo line
// search on the projected point), enqueued into the step graph: every
// evaluation (the dense loss + gradient, the telescoped history objective, the
// history / lambda gradient terms) and every scalar of the recursion stay on
// the device.  Each of the lbfgs_iters iterations is a direction kernel, the
// first line-search trial (trial point, evaluation, Armijo test), a WHILE
// conditional node whose body is one further trial and which runs only while
// the Armijo test rejects, and an update kernel.
// ---------------------------------------------------------------------------
template <typename T>
sgcp_status enqueue_lbfgs(sgcp_ctx* c) {
    const int d = c->ndim, R = c->R;
    const size_t nb = (size_t)c->N * sizeof(T);
    const void* Aptr[4];
    void* Gptr[4];
    for (int k = 0; k < d; ++k) {
        Aptr[k] = offs(c->A, c->row_off[k] * R, sizeof(T));
        Gptr[k] = offs(c->G, c->row_off[k] * R, sizeof(T));
    }
    GramArgs<T> ga{};
    ga.ndim = d;
    ga.R = R;
    for (int k = 0; k < 4; ++k) {
        ga.dims[k] = c->dims[k];
        ga.row_off[k] = c->row_off[k];
    }
    ga.A = (const T*)c->A;
    ga.Abar = (const T*)c->Abar;
    ga.part = (T*)c->gpart;
    ga.nblk = c->gram_nblk;
    ga.rows_per_block = c->gram_rpb;
    ga.out = c->grams;
    FactorUpdateArgs<T> fu{};
    fu.ndim = d;
    fu.R = R;
    fu.nrows = c->nrows;
    for (int k = 0; k < 4; ++k) fu.row_off[k] = c->row_off[k];
    fu.A = (T*)c->A;
    fu.Abar = (const T*)c->Abar;
    fu.G = (T*)c->G;
    fu.u = (T*)c->u;
    fu.v = (T*)c->v;
    fu.B = c->P.H > 0 ? (const T*)c->Bc : nullptr;
    fu.C = c->P.H > 0 ? (const T*)c->Cc : nullptr;
    fu.hist_len = c->hist_len_dev;
    fu.lam = c->P.lambda;
    fu.beta1 = c->P.beta1;
    fu.beta2 = c->P.beta2;
    fu.eps = c->P.adam_eps;
    fu.lower = c->lower;
    fu.rate = c->rates_f;
    fu.grad_only = 1;
    SolverState* sf = c->st_f;
    // F(A) into sf->F_new and the full gradient of eq. gcp_stream_objective into G, on c->stream;
    // every kernel skips while *skip (the solve has stopped)
    const int32_t* skip = nullptr;
    auto eval = [&]() -> sgcp_status {
        CK(cudaMemsetAsync(c->G, 0, nb, c->stream), "clear G");
        CK(cudaMemsetAsync(&sf->F_new, 0, sizeof(double), c->stream), "clear F");
        sgcp_status e2 = enqueue_gradient(c, false, c->slice_dev, SGCP_SAMPLES_FACTOR_GRAD, 0,
                                          SGCP_WANT_FACTORS | SGCP_WANT_LOSS, c->s, Aptr, Gptr, nullptr, &sf->F_new,
                                          c->P.loss, nullptr, skip);
        if (e2) return e2;
        GramArgs<T> g6 = ga;
        g6.npairs = 6;
        const int su[6] = {SEL_A, SEL_ABAR, SEL_ABAR, SEL_D, SEL_D, SEL_ABAR};
        const int sv[6] = {SEL_A, SEL_ABAR, SEL_A, SEL_D, SEL_A, SEL_D};
        for (int i = 0; i < 6; ++i) {
            g6.sel_u[i] = su[i];
            g6.sel_v[i] = sv[i];
        }
        g6.skip = skip;
        CK(launch_gram<T>(g6, c->nrows, c->stream, &c->launches), "gram6");
        CK(launch_obj_finish_f(sf, d, R, c->grams, c->SH, c->hist_len_dev, c->P.lambda, 0, c->err, skip, c->stream,
                               &c->launches),
           "objective");
        // history coefficients from the same Grams: A'A is pair 0 and D'A pair 4 of the six
        if (c->P.H > 0)
            CK(launch_hist_coeffs<T>(d, R, c->grams, 4, c->SH, c->hist_len_dev, (T*)c->Bc, (T*)c->Cc, skip, c->stream,
                                     &c->launches),
               "hist coeffs");
        fu.skip = skip;
        CK(launch_factor_update<T>(fu, c->stream, &c->launches), "gradient terms");
        return SGCP_OK;
    };
    LbfgsArgs<T> la{};
    la.ls = c->lb_state;
    la.sf = sf;
    la.A = (T*)c->A;
    la.G = (const T*)c->G;
    la.x = (T*)c->lb_x;
    la.g = (T*)c->lb_g;
    la.pd = (T*)c->lb_p;
    la.S = (T* const*)c->lb_tab;
    la.Y = (T* const*)(c->lb_tab + kLbfgsSlots);
    la.n = c->N;
    la.m = c->P.lbfgs_mem;
    la.lower = c->lower;

    if (sgcp_status e = eval()) return e;
    CK(launch_lbfgs_begin<T>(la, c->stream, &c->launches), "lbfgs begin");
    for (int it = 0; it < c->P.lbfgs_iters; ++it) {
        cudaStreamCaptureStatus cs;
        cudaGraph_t g = nullptr;
        CK(cudaStreamGetCaptureInfo(c->stream, &cs, nullptr, &g, nullptr, nullptr, nullptr), "capture info");
        if (cs != cudaStreamCaptureStatusActive) return fail(c, SGCP_ERR_CUDA, "lbfgs: step graph not capturing");
        // 0 at every graph launch; an Armijo test that rejects its trial raises it
        cudaGraphConditionalHandle h;
        CK(cudaGraphConditionalHandleCreate(&h, g, 0u, cudaGraphCondAssignDefault), "conditional handle");
        CK(launch_lbfgs_direction<T>(la, c->stream, &c->launches), "lbfgs direction");
        // the first trial (step 1) in line: every kernel of it skips once the solve has stopped
        skip = &c->lb_state->done;
        CK(launch_lbfgs_trial<T>(la, c->stream, &c->launches), "lbfgs trial");
        if (sgcp_status e = eval()) return e;
        skip = nullptr;
        CK(launch_lbfgs_armijo<T>(la, h, c->stream, &c->launches), "lbfgs armijo");
        // further trials (step 1/2, 1/4, ...) only when it was rejected: a WHILE node whose body is
        // one trial, captured on the side stream
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        CK(cudaStreamGetCaptureInfo(c->stream, &cs, nullptr, &g, &deps, nullptr, &nd), "capture info");
        cudaGraphNodeParams np{};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        CK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &np), "line-search node");
        cudaGraph_t body = np.conditional.phGraph_out[0];
        CK(cudaStreamUpdateCaptureDependencies(c->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies),
           "capture dependencies");
        cudaStream_t main = c->stream;
        CK(cudaStreamBeginCaptureToGraph(c->lb_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed),
           "begin body capture");
        c->stream = c->lb_stream;
        sgcp_status e = SGCP_OK;
        cudaError_t ce = launch_lbfgs_trial<T>(la, c->stream, &c->launches);
        if (ce == cudaSuccess) e = eval();
        if (ce == cudaSuccess && e == SGCP_OK) ce = launch_lbfgs_armijo<T>(la, h, c->stream, &c->launches);
        c->stream = main;
        cudaGraph_t out = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(c->lb_stream, &out);
        if (e) return e;
        if (ce != cudaSuccess) return cuda_fail(c, ce, "line-search body");
        if (ee != cudaSuccess) return cuda_fail(c, ee, "end body capture");
        CK(launch_lbfgs_update<T>(la, c->stream, &c->launches), "lbfgs update");
    }
    CK(launch_lbfgs_finish(c->lb_state, sf, c->stream, &c->launches), "lbfgs finish");
    CK(cudaMemsetAsync(c->G, 0, nb, c->stream), "clear G");
    return SGCP_OK;
}

// ---------------------------------------------------------------------------
// Warm start: static GCP-SGD on the first n slices stacked as a (d+1)-way
// tensor whose last mode indexes the slices (Sec. 4.4, Sec. 6), with S
// (n x R) that mode's factor matrix.  The loss gradient of the stack splits by
// slice: dF/dA^(k) = sum_h Y_h(k) Z_k diag(S_h) and dF/dS_h = Z' vec(Y_h), so
// each iteration runs the fused gradient kernel once per slice at s = S_h,
// accumulating G^(k) and writing row h of the S gradient.  The variables
// [A^(1..d); S] sit in one buffer, so the ADAM row update, the epoch test and
// the rollback are the factor solver's kernels (Alg. 2, Alg. 4 without the
// history term); lambda regularises every matrix of the stack.  Sparse slices
// are sampled per slice (p + q samples each, slice h at time index h), each
// with its own nonzero hash.
// ---------------------------------------------------------------------------
template <typename T>
sgcp_status warm_start_impl(sgcp_ctx* c, int n, const sgcp_slice* X, const void* S_init, void* S_out,
                            sgcp_warm_stats* out) {
    const int d = c->ndim, R = c->R;
    const sgcp_params& P = c->P;
    const bool sparse = X[0].is_sparse != 0;
    const int64_t rows = c->nrows + n, N2 = rows * R;
    const size_t nb = (size_t)N2 * sizeof(T);
    cudaStream_t st = c->stream;
    std::vector<void*> tmp;   // released (after the stream has drained) on every return path
    auto grab = [&](void** p, size_t bytes) -> sgcp_status {
        sgcp_status e = dalloc(c, p, bytes);
        if (e == SGCP_OK) tmp.push_back(*p);
        return e;
    };
    struct Release {
        sgcp_ctx* c;
        std::vector<void*>* v;
        ~Release() {
            if (c->stream) cudaStreamSynchronize(c->stream);
            for (void* p : *v) dfree(c, p);
        }
    } release{c, &tmp};

    void *W = nullptr, *G2 = nullptr, *u2 = nullptr, *v2 = nullptr, *uo2 = nullptr, *vo2 = nullptr, *ao2 = nullptr;
    void *rates = nullptr, *sst = nullptr;
    void** bufs[] = {&W, &G2, &u2, &v2, &uo2, &vo2, &ao2};
    for (void** b : bufs)
        if (sgcp_status e = grab(b, nb)) return e;
    if (sgcp_status e = grab(&rates, (size_t)(P.tau_f > 0 ? P.tau_f : 1) * sizeof(double))) return e;
    if (sgcp_status e = grab(&sst, sizeof(SolverState))) return e;
    SolverState* sw = (SolverState*)sst;

    // the slices on the device: descriptors, staged copies, hashes
    std::vector<SliceDesc> desc(n);
    std::vector<unsigned long long*> keys(n, nullptr);
    std::vector<int> hl(n, 0);
    for (int h = 0; h < n; ++h) {
        const sgcp_slice& x = X[h];
        const int64_t nnz = sparse ? x.nnz : omega_of(c);
        const void* idx_d = x.idx;
        const void* vals_d = x.vals;
        const bool restage = !x.on_host && !sparse && c->tc && (reinterpret_cast<uintptr_t>(x.vals) & 15) != 0;
        if (x.on_host || restage) {
            const size_t ib = sparse ? (size_t)nnz * d * sizeof(int32_t) : 0;
            const size_t vb = (size_t)nnz * (sparse ? sizeof(float) : c->esz);
            const cudaMemcpyKind kind = x.on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
            void *ip = nullptr, *vp = nullptr;
            if (ib) {
                if (sgcp_status e = grab(&ip, ib)) return e;
                CK(cudaMemcpyAsync(ip, x.idx, ib, kind, st), "stage slice idx");
            }
            if (vb) {
                if (sgcp_status e = grab(&vp, vb)) return e;
                CK(cudaMemcpyAsync(vp, x.vals, vb, kind, st), "stage slice vals");
            }
            idx_d = ip;
            vals_d = vp;
        }
        desc[h].idx = (const int32_t*)idx_d;
        desc[h].vals = vals_d;
        desc[h].nnz = nnz;
        desc[h].t = h + 1;
        if (sparse && nnz > 0) {
            int b = 10;
            while (((int64_t)1 << b) < 2 * nnz) ++b;
            hl[h] = b;
            void* kp = nullptr;
            if (sgcp_status e = grab(&kp, ((size_t)1 << b) * sizeof(unsigned long long))) return e;
            keys[h] = (unsigned long long*)kp;
            CK(cudaMemsetAsync(kp, 0xFF, ((size_t)1 << b) * sizeof(unsigned long long), st), "clear hash");
            CK(launch_hash_build(desc[h], d, c->dims, keys[h], b, c->err, st), "hash");
            c->launches += 1;
        }
    }

    // the stacked variables: the context's factors, then S (given, or ones)
    CK(cudaMemcpyAsync(W, c->A, (size_t)c->N * sizeof(T), cudaMemcpyDeviceToDevice, st), "stack factors");
    T* S = (T*)offs(W, c->nrows * R, sizeof(T));
    if (S_init) {
        CK(cudaMemcpyAsync(S, S_init, (size_t)n * R * sizeof(T), cudaMemcpyDeviceToDevice, st), "stack S");
    } else {
        std::vector<T> ones((size_t)n * R, T(1));
        CK(cudaMemcpyAsync(S, ones.data(), ones.size() * sizeof(T), cudaMemcpyHostToDevice, st), "stack S");
        CK(cudaStreamSynchronize(st), "stack S");   // the host vector dies here
    }
    CK(cudaMemsetAsync(G2, 0, nb, st), "clear G");
    CK(launch_adam_reset<T>(N2, (const T*)W, (T*)u2, (T*)v2, (T*)ao2, (T*)uo2, (T*)vo2, 0, (T*)W, st, &c->launches),
       "adam init");
    SolverState s0{};
    s0.b1pow = 1.0;
    s0.b2pow = 1.0;
    CK(cudaMemcpyAsync(sw, &s0, sizeof(s0), cudaMemcpyHostToDevice, st), "solver state");
    CK(cudaStreamSynchronize(st), "solver state");
    CK(launch_solver_init(sw, P.alpha_f, 1, st, &c->launches), "solver init");

    const void* Aw[4];
    void* Gw[4];
    for (int k = 0; k < d; ++k) {
        Aw[k] = offs(W, c->row_off[k] * R, sizeof(T));
        Gw[k] = offs(G2, c->row_off[k] * R, sizeof(T));
    }
    // one slice's fused kernel at s = S_h
    auto slice_grad = [&](int h, int set, uint32_t draw, int want, void* gs, double* f,
                          const int32_t* skip) -> sgcp_status {
        const void* sh = offs(S, (int64_t)h * R, sizeof(T));
        if (sparse) {
            SparseGradArgs a = sparse_args(c, nullptr, set, draw, want, sh, Aw, Gw, gs, f, P.loss, nullptr, skip);
            a.inline_slice = desc[h];
            a.hkeys = keys[h];
            a.hlog2 = hl[h];
            a.nhot = 0;
            const bool obj = set == SGCP_SAMPLES_FACTOR_OBJ;
            CK(launch_sparse_grad(a, obj ? P.p_obj + P.q_obj : P.p + P.q, st, &c->launches), "sparse gradient");
        } else if (c->f64) {
            DenseGradArgs<double> a = dense_args<double>(c, nullptr, want, sh, Aw, Gw, gs, f, P.loss, nullptr, skip);
            a.inline_slice = desc[h];
            a.xmap = nullptr;
            CK(launch_dense_grad<double>(a, st, &c->launches), "dense gradient");
        } else {
            DenseGradArgs<float> a = dense_args<float>(c, nullptr, want, sh, Aw, Gw, gs, f, P.loss, nullptr, skip);
            a.inline_slice = desc[h];
            a.xmap = nullptr;
            if (c->tc)
                CK(launch_dense_grad_tc(a, P.precision == SGCP_PREC_BF16_MTTKRP, c->err, st, &c->launches),
                   "dense tensor-core gradient");
            else
                CK(launch_dense_grad<float>(a, st, &c->launches), "dense gradient");
        }
        return SGCP_OK;
    };
    auto objective = [&](int set_cur, const int32_t* skip) -> sgcp_status {
        CK(cudaMemsetAsync(&sw->F_new, 0, sizeof(double), st), "clear F");
        for (int h = 0; h < n; ++h)
            if (sgcp_status e = slice_grad(h, SGCP_SAMPLES_FACTOR_OBJ, 0, SGCP_WANT_LOSS, nullptr, &sw->F_new, skip))
                return e;
        CK(launch_reg_objective<T>(sw, (const T*)W, N2, P.lambda, set_cur, c->err, skip, st, &c->launches),
           "objective");
        return SGCP_OK;
    };
    if (sgcp_status e = objective(1, nullptr)) return e;
    FactorUpdateArgs<T> fu{};
    fu.ndim = d;
    fu.R = R;
    fu.nrows = rows;
    for (int k = 0; k < 4; ++k) fu.row_off[k] = k < d ? c->row_off[k] : c->nrows;
    fu.A = (T*)W;
    fu.Abar = (const T*)W;   // no history term: the reference factors are not read
    fu.G = (T*)G2;
    fu.u = (T*)u2;
    fu.v = (T*)v2;
    fu.B = nullptr;
    fu.C = nullptr;
    fu.hist_len = c->hist_len_dev;
    fu.lam = P.lambda;
    fu.beta1 = P.beta1;
    fu.beta2 = P.beta2;
    fu.eps = P.adam_eps;
    fu.lower = c->lower;
    const int32_t* skip = &sw->done;
    fu.skip = skip;
    for (int e = 0; e < P.kappa_f; ++e) {
        CK(launch_epoch_begin(sw, P.tol_f, (double*)rates, P.tau_f, P.beta1, P.beta2, st, &c->launches),
           "epoch begin");
        for (int it = 0; it < P.tau_f; ++it) {
            for (int h = 0; h < n; ++h)
                if (sgcp_status e2 = slice_grad(h, SGCP_SAMPLES_FACTOR_GRAD, (uint32_t)(e * P.tau_f + it),
                                                SGCP_WANT_FACTORS | SGCP_WANT_TEMPORAL,
                                                offs(G2, (c->nrows + h) * R, sizeof(T)), nullptr, skip))
                    return e2;
            fu.rate = (const double*)rates + it;
            CK(launch_factor_update<T>(fu, st, &c->launches), "stacked update");
        }
        if (sgcp_status e2 = objective(0, skip)) return e2;
        CK(launch_epoch_end<T>(sw, N2, (T*)W, (T*)u2, (T*)v2, (T*)ao2, (T*)uo2, (T*)vo2, P.tau_f, P.alpha_decay,
                               P.beta1, P.beta2, st, &c->launches),
           "epoch end");
    }
    // the stream's state at t = n: factors (also Abar and the ADAM checkpoint), s = S_n, and the
    // window filled by the reservoir rule of Alg. 1 as the warm-start slices enter in order
    const size_t na = (size_t)c->N * sizeof(T);
    CK(cudaMemcpyAsync(c->A, W, na, cudaMemcpyDeviceToDevice, st), "factors");
    CK(cudaMemcpyAsync(c->Abar, W, na, cudaMemcpyDeviceToDevice, st), "Abar");
    CK(cudaMemcpyAsync(c->a_o, W, na, cudaMemcpyDeviceToDevice, st), "checkpoint");
    CK(cudaMemcpyAsync(c->s, offs(S, (int64_t)(n - 1) * R, sizeof(T)), (size_t)R * sizeof(T),
                       cudaMemcpyDeviceToDevice, st),
       "s");
    if (S_out) CK(cudaMemcpyAsync(S_out, S, (size_t)n * R * sizeof(T), cudaMemcpyDeviceToDevice, st), "S out");
    for (int h = 1; h <= n && P.H > 0; ++h) {
        int slot = -1;
        int len = (int)c->hist_t.size();
        if (len < P.H) {
            slot = len;
            c->hist_t.push_back(h);
            len += 1;
        } else {
            const uint32_t j = reservoir_index(P.seed, h);
            if ((int64_t)j <= P.H) {
                slot = (int)j - 1;
                c->hist_t[slot] = h;
            }
        }
        if (slot >= 0) {
            CK(launch_hist_update<T>(R, (T*)c->s_hist, c->h_dev, c->hist_len_dev, slot, h, len,
                                     (const T*)offs(S, (int64_t)(h - 1) * R, sizeof(T)), st, &c->launches),
               "history");
            if (c->stored_hist)
                if (sgcp_status e = store_slice(c, slot, sparse, desc[h - 1], h)) return e;
        }
    }
    SolverState fin{};
    CK(cudaMemcpyAsync(&fin, sw, sizeof(fin), cudaMemcpyDeviceToHost, st), "read state");
    CK(cudaStreamSynchronize(st), "warm start");
    if (out) {
        out->F = fin.F_cur;
        out->epochs = fin.epoch;
        out->accept = fin.accept;
    }
    c->t = n;
    c->loaded = false;
    return SGCP_OK;
}

sgcp_status build_graph(sgcp_ctx* c, bool sparse) {
    const int gi = sparse ? 1 : 0;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed), "begin capture");
    const int64_t before = c->launches;
    sgcp_status st = c->f64 ? enqueue_step<double>(c, sparse, true) : enqueue_step<float>(c, sparse, true);
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    c->launches = before;
    if (st != SGCP_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
    size_t n = 0;
    cudaGraphGetNodes(g, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    if (n) cudaGraphGetNodes(g, nodes.data(), &n);
    int64_t kernels = 0;
    for (size_t i = 0; i < n; ++i) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nodes[i], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++kernels;
    }
    e = cudaGraphInstantiate(&c->graph[gi], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(c, e, "instantiate graph");
    c->graph_kernels[gi] = kernels;
    return SGCP_OK;
}

sgcp_status check_ready(sgcp_ctx* c) {
    if (!c) return SGCP_ERR_ARG;
    if (c->sticky != SGCP_OK) return SGCP_ERR_STATE;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    return SGCP_OK;
}

sgcp_status status_from_err(int bits) {
    if (bits & ERRB_TIMEOUT) return SGCP_ERR_TIMEOUT;
    if (bits & (ERRB_COORD | ERRB_DUP)) return SGCP_ERR_DATA;
    if (bits & ERRB_SAMPLING) return SGCP_ERR_SAMPLING_LIMIT;
    if (bits & (ERRB_NUMERIC | ERRB_SOLVE)) return SGCP_ERR_NUMERIC;
    if (bits) return SGCP_ERR_STATE;
    return SGCP_OK;
}

}  // namespace

extern "C" {

const char* sgcp_version(void) { return "sgcp 0.1.0 (sm_103a)"; }

const char* sgcp_status_string(sgcp_status s) {
    switch (s) {
        case SGCP_OK: return "SGCP_OK";
        case SGCP_ERR_ARG: return "SGCP_ERR_ARG";
        case SGCP_ERR_CUDA: return "SGCP_ERR_CUDA";
        case SGCP_ERR_OOM: return "SGCP_ERR_OOM";
        case SGCP_ERR_SAMPLING_LIMIT: return "SGCP_ERR_SAMPLING_LIMIT";
        case SGCP_ERR_TIMEOUT: return "SGCP_ERR_TIMEOUT";
        case SGCP_ERR_NUMERIC: return "SGCP_ERR_NUMERIC";
        case SGCP_ERR_STATE: return "SGCP_ERR_STATE";
        case SGCP_ERR_UNSUPPORTED: return "SGCP_ERR_UNSUPPORTED";
        case SGCP_ERR_DATA: return "SGCP_ERR_DATA";
    }
    return "SGCP_ERR_UNKNOWN";
}

sgcp_status sgcp_params_default(sgcp_params* p) {
    if (!p) return SGCP_ERR_ARG;
    std::memset(p, 0, sizeof(*p));
    p->ndim = 3;
    p->rank = 8;
    p->loss = SGCP_LOSS_GAUSSIAN;
    p->precision = SGCP_PREC_F32;
    p->lower_bound = std::nan("");
    p->log_eps = 1e-10;
    p->H = 0;
    p->temporal = SGCP_TEMPORAL_ADAM;
    p->w = 1.0;
    p->theta = 1.0;
    p->lambda = 0.0;
    p->mu = 0.0;
    p->tol_w = -INFINITY;
    p->tol_f = -INFINITY;
    p->kappa_w = 5;
    p->kappa_f = 5;
    p->tau_w = 100;
    p->tau_f = 100;
    p->alpha_w = 0.1;
    p->alpha_f = 1e-3;
    p->beta1 = 0.9;
    p->beta2 = 0.999;
    p->adam_eps = 1e-8;
    p->alpha_decay = 0.1;
    p->zero_attempt_cap = 64;
    p->optimizer = SGCP_OPT_ADAM;
    p->lbfgs_mem = 5;
    p->lbfgs_iters = 10;
    p->sparse_cpl = 0;
    p->hot_rows = -1;
    p->seed = 0;
    return SGCP_OK;
}

sgcp_status sgcp_create(const sgcp_params* params, const void* const* init_factors, int32_t n_hist,
                        const int64_t* hist_t, const void* hist_s, int64_t t0, const sgcp_allocator* allocator,
                        void* cuda_stream, sgcp_ctx** out) {
    if (!params || !init_factors || !out) return SGCP_ERR_ARG;
    if (allocator && (!allocator->alloc || !allocator->free)) return SGCP_ERR_ARG;
    *out = nullptr;
    const sgcp_params& P = *params;
    if (P.ndim < 2 || P.ndim > 4) return SGCP_ERR_UNSUPPORTED;
    if (P.rank < 4 || P.rank > 128 || P.rank % 4 != 0) return SGCP_ERR_UNSUPPORTED;
    if (P.loss < 0 || P.loss > 3) return SGCP_ERR_ARG;
    if (P.precision < 0 || P.precision > 3) return SGCP_ERR_ARG;
    if ((P.precision == SGCP_PREC_BF16_MTTKRP || P.precision == SGCP_PREC_F16_MTTKRP) &&
        (P.ndim != 3 || P.rank % 16 != 0 || P.rank > 64))
        return SGCP_ERR_UNSUPPORTED;   // the tensor-core dense kernel covers 3-way slices, R in {16, 32, 48, 64}
    if (P.optimizer != SGCP_OPT_ADAM && P.optimizer != SGCP_OPT_LBFGS) return SGCP_ERR_ARG;
    if (P.optimizer == SGCP_OPT_LBFGS && (P.lbfgs_mem < 1 || P.lbfgs_mem > 64 || P.lbfgs_iters < 0)) return SGCP_ERR_ARG;
    if (P.temporal == SGCP_TEMPORAL_LSQ && P.loss != SGCP_LOSS_GAUSSIAN) return SGCP_ERR_ARG;
    if (P.H < 0 || n_hist < 0 || n_hist > P.H || (n_hist > 0 && (!hist_t || !hist_s))) return SGCP_ERR_ARG;
    if (P.kappa_w < 0 || P.kappa_f < 0 || P.tau_w < 0 || P.tau_f < 0 || P.kappa_w > 32 || P.kappa_f > 32)
        return SGCP_ERR_ARG;
    if (P.p < 0 || P.q < 0 || P.p_obj < 0 || P.q_obj < 0 || P.p + P.q >= ((int64_t)1 << 32) ||
        P.p_obj + P.q_obj >= ((int64_t)1 << 32) || P.zero_attempt_cap < 1)
        return SGCP_ERR_ARG;
    double omega = 1.0;
    for (int k = 0; k < P.ndim; ++k) {
        if (P.dims[k] < 1 || P.dims[k] > 0x7fffffff) return SGCP_ERR_ARG;
        omega *= (double)P.dims[k];
    }
    if (omega > 9.0e18) return SGCP_ERR_UNSUPPORTED;
    for (int k = 0; k < P.ndim; ++k)   // row offsets are 32-bit inside the kernels
        if ((double)P.dims[k] * P.rank >= 2147483648.0) return SGCP_ERR_UNSUPPORTED;
    if (P.sparse_cpl != 0 && P.sparse_cpl != 4 && P.sparse_cpl != 8 && P.sparse_cpl != 16) return SGCP_ERR_ARG;
    if ((P.history_kind != SGCP_HISTORY_MODEL && P.history_kind != SGCP_HISTORY_SLICES) || P.reserved != 0)
        return SGCP_ERR_ARG;
    if (P.history_kind == SGCP_HISTORY_SLICES && P.optimizer != SGCP_OPT_ADAM) return SGCP_ERR_UNSUPPORTED;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return SGCP_ERR_CUDA;   // no usable CUDA device
    }
    sgcp_ctx* c = new (std::nothrow) sgcp_ctx();
    if (!c) return SGCP_ERR_OOM;
    c->P = P;
    c->stored_hist = P.history_kind == SGCP_HISTORY_SLICES && P.H > 0;
    if (allocator) {
        c->ualloc = *allocator;
        c->custom_alloc = true;
    }
    c->ndim = P.ndim;
    c->R = P.rank;
    c->f64 = P.precision == SGCP_PREC_F64;
    c->tc = P.precision == SGCP_PREC_BF16_MTTKRP || P.precision == SGCP_PREC_F16_MTTKRP;
    c->esz = c->f64 ? 8 : 4;
    if (std::isnan(P.lower_bound))
        c->lower = (P.loss == SGCP_LOSS_POISSON || P.loss == SGCP_LOSS_BERNOULLI_ODDS) ? 0.0 : -INFINITY;
    else
        c->lower = P.lower_bound;
    for (int k = 0; k < c->ndim; ++k) {
        c->dims[k] = P.dims[k];
        c->row_off[k] = c->nrows;
        c->nrows += P.dims[k];
    }
    for (int k = c->ndim; k < 4; ++k) c->row_off[k] = c->nrows;
    c->N = c->nrows * c->R;
    c->device = dev;
    c->nhot = P.hot_rows < 0 ? 4 : (P.hot_rows > kMaxHot ? kMaxHot : P.hot_rows);
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return SGCP_ERR_CUDA;
        }
        c->own_stream = true;
    }
    auto bail = [&](sgcp_status st) {
        sgcp_destroy(c);
        return st;
    };
    if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess)
        return bail(SGCP_ERR_CUDA);
    {
        int64_t maxI = 0;
        for (int k = 0; k < c->ndim; ++k) maxI = c->dims[k] > maxI ? c->dims[k] : maxI;
        gram_geometry(maxI, &c->gram_nblk, &c->gram_rpb);
    }
    const size_t nb = (size_t)c->N * c->esz, rb = (size_t)c->R * c->esz;
    void** vecN[] = {&c->A, &c->Abar, &c->G, &c->u, &c->v, &c->u_o, &c->v_o, &c->a_o};
    for (void** p : vecN)
        if (sgcp_status st = dalloc(c, p, nb)) return bail(st);
    void** vecR[] = {&c->s, &c->s_u, &c->s_v, &c->s_uo, &c->s_vo, &c->s_ao, &c->gs};
    for (void** p : vecR)
        if (sgcp_status st = dalloc(c, p, rb)) return bail(st);
    for (void** p : {&c->s2, &c->gs3})
        if (sgcp_status st = dalloc(c, p, 3 * rb)) return bail(st);
    const int Hs = P.H > 0 ? P.H : 1;
    const size_t RR = (size_t)c->R * c->R;
    sgcp_status st = SGCP_OK;
    if ((st = dalloc(c, &c->s_hist, (size_t)Hs * rb)) || (st = dalloc_t(c, &c->h_dev, Hs * sizeof(int64_t))) ||
        (st = dalloc_t(c, &c->hist_len_dev, sizeof(int32_t))) || (st = dalloc_t(c, &c->SH, RR * sizeof(double))) ||
        (st = dalloc_t(c, &c->grams, 6 * c->ndim * RR * sizeof(double))) ||
        (st = dalloc(c, &c->gpart, (size_t)6 * c->ndim * c->gram_nblk * RR * c->esz)) ||
        (st = dalloc(c, &c->Bc, c->ndim * RR * c->esz)) || (st = dalloc(c, &c->Cc, c->ndim * RR * c->esz)) ||
        (c->esz == 4 && c->R <= 32 && P.H > 0 && !c->stored_hist &&
         (st = dalloc_t(c, &c->gacc, 4 * (size_t)c->ndim * RR * sizeof(float)))) ||
        (c->stored_hist &&
         ((st = dalloc_t(c, &c->hist_desc, (size_t)P.H * sizeof(SliceDesc))) ||
          (st = dalloc(c, &c->hist_w, (size_t)P.H * c->esz)) ||
          (st = dalloc_t(c, &c->hist_skip, (size_t)P.H * sizeof(int32_t))) ||
          (st = dalloc_t(c, &c->zero_i, sizeof(int32_t))))) ||
        (st = dalloc_t(c, &c->lsq_work, (RR + c->R) * sizeof(double))) ||
        (st = dalloc_t(c, &c->st_w, sizeof(SolverState))) || (st = dalloc_t(c, &c->st_f, sizeof(SolverState))) ||
        (st = dalloc_t(c, &c->rates_w, (P.tau_w > 0 ? P.tau_w : 1) * sizeof(double))) ||
        (st = dalloc_t(c, &c->rates_f, (P.tau_f > 0 ? P.tau_f : 1) * sizeof(double))) ||
        (st = dalloc_t(c, &c->err, sizeof(int))) || (st = dalloc_t(c, &c->slice_dev, sizeof(SliceDesc))) ||
        (st = dalloc_t(c, &c->metric, 2 * sizeof(double))) ||
        (st = dalloc_t(c, &c->counts, c->nrows * sizeof(int32_t))) ||
        (st = dalloc_t(c, &c->hot, c->nrows * sizeof(int32_t))) ||
        (st = dalloc_t(c, &c->hot_rows, c->ndim * kMaxHot * sizeof(int32_t))) ||
        (c->tc && (st = dalloc(c, &c->xmap, 128))))
        return bail(st);
    if (P.optimizer == SGCP_OPT_LBFGS) {
        // L-BFGS work vectors, m + 1 pair slots and their pointer table, the iteration state
        void* tab[2 * kLbfgsSlots] = {};
        for (int i = 0; i <= P.lbfgs_mem; ++i)
            if ((st = dalloc(c, &tab[i], nb)) || (st = dalloc(c, &tab[kLbfgsSlots + i], nb))) return bail(st);
        if ((st = dalloc(c, &c->lb_x, nb)) || (st = dalloc(c, &c->lb_g, nb)) || (st = dalloc(c, &c->lb_p, nb)) ||
            (st = dalloc_t(c, &c->lb_tab, sizeof(tab))) || (st = dalloc_t(c, &c->lb_state, sizeof(LbfgsState))))
            return bail(st);
        if (cudaStreamCreateWithFlags(&c->lb_stream, cudaStreamNonBlocking) != cudaSuccess) return bail(SGCP_ERR_CUDA);
        if (cudaMemcpyAsync(c->lb_tab, tab, sizeof(tab), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)   // tab dies with this scope
            return bail(SGCP_ERR_CUDA);
    }
    cudaStream_t s = c->stream;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < c->ndim && e == cudaSuccess; ++k) {
        if (!init_factors[k]) return bail(SGCP_ERR_ARG);
        e = cudaMemcpyAsync(offs(c->A, c->row_off[k] * c->R, c->esz), init_factors[k],
                            (size_t)c->dims[k] * c->R * c->esz, cudaMemcpyDeviceToDevice, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->Abar, c->A, nb, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->a_o, c->A, nb, cudaMemcpyDeviceToDevice, s);
    void* zeroN[] = {c->G, c->u, c->v, c->u_o, c->v_o};
    for (void* p : zeroN)
        if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, nb, s);
    void* zeroR[] = {c->s, c->s_u, c->s_v, c->s_uo, c->s_vo, c->s_ao, c->gs};
    for (void* p : zeroR)
        if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, rb, s);
    for (void* p : {c->s2, c->gs3})
        if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, 3 * rb, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->s_hist, 0, (size_t)Hs * rb, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->SH, 0, RR * sizeof(double), s);
    SolverState st0{};
    st0.b1pow = 1.0;   // beta^i at i = 0
    st0.b2pow = 1.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->st_w, &st0, sizeof(SolverState), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->st_f, &st0, sizeof(SolverState), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->err, 0, sizeof(int), s);
    if (e == cudaSuccess && c->gacc) e = cudaMemsetAsync(c->gacc, 0, 4 * (size_t)c->ndim * RR * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->Bc, 0, c->ndim * RR * c->esz, s);
    if (c->stored_hist) {
        if (e == cudaSuccess) e = cudaMemsetAsync(c->hist_desc, 0, (size_t)P.H * sizeof(SliceDesc), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->hist_skip, 0xFF, (size_t)P.H * sizeof(int32_t), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->zero_i, 0, sizeof(int32_t), s);
        c->hs_idx.assign(P.H, nullptr);
        c->hs_vals.assign(P.H, nullptr);
        c->hs_keys.assign(P.H, nullptr);
        c->hs_idx_cap.assign(P.H, 0);
        c->hs_vals_cap.assign(P.H, 0);
        c->hs_keys_cap.assign(P.H, 0);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(c->Cc, 0, c->ndim * RR * c->esz, s);
    std::vector<int64_t> hv(Hs, 0);
    for (int i = 0; i < n_hist; ++i) {
        if (hist_t[i] > t0) return bail(SGCP_ERR_ARG);
        hv[i] = hist_t[i];
        c->hist_t.push_back(hist_t[i]);
    }
    if (e == cudaSuccess && n_hist > 0)
        e = cudaMemcpyAsync(c->s_hist, hist_s, (size_t)n_hist * rb, cudaMemcpyDeviceToDevice, s);
    // host -> device copies of small init data, then wait (the host vectors die here)
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_dev, hv.data(), Hs * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    int32_t nh = n_hist;
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->hist_len_dev, &nh, sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cuda_fail(c, e, "create");
        return bail(e == cudaErrorMemoryAllocation ? SGCP_ERR_OOM : SGCP_ERR_CUDA);
    }
    c->t = t0;
    *out = c;
    return SGCP_OK;
}

void sgcp_destroy(sgcp_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
    for (int i = 0; i < 2; ++i)
        if (c->graph[i]) cudaGraphExecDestroy(c->graph[i]);
    for (void* p : c->allocs) c->custom_alloc ? c->ualloc.free(p, c->ualloc.user) : (void)cudaFree(p);
    c->allocs.clear();
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->lb_stream) cudaStreamDestroy(c->lb_stream);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->ev_staged) cudaEventDestroy(c->ev_staged);
    for (int i = 0; i < 2; ++i)
        if (c->ev_stage_used[i]) cudaEventDestroy(c->ev_stage_used[i]);
    delete c;
}

const char* sgcp_last_error(const sgcp_ctx* c) { return c ? c->last_error.c_str() : "null context"; }

sgcp_status sgcp_ingest(sgcp_ctx* c, const sgcp_slice* X) {
    if (sgcp_status st = check_ready(c)) return st;
    return load_slice(c, X, c->t + 1, true);
}

sgcp_status sgcp_gradient(sgcp_ctx* c, const sgcp_slice* X, const void* s, const void* const* A,
                          const sgcp_grad_opts* opts, void* const* G_out, void* gs_out, double* f_out) {
    if (sgcp_status st = check_ready(c)) return st;
    if (!opts || !s || !A) return fail(c, SGCP_ERR_ARG, "gradient: NULL argument");
    if ((reinterpret_cast<uintptr_t>(s) & 15) != 0)
        return fail(c, SGCP_ERR_ARG, "gradient: s is not 16-byte aligned");   // read as 16-byte vectors
    const int want = opts->want;
    if (want & ~7) return fail(c, SGCP_ERR_ARG, "gradient: bad want bits");
    if ((want & SGCP_WANT_FACTORS) && !G_out) return fail(c, SGCP_ERR_ARG, "gradient: G_out is NULL");
    if ((want & SGCP_WANT_TEMPORAL) && !gs_out) return fail(c, SGCP_ERR_ARG, "gradient: gs_out is NULL");
    if ((want & SGCP_WANT_LOSS) && !f_out) return fail(c, SGCP_ERR_ARG, "gradient: f_out is NULL");
    if (opts->sample_set < 0 || opts->sample_set > 3) return fail(c, SGCP_ERR_ARG, "gradient: bad sample set");
    for (int k = 0; k < c->ndim; ++k) {
        if (!A[k]) return fail(c, SGCP_ERR_ARG, "gradient: A[%d] is NULL", k);
        if ((want & SGCP_WANT_FACTORS) && !G_out[k]) return fail(c, SGCP_ERR_ARG, "gradient: G_out[%d] is NULL", k);
        // factor rows are read and gradient rows accumulated with 16-byte vector accesses
        if ((reinterpret_cast<uintptr_t>(A[k]) & 15) != 0)
            return fail(c, SGCP_ERR_ARG, "gradient: A[%d] is not 16-byte aligned", k);
        if ((want & SGCP_WANT_FACTORS) && (reinterpret_cast<uintptr_t>(G_out[k]) & 15) != 0)
            return fail(c, SGCP_ERR_ARG, "gradient: G_out[%d] is not 16-byte aligned", k);
    }
    if (sgcp_status st = load_slice(c, X, opts->t, false)) return st;
    if (!X->is_sparse)
        if (sgcp_status st = prepare_xmap(c)) return st;
    if (!opts->accumulate) {
        if (want & SGCP_WANT_FACTORS)
            for (int k = 0; k < c->ndim; ++k)
                CK(cudaMemsetAsync(G_out[k], 0, (size_t)c->dims[k] * c->R * c->esz, c->stream), "clear G");
        if (want & SGCP_WANT_TEMPORAL) CK(cudaMemsetAsync(gs_out, 0, (size_t)c->R * c->esz, c->stream), "clear gs");
        if (want & SGCP_WANT_LOSS) CK(cudaMemsetAsync(f_out, 0, sizeof(double), c->stream), "clear f");
    }
    if (want == 0) return SGCP_OK;
    return enqueue_gradient(c, X->is_sparse != 0, nullptr, opts->sample_set, opts->draw, want, s, A, G_out, gs_out,
                            f_out, c->P.loss, opts->y_scale, nullptr);
}

sgcp_status sgcp_sample_coords(sgcp_ctx* c, const sgcp_slice* X, int32_t set, int64_t t, uint32_t draw,
                               int32_t* coords_out, int32_t* attempt_out) {
    if (sgcp_status st = check_ready(c)) return st;
    if (!X || !X->is_sparse || !coords_out || set < 0 || set > 3)
        return fail(c, SGCP_ERR_ARG, "sample_coords: bad argument");
    if (sgcp_status st = load_slice(c, X, t, false)) return st;
    const void* Adummy[4] = {c->A, c->A, c->A, c->A};
    SparseGradArgs a = sparse_args(c, nullptr, set, draw, 0, c->s, Adummy, nullptr, nullptr, nullptr, c->P.loss,
                                   nullptr, nullptr);
    a.coords_out = coords_out;
    a.attempt_out = attempt_out;
    const bool obj = (set == SGCP_SAMPLES_FACTOR_OBJ || set == SGCP_SAMPLES_TEMPORAL_OBJ);
    const int64_t total = obj ? c->P.p_obj + c->P.q_obj : c->P.p + c->P.q;
    CK(launch_sample_coords(a, total, c->stream, &c->launches), "sample coords");
    return SGCP_OK;
}

sgcp_status sgcp_step(sgcp_ctx* c, const sgcp_slice* X) {
    if (sgcp_status st = check_ready(c)) return st;
    if (!X) return fail(c, SGCP_ERR_ARG, "step: slice is NULL");
    const int64_t t = c->t + 1;
    const bool sparse = X->is_sparse != 0;
    if (sparse && (c->P.p + c->P.q == 0 || c->P.p_obj + c->P.q_obj == 0) && c->P.temporal != SGCP_TEMPORAL_LSQ)
        return fail(c, SGCP_ERR_ARG, "step: sparse slices need p + q > 0 and p_obj + q_obj > 0");
    if (sparse && c->P.optimizer == SGCP_OPT_LBFGS)
        return fail(c, SGCP_ERR_UNSUPPORTED, "step: the L-BFGS factor solver needs dense slices");
    if (c->stored_hist && c->hist_sparse >= 0 && c->hist_sparse != (sparse ? 1 : 0))
        return fail(c, SGCP_ERR_ARG, "step: a stored-slice history holds slices of one kind (all dense or all sparse)");
    if (sgcp_status st = load_slice(c, X, t, false)) return st;
    CK(launch_write_desc(c->slice_dev, c->cur, c->stream, &c->launches), "slice descriptor");
    if (!sparse)
        if (sgcp_status st = prepare_xmap(c)) return st;
    const int gi = sparse ? 1 : 0;
    if (!c->graph[gi])
        if (sgcp_status st = build_graph(c, sparse)) return st;
    CK(cudaGraphLaunch(c->graph[gi], c->stream), "graph launch");
    c->launches += c->graph_kernels[gi];
    // reservoir update of the history window (Alg. 1), decided on the host from t alone
    if (c->P.H > 0) {
        int slot = -1;
        int len = (int)c->hist_t.size();
        if (len < c->P.H) {
            slot = len;
            c->hist_t.push_back(t);
            len += 1;
        } else {
            const uint32_t j = reservoir_index(c->P.seed, t);
            if ((int64_t)j <= c->P.H) {
                slot = (int)j - 1;
                c->hist_t[slot] = t;
            }
        }
        if (slot >= 0) {
            cudaError_t e = c->f64 ? launch_hist_update<double>(c->R, (double*)c->s_hist, c->h_dev, c->hist_len_dev,
                                                                 slot, t, len, (const double*)c->s, c->stream,
                                                                 &c->launches)
                                   : launch_hist_update<float>(c->R, (float*)c->s_hist, c->h_dev, c->hist_len_dev,
                                                               slot, t, len, (const float*)c->s, c->stream,
                                                               &c->launches);
            if (e != cudaSuccess) return cuda_fail(c, e, "history update");
            if (c->stored_hist)
                if (sgcp_status st = store_slice(c, slot, sparse, c->cur, t)) return st;
        }
    }
    c->t = t;
    return SGCP_OK;
}

sgcp_status sgcp_warm_start(sgcp_ctx* c, int32_t n, const sgcp_slice* X, const void* S_init, void* S_out,
                            sgcp_warm_stats* stats_out) {
    if (sgcp_status st = check_ready(c)) return st;
    if (n < 1 || !X) return fail(c, SGCP_ERR_ARG, "warm start: need n >= 1 slices");
    if (c->t != 0 || !c->hist_t.empty())
        return fail(c, SGCP_ERR_ARG, "warm start: the context has processed slices or holds a history window");
    const bool sparse = X[0].is_sparse != 0;
    for (int h = 0; h < n; ++h) {
        const sgcp_slice& x = X[h];
        if ((x.is_sparse != 0) != sparse) return fail(c, SGCP_ERR_ARG, "warm start: mixed sparse and dense slices");
        if (sparse) {
            if (c->f64) return fail(c, SGCP_ERR_UNSUPPORTED, "warm start: sparse slices need a float context");
            if (x.nnz < 0 || x.nnz > omega_of(c) || x.nnz >= (int64_t)1 << 31)
                return fail(c, SGCP_ERR_ARG, "warm start: slice %d nnz out of range", h);
            if (x.nnz > 0 && (!x.idx || !x.vals)) return fail(c, SGCP_ERR_ARG, "warm start: slice %d without data", h);
        } else {
            if (!x.vals) return fail(c, SGCP_ERR_ARG, "warm start: dense slice %d without vals", h);
            if (c->ndim > 3) return fail(c, SGCP_ERR_UNSUPPORTED, "warm start: dense slices support ndim <= 3");
        }
    }
    if (sparse && (c->P.p + c->P.q == 0 || c->P.p_obj + c->P.q_obj == 0))
        return fail(c, SGCP_ERR_ARG, "warm start: sparse slices need p + q > 0 and p_obj + q_obj > 0");
    return c->f64 ? warm_start_impl<double>(c, n, X, S_init, S_out, stats_out)
                  : warm_start_impl<float>(c, n, X, S_init, S_out, stats_out);
}

sgcp_status sgcp_slice_loss(sgcp_ctx* c, const sgcp_slice* X, const void* s, const void* const* A, int32_t exact,
                            int64_t t, double* out) {
    if (sgcp_status st = check_ready(c)) return st;
    if (!X || !s || !A || !out) return fail(c, SGCP_ERR_ARG, "slice_loss: NULL argument");
    if ((reinterpret_cast<uintptr_t>(s) & 15) != 0) return fail(c, SGCP_ERR_ARG, "slice_loss: s is not 16-byte aligned");
    for (int k = 0; k < c->ndim; ++k)
        if (!A[k] || (reinterpret_cast<uintptr_t>(A[k]) & 15) != 0)
            return fail(c, SGCP_ERR_ARG, "slice_loss: A[%d] is NULL or not 16-byte aligned", k);
    const bool sparse = X->is_sparse != 0;
    if (sparse && exact && c->ndim > 3)
        return fail(c, SGCP_ERR_UNSUPPORTED, "slice_loss: the exact loss of a sparse slice needs ndim <= 3");
    if (sparse && !exact && c->P.p_obj + c->P.q_obj == 0)
        return fail(c, SGCP_ERR_ARG, "slice_loss: the sampled loss needs p_obj + q_obj > 0");
    if (sgcp_status st = load_slice(c, X, t, false)) return st;
    if (!sparse)
        if (sgcp_status st = prepare_xmap(c)) return st;
    CK(cudaMemsetAsync(c->metric, 0, 2 * sizeof(double), c->stream), "clear loss");
    if (sparse)
        CK(launch_sum_squares<float>((const float*)c->cur.vals, c->cur.nnz, c->metric + 1, c->stream, &c->launches),
           "norm");
    else if (c->f64)
        CK(launch_sum_squares<double>((const double*)c->cur.vals, c->cur.nnz, c->metric + 1, c->stream, &c->launches),
           "norm");
    else
        CK(launch_sum_squares<float>((const float*)c->cur.vals, c->cur.nnz, c->metric + 1, c->stream, &c->launches),
           "norm");
    if (!sparse || !exact) {
        // dense: the exact sum over every entry; sparse: the objective sample set at time index t
        sgcp_status st = enqueue_gradient(c, sparse, nullptr, SGCP_SAMPLES_FACTOR_OBJ, 0, SGCP_WANT_LOSS, s, A, nullptr,
                                          nullptr, c->metric, c->P.loss, nullptr, nullptr);
        if (st) return st;
    } else {
        // every entry of a sparse slice: sum_i f(0, m_i) over the whole index space (the dense loss
        // kernel on the all-zero slice), plus f(x, m) - f(0, m) over the nonzeros
        DenseGradArgs<float> z = dense_args<float>(c, nullptr, SGCP_WANT_LOSS, s, A, nullptr, nullptr, c->metric,
                                                   c->P.loss, nullptr, nullptr);
        z.inline_slice.vals = nullptr;
        z.inline_slice.nnz = omega_of(c);
        z.xmap = nullptr;
        CK(launch_dense_grad<float>(z, c->stream, &c->launches), "model loss");
        SparseGradArgs a = sparse_args(c, nullptr, SGCP_SAMPLES_FACTOR_OBJ, 0, SGCP_WANT_LOSS, s, A, nullptr, nullptr,
                                       c->metric, c->P.loss, nullptr, nullptr);
        a.all_nnz = 1;
        a.f_minus_zero = 1;
        CK(launch_sparse_grad(a, (int64_t)1 << 40, c->stream, &c->launches), "nonzero loss");
    }
    CK(cudaMemcpyAsync(out, c->metric, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "read loss");
    CK(cudaStreamSynchronize(c->stream), "slice loss");
    return SGCP_OK;
}

sgcp_status sgcp_kruskal_score(int32_t nmodes, int32_t rank, const int64_t* dims, int32_t precision,
                               const void* const* A, const void* const* B, double* score_out, int32_t* perm_out,
                               void* cuda_stream) {
    if (nmodes < 1 || nmodes > 8 || rank < 1 || rank > 128 || !dims || !A || !B || !score_out) return SGCP_ERR_ARG;
    if (precision != SGCP_PREC_F32 && precision != SGCP_PREC_F64) return SGCP_ERR_ARG;
    for (int k = 0; k < nmodes; ++k)
        if (dims[k] < 1 || !A[k] || !B[k]) return SGCP_ERR_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t RR = (size_t)rank * rank;
    const size_t bytes = (nmodes * RR + 2 * (size_t)nmodes * rank + 1) * sizeof(double) + rank * sizeof(int32_t);
    void* scratch = nullptr;
    if (cudaMallocAsync(&scratch, bytes, st) != cudaSuccess) {
        cudaGetLastError();
        return SGCP_ERR_OOM;
    }
    double* C = (double*)scratch;
    double* na = C + nmodes * RR;
    double* nb = na + (size_t)nmodes * rank;
    double* sc = nb + (size_t)nmodes * rank;
    int32_t* pm = (int32_t*)(sc + 1);
    cudaError_t e = precision == SGCP_PREC_F64
                        ? launch_congruence<double>(nmodes, rank, dims, (const double* const*)A,
                                                    (const double* const*)B, C, na, nb, sc, pm, st)
                        : launch_congruence<float>(nmodes, rank, dims, (const float* const*)A, (const float* const*)B,
                                                   C, na, nb, sc, pm, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(score_out, sc, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && perm_out)
        e = cudaMemcpyAsync(perm_out, pm, rank * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(scratch, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SGCP_ERR_CUDA;
    }
    return SGCP_OK;
}

sgcp_status sgcp_factors(sgcp_ctx* c, void* const* A_out, void* s_out, int64_t* t_out) {
    if (!c) return SGCP_ERR_ARG;
    if (A_out)
        for (int k = 0; k < c->ndim; ++k) {
            if (!A_out[k]) continue;
            CK(cudaMemcpyAsync(A_out[k], offs(c->A, c->row_off[k] * c->R, c->esz), (size_t)c->dims[k] * c->R * c->esz,
                               cudaMemcpyDeviceToDevice, c->stream),
               "copy factors");
        }
    if (s_out) CK(cudaMemcpyAsync(s_out, c->s, (size_t)c->R * c->esz, cudaMemcpyDeviceToDevice, c->stream), "copy s");
    if (t_out) *t_out = c->t;
    return SGCP_OK;
}

sgcp_status sgcp_history(sgcp_ctx* c, int64_t* h_out, void* s_out, int32_t* n_out) {
    if (!c) return SGCP_ERR_ARG;
    const int n = (int)c->hist_t.size();
    if (n_out) *n_out = n;
    if (h_out)
        for (int i = 0; i < n; ++i) h_out[i] = c->hist_t[i];
    if (s_out && n)
        CK(cudaMemcpyAsync(s_out, c->s_hist, (size_t)n * c->R * c->esz, cudaMemcpyDeviceToDevice, c->stream),
           "copy history");
    return SGCP_OK;
}

sgcp_status sgcp_check(sgcp_ctx* c) {
    if (!c) return SGCP_ERR_ARG;
    if (c->sticky != SGCP_OK) return SGCP_ERR_STATE;
    cudaSetDevice(c->device);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "synchronize");
    int bits = 0;
    e = cudaMemcpy(&bits, c->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "read error word");
    if (bits) {
        c->sticky = status_from_err(bits);
        char buf[128];
        snprintf(buf, sizeof(buf), "device error bits 0x%x", bits);
        c->last_error = buf;
        return c->sticky;
    }
    return SGCP_OK;
}

sgcp_status sgcp_stats(sgcp_ctx* c, sgcp_stats_t* out) {
    if (!c || !out) return SGCP_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
    sgcp_status st = sgcp_check(c);
    SolverState w{}, f{};
    int bits = 0;
    cudaMemcpy(&w, c->st_w, sizeof(w), cudaMemcpyDeviceToHost);
    cudaMemcpy(&f, c->st_f, sizeof(f), cudaMemcpyDeviceToHost);
    cudaMemcpy(&bits, c->err, sizeof(int), cudaMemcpyDeviceToHost);
    out->t = c->t;
    out->iter = f.i;
    out->F_w = w.F_cur;
    out->F_f = f.F_cur;
    out->epochs_w = w.epoch;
    out->epochs_f = f.epoch;
    out->accept_w = w.accept;
    out->accept_f = f.accept;
    out->alpha_w = w.alpha;
    out->alpha_f = f.alpha;
    out->hist_len = (int32_t)c->hist_t.size();
    out->error_bits = bits;
    out->kernels_launched = c->launches;
    out->evals_f = c->P.optimizer == SGCP_OPT_LBFGS ? f.evals : 0;
    return st;
}

sgcp_status sgcp_objectives_async(sgcp_ctx* c, double* out) {
    if (!c || !out) return SGCP_ERR_ARG;
    if (sgcp_status st = check_ready(c)) return st;
    const size_t off = offsetof(SolverState, F_cur);
    cudaError_t e = cudaMemcpyAsync(out, reinterpret_cast<const char*>(c->st_w) + off, sizeof(double),
                                    cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out + 1, reinterpret_cast<const char*>(c->st_f) + off, sizeof(double),
                            cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "objective read-back");
    return SGCP_OK;
}

// Checkpoint layout: header, then Abar, s, history weights, u, v (element type T).
struct CkptHeader {
    uint64_t magic;
    int32_t ndim, R, H, hist_len, esz, pad;
    int64_t dims[4];
    int64_t t;
    int64_t iter;
    int64_t hist_t[1];   // followed by H - 1 more
};

static size_t ckpt_size(const sgcp_ctx* c) {
    const int Hs = c->P.H > 0 ? c->P.H : 1;
    return sizeof(CkptHeader) + (size_t)(Hs - 1) * sizeof(int64_t) +
           ((size_t)3 * c->N + c->R + (size_t)Hs * c->R) * c->esz;
}

sgcp_status sgcp_state_size(const sgcp_ctx* c, size_t* size) {
    if (!c || !size) return SGCP_ERR_ARG;
    if (c->stored_hist) return SGCP_ERR_UNSUPPORTED;   // the stored slices are not part of a checkpoint
    *size = ckpt_size(c);
    return SGCP_OK;
}

sgcp_status sgcp_state_export(sgcp_ctx* c, void* buf, size_t size) {
    if (!c || !buf) return SGCP_ERR_ARG;
    if (c->stored_hist) return fail(c, SGCP_ERR_UNSUPPORTED, "state_export: a stored-slice history is not checkpointed");
    if (size < ckpt_size(c)) return fail(c, SGCP_ERR_ARG, "state_export: buffer too small");
    if (sgcp_status st = sgcp_check(c)) return st;
    const int Hs = c->P.H > 0 ? c->P.H : 1;
    CkptHeader* h = (CkptHeader*)buf;
    h->magic = 0x5347435053544154ull;
    h->ndim = c->ndim;
    h->R = c->R;
    h->H = c->P.H;
    h->hist_len = (int32_t)c->hist_t.size();
    h->esz = (int32_t)c->esz;
    h->pad = 0;
    for (int k = 0; k < 4; ++k) h->dims[k] = c->dims[k];
    h->t = c->t;
    SolverState f{};
    CK(cudaMemcpy(&f, c->st_f, sizeof(f), cudaMemcpyDeviceToHost), "read state");
    h->iter = f.i;
    for (int i = 0; i < Hs; ++i) h->hist_t[i] = i < (int)c->hist_t.size() ? c->hist_t[i] : 0;
    char* p = (char*)buf + sizeof(CkptHeader) + (size_t)(Hs - 1) * sizeof(int64_t);
    const size_t nb = (size_t)c->N * c->esz;
    CK(cudaMemcpy(p, c->Abar, nb, cudaMemcpyDeviceToHost), "export");
    p += nb;
    CK(cudaMemcpy(p, c->s, (size_t)c->R * c->esz, cudaMemcpyDeviceToHost), "export");
    p += (size_t)c->R * c->esz;
    CK(cudaMemcpy(p, c->s_hist, (size_t)Hs * c->R * c->esz, cudaMemcpyDeviceToHost), "export");
    p += (size_t)Hs * c->R * c->esz;
    CK(cudaMemcpy(p, c->u, nb, cudaMemcpyDeviceToHost), "export");
    p += nb;
    CK(cudaMemcpy(p, c->v, nb, cudaMemcpyDeviceToHost), "export");
    return SGCP_OK;
}

sgcp_status sgcp_state_import(sgcp_ctx* c, const void* buf, size_t size) {
    if (!c || !buf) return SGCP_ERR_ARG;
    if (c->stored_hist) return fail(c, SGCP_ERR_UNSUPPORTED, "state_import: a stored-slice history is not checkpointed");
    if (sgcp_status st = check_ready(c)) return st;
    if (size < ckpt_size(c)) return fail(c, SGCP_ERR_ARG, "state_import: buffer too small");
    const CkptHeader* h = (const CkptHeader*)buf;
    if (h->magic != 0x5347435053544154ull || h->ndim != c->ndim || h->R != c->R || h->H != c->P.H ||
        h->esz != (int32_t)c->esz)
        return fail(c, SGCP_ERR_ARG, "state_import: checkpoint does not match this context");
    for (int k = 0; k < c->ndim; ++k)
        if (h->dims[k] != c->dims[k]) return fail(c, SGCP_ERR_ARG, "state_import: dims differ");
    const int Hs = c->P.H > 0 ? c->P.H : 1;
    CK(cudaStreamSynchronize(c->stream), "sync");
    const char* p = (const char*)buf + sizeof(CkptHeader) + (size_t)(Hs - 1) * sizeof(int64_t);
    const size_t nb = (size_t)c->N * c->esz;
    CK(cudaMemcpy(c->Abar, p, nb, cudaMemcpyHostToDevice), "import");
    CK(cudaMemcpy(c->A, p, nb, cudaMemcpyHostToDevice), "import");
    CK(cudaMemcpy(c->a_o, p, nb, cudaMemcpyHostToDevice), "import");
    p += nb;
    CK(cudaMemcpy(c->s, p, (size_t)c->R * c->esz, cudaMemcpyHostToDevice), "import");
    p += (size_t)c->R * c->esz;
    CK(cudaMemcpy(c->s_hist, p, (size_t)Hs * c->R * c->esz, cudaMemcpyHostToDevice), "import");
    p += (size_t)Hs * c->R * c->esz;
    CK(cudaMemcpy(c->u, p, nb, cudaMemcpyHostToDevice), "import");
    CK(cudaMemcpy(c->u_o, p, nb, cudaMemcpyHostToDevice), "import");
    p += nb;
    CK(cudaMemcpy(c->v, p, nb, cudaMemcpyHostToDevice), "import");
    CK(cudaMemcpy(c->v_o, p, nb, cudaMemcpyHostToDevice), "import");
    c->hist_t.clear();
    std::vector<int64_t> hv(Hs, 0);
    for (int i = 0; i < h->hist_len; ++i) {
        c->hist_t.push_back(h->hist_t[i]);
        hv[i] = h->hist_t[i];
    }
    CK(cudaMemcpy(c->h_dev, hv.data(), Hs * sizeof(int64_t), cudaMemcpyHostToDevice), "import");
    int32_t nh = h->hist_len;
    CK(cudaMemcpy(c->hist_len_dev, &nh, sizeof(int32_t), cudaMemcpyHostToDevice), "import");
    SolverState f{};
    CK(cudaMemcpy(&f, c->st_f, sizeof(f), cudaMemcpyDeviceToHost), "import");
    f.i = (int32_t)h->iter;
    f.b1pow = std::pow(c->P.beta1, (double)f.i);
    f.b2pow = std::pow(c->P.beta2, (double)f.i);
    CK(cudaMemcpy(c->st_f, &f, sizeof(f), cudaMemcpyHostToDevice), "import");
    CK(cudaMemset(c->G, 0, nb), "import");
    c->t = h->t;
    c->loaded = false;
    return SGCP_OK;
}

}  // extern "C"
