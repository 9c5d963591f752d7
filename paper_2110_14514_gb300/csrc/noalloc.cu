// Stochastic sparse GCP gradient that allocates no device memory.
//
// Some callers cannot let a library allocate: a serving process that reserves
// its whole GPU memory budget at start-up and hands out nothing afterwards,
// or a latency-critical loop in which a cudaMalloc (which may synchronise the
// device) is not acceptable.  For them this file provides one entry point that
// computes the same fused sample -> model -> loss-derivative -> MTTKRP
// gradient as sgcp_gradient does for a sparse slice, but keeps its only
// scratch structure -- the nonzero-membership hash table used to reject zero
// samples -- in a fixed file-scope device array instead of memory owned by a
// context.  The caller passes every input and output.
//
// The array is 2^19 slots of 8 bytes (4 MiB).  Every GPU that loads the
// library holds it until the process exits.  The table is kept at most half
// full, so the entry point accepts at most 262144 nonzeros per slice and
// answers SGCP_ERR_UNSUPPORTED above that.  All calls share the one array and
// it keeps the previous call's keys, so each call clears the part it uses;
// two calls whose work overlaps on the GPU (different streams, or different
// host threads) race on it and must be serialised by the caller.
#include <mutex>

#include "internal.h"
#include "sgcp.h"

using namespace sgcp;

namespace {

constexpr int kNoAllocLog2 = 19;
constexpr int64_t kNoAllocSlots = (int64_t)1 << kNoAllocLog2;
constexpr int64_t kNoAllocMaxNnz = kNoAllocSlots / 2;
constexpr int kMaxDevices = 64;

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {nullptr};

}  // namespace

// The scratch table itself.  In host code this name only stands for the
// symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned long long g_noalloc_hash[kNoAllocSlots];

namespace {

// Per-device set-up, done by the first call on each device with that device
// current: look up the device address of the scratch table.
sgcp_status scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return SGCP_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return SGCP_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_hash);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return SGCP_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return SGCP_OK;
}

uint32_t nz_purpose(int set) {
    switch (set) {
        case SGCP_SAMPLES_FACTOR_GRAD: return PUR_GRAD_NZ;
        case SGCP_SAMPLES_FACTOR_OBJ: return PUR_OBJ_NZ;
        case SGCP_SAMPLES_TEMPORAL_GRAD: return PUR_TGRAD_NZ;
        default: return PUR_TOBJ_NZ;
    }
}

}  // namespace

extern "C" sgcp_status sgcp_gradient_sparse_noalloc(const sgcp_params* params, int64_t nnz, const int32_t* idx,
                                                    const float* vals, const float* s, const float* const* A,
                                                    const sgcp_grad_opts* opts, float* const* G_out, float* gs_out,
                                                    double* f_out, int32_t* err_out, void* cuda_stream) {
    if (!params || !opts || !s || !A) return SGCP_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(s) & 15) != 0) return SGCP_ERR_ARG;   // read as 16-byte vectors
    const sgcp_params& P = *params;
    if (P.ndim < 2 || P.ndim > 4 || P.rank < 4 || P.rank > 128 || P.rank % 4 != 0) return SGCP_ERR_UNSUPPORTED;
    if (P.loss < 0 || P.loss > 3 || P.zero_attempt_cap < 1) return SGCP_ERR_ARG;
    if (P.precision == SGCP_PREC_F64) return SGCP_ERR_UNSUPPORTED;
    if (P.sparse_cpl != 0 && P.sparse_cpl != 4 && P.sparse_cpl != 8 && P.sparse_cpl != 16) return SGCP_ERR_ARG;
    const int want = opts->want;
    if ((want & ~7) || opts->sample_set < 0 || opts->sample_set > 3) return SGCP_ERR_ARG;
    if ((want & SGCP_WANT_FACTORS) && !G_out) return SGCP_ERR_ARG;
    if ((want & SGCP_WANT_TEMPORAL) && !gs_out) return SGCP_ERR_ARG;
    if ((want & SGCP_WANT_LOSS) && !f_out) return SGCP_ERR_ARG;
    double omega = 1.0;
    for (int k = 0; k < P.ndim; ++k) {
        if (P.dims[k] < 1 || P.dims[k] > 0x7fffffff) return SGCP_ERR_ARG;
        if ((double)P.dims[k] * P.rank >= 2147483648.0) return SGCP_ERR_UNSUPPORTED;
        if (!A[k] || ((want & SGCP_WANT_FACTORS) && !G_out[k])) return SGCP_ERR_ARG;
        if ((reinterpret_cast<uintptr_t>(A[k]) & 15) != 0 ||
            ((want & SGCP_WANT_FACTORS) && (reinterpret_cast<uintptr_t>(G_out[k]) & 15) != 0))
            return SGCP_ERR_ARG;
        omega *= (double)P.dims[k];
    }
    if (omega > 9.0e18) return SGCP_ERR_UNSUPPORTED;
    if (nnz < 0 || (double)nnz > omega) return SGCP_ERR_ARG;
    if (nnz > kNoAllocMaxNnz) return SGCP_ERR_UNSUPPORTED;   // beyond the fixed scratch table
    if (nnz > 0 && (!idx || !vals)) return SGCP_ERR_ARG;
    const bool obj = (opts->sample_set == SGCP_SAMPLES_FACTOR_OBJ || opts->sample_set == SGCP_SAMPLES_TEMPORAL_OBJ);
    const int64_t p = obj ? P.p_obj : P.p, q = obj ? P.q_obj : P.q;
    if (p < 0 || q < 0 || p + q >= ((int64_t)1 << 32)) return SGCP_ERR_ARG;

    void* table = nullptr;
    if (sgcp_status st = scratch_address(&table)) return st;
    unsigned long long* keys = (unsigned long long*)table;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    int hl = 10;
    while (((int64_t)1 << hl) < 2 * nnz) ++hl;   // hl <= kNoAllocLog2 by the nnz limit

    // outputs are overwritten unless opts->accumulate; the used part of the table starts empty (all ones)
    cudaError_t e = cudaSuccess;
    const bool clear = opts->accumulate == 0;
    if (err_out) e = cudaMemsetAsync(err_out, 0, sizeof(int32_t), stream);
    if (e == cudaSuccess && clear && (want & SGCP_WANT_FACTORS))
        for (int k = 0; k < P.ndim && e == cudaSuccess; ++k)
            e = cudaMemsetAsync(G_out[k], 0, (size_t)P.dims[k] * P.rank * sizeof(float), stream);
    if (e == cudaSuccess && clear && (want & SGCP_WANT_TEMPORAL))
        e = cudaMemsetAsync(gs_out, 0, (size_t)P.rank * sizeof(float), stream);
    if (e == cudaSuccess && clear && (want & SGCP_WANT_LOSS)) e = cudaMemsetAsync(f_out, 0, sizeof(double), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(keys, 0xFF, ((size_t)1 << hl) * sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return SGCP_ERR_CUDA;
    if (want == 0) return SGCP_OK;

    SliceDesc sd{};
    sd.idx = idx;
    sd.vals = vals;
    sd.nnz = nnz;
    sd.t = opts->t;
    if (nnz > 0 && launch_hash_build(sd, P.ndim, P.dims, keys, hl, err_out, stream) != cudaSuccess)
        return SGCP_ERR_CUDA;

    SparseGradArgs a{};
    a.slice = nullptr;
    a.inline_slice = sd;
    a.ndim = P.ndim;
    a.R = P.rank;
    for (int k = 0; k < 4; ++k) a.dims[k] = k < P.ndim ? P.dims[k] : 1;
    for (int k = 0; k < P.ndim; ++k) {
        a.A[k] = A[k];
        a.G[k] = (want & SGCP_WANT_FACTORS) ? G_out[k] : nullptr;
        a.hot[k] = nullptr;
    }
    a.s = s;
    a.gs = gs_out;
    a.f = f_out;
    a.hkeys = keys;
    a.hlog2 = hl;
    a.hot_rows = nullptr;
    a.nhot = 0;                 // no hot-row tables: they would be more scratch
    a.key0 = (uint32_t)(P.seed & 0xFFFFFFFFu);
    a.key1 = (uint32_t)(P.seed >> 32);
    a.draw = opts->draw;
    a.pur_nz = nz_purpose(opts->sample_set);
    a.pur_z = a.pur_nz + 1;
    a.p = p;
    a.q = q;
    a.all_nnz = 0;
    a.cap = P.zero_attempt_cap;
    a.want = want;
    a.loss = P.loss;
    a.eps = (float)P.log_eps;
    a.y_scale = (const float*)opts->y_scale;
    a.err = err_out;
    a.skip = nullptr;
    a.cpl = P.sparse_cpl;
    if (launch_sparse_grad(a, p + q, stream, nullptr) != cudaSuccess) return SGCP_ERR_CUDA;
    return SGCP_OK;
}
