// Shared device helpers of the streaming-GCP library: Philox4x32-10, bounded
// integers, GCP losses, error bits and the device-resident step descriptor.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#define SGCP_FULL_MASK 0xffffffffu

namespace sgcp {

// ---------------------------------------------------------------------------
// Device error word bits (latched with atomicOr, read by sgcp_check).
// ---------------------------------------------------------------------------
enum ErrBits : int {
    ERRB_COORD = 1,      // a COO coordinate outside [0, I_k)
    ERRB_DUP = 2,        // a COO coordinate repeated
    ERRB_SAMPLING = 4,   // a zero-sample slot exhausted its attempts
    ERRB_NUMERIC = 8,    // non-finite objective
    ERRB_HASH = 16,      // nonzero hash table full (cannot happen at load <= 1/2)
    ERRB_SOLVE = 32,     // least-squares normal matrix not positive definite
    ERRB_TIMEOUT = 64    // a bounded wait inside a kernel gave up
};

// Purposes of the Philox counter (high byte of counter word 3).
enum Purpose : uint32_t {
    PUR_GRAD_NZ = 0, PUR_GRAD_Z = 1, PUR_OBJ_NZ = 2, PUR_OBJ_Z = 3, PUR_RESERVOIR = 4,
    PUR_TGRAD_NZ = 5, PUR_TGRAD_Z = 6, PUR_TOBJ_NZ = 7, PUR_TOBJ_Z = 8,
    PUR_HGRAD_NZ = 9, PUR_HGRAD_Z = 10, PUR_HOBJ_NZ = 11, PUR_HOBJ_Z = 12   // stored history slices
};

// Loss ids; LOSS_IDENTITY_X is internal: y = x, f = 0 (gives Z' vec(X) for the
// least-squares temporal solve).
enum LossId : int { LOSS_GAUSSIAN = 0, LOSS_POISSON = 1, LOSS_ODDS = 2, LOSS_LOGIT = 3, LOSS_IDENTITY_X = 4 };

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 3.3): 10 rounds of
//   (c0, c1, c2, c3) <- (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
// with the key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
__host__ __device__ inline void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
#ifdef __CUDA_ARCH__
        const uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
        const uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
#else
        const uint64_t p0 = (uint64_t)M0 * c[0], p1 = (uint64_t)M1 * c[2];
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

// Multiply-shift bounded integer: floor(u * n / 2^32), n <= 2^32 - 1.
__host__ __device__ inline uint32_t bounded_u32(uint32_t u, uint32_t n) {
#ifdef __CUDA_ARCH__
    return __umulhi(u, n);
#else
    return (uint32_t)(((uint64_t)u * n) >> 32);
#endif
}

__host__ __device__ inline uint32_t counter_word3(uint32_t purpose, int64_t t) {
    return (purpose << 24) | ((uint32_t)t & 0xFFFFFFu);
}

// ---------------------------------------------------------------------------
// GCP losses (Sec. 2.2): f(x, m) and y = df/dm.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void loss_eval(int loss, T x, T m, T eps, T& f, T& y) {
    switch (loss) {
        case LOSS_GAUSSIAN: {
            const T d = m - x;
            f = d * d;
            y = T(2) * d;
            break;
        }
        case LOSS_POISSON: {
            const T me = m + eps;
            f = m - x * log(me);
            y = T(1) - x / me;
            break;
        }
        case LOSS_ODDS: {
            const T me = m + eps;
            f = log(m + T(1)) - x * log(me);
            y = T(1) / (m + T(1)) - x / me;
            break;
        }
        case LOSS_LOGIT: {
            f = (m > T(0) ? m : T(0)) + log1p(exp(-fabs(m))) - x * m;
            y = T(1) / (T(1) + exp(-m)) - x;
            break;
        }
        default: {  // LOSS_IDENTITY_X
            f = T(0);
            y = x;
            break;
        }
    }
}

// y = df/dm alone (no loss value): the gradient kernels call this when the
// loss is not requested, so the log / log1p of f are never evaluated.
template <typename T>
__device__ __forceinline__ T loss_dfdm(int loss, T x, T m, T eps) {
    switch (loss) {
        case LOSS_GAUSSIAN: return T(2) * (m - x);
        case LOSS_POISSON: return T(1) - x / (m + eps);
        case LOSS_ODDS: return T(1) / (m + T(1)) - x / (m + eps);
        case LOSS_LOGIT: return T(1) / (T(1) + exp(-m)) - x;
        default: return x;
    }
}

// ---------------------------------------------------------------------------
// Device-resident description of the slice currently loaded; kernels captured
// in a CUDA graph read it so that one graph serves every slice.
// ---------------------------------------------------------------------------
struct SliceDesc {
    const int32_t* idx;   // sparse: [nnz][ndim]
    const void* vals;     // sparse: [nnz]; dense: full slice, C order
    int64_t nnz;          // sparse: number of nonzeros; dense: prod I_k
    int64_t t;            // time index of the slice (the sample counter's t-field)
    // A slice kept in the history window (stored-slice history) carries its own nonzero hash and
    // a draw base added to every sample draw index; both are null / 0 for the current slice.
    const unsigned long long* hkeys;
    int32_t hlog2;
    uint32_t draw_base;
};

// Device-resident scalars of one solver (Alg. 2-4).
struct SolverState {
    double F_cur;      // current accepted estimate
    double F_old;      // estimate at the start of the epoch
    double F_new;      // accumulator of the estimate after the epoch
    double alpha;      // learning rate
    int32_t i;         // iteration counter for the bias correction
    int32_t epoch;     // epochs run
    int32_t done;      // set once the estimate is <= tol (Alg. 3/4 loop test)
    uint32_t accept;   // bit e = epoch e accepted
    uint32_t ticket;   // last-block counter (epoch end, fused temporal step)
    int32_t evals;     // objective evaluations of the last L-BFGS factor solve (0 for ADAM)
    double b1pow;      // beta1^i, i = iterations accepted before the current epoch
    double b2pow;      // beta2^i
};

// ADAM bias-corrected learning rate of iteration i + j, i.e. the j-th
// iteration of the current epoch (Alg. 2 with exponent i + j + 1):
// alpha sqrt(1 - beta2^(i+j+1)) / (1 - beta1^(i+j+1)).  k_epoch_begin
// evaluates it once per epoch for every j; the per-iteration kernels read it.
__host__ __device__ inline double adam_rate(const SolverState& s, double beta1, double beta2, int j) {
    return s.alpha * sqrt(1.0 - s.b2pow * pow(beta2, (double)(j + 1))) / (1.0 - s.b1pow * pow(beta1, (double)(j + 1)));
}

// Parameters of the temporal-weight ADAM step fused into the last block of a
// temporal-gradient kernel (Alg. 3: g = Z'y + mu s; Alg. 2 Step).
template <typename T>
struct TemporalStep {
    T* s;
    T* u;
    T* v;
    SolverState* st;      // ticket only
    const double* rate;   // bias-corrected learning rate of this iteration
    double mu, beta1, beta2, eps, lower;
};

// Last-block election: every block fences its global writes and takes a
// ticket; the block that takes the last one sees all of them.
// Two FP32 fused multiply-adds in one instruction (fma.rn.f32x2, Blackwell): each half is
// rounded exactly as fmaf would round it.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n.reg .b64 ra, rb, rc, rd;\nmov.b64 ra, {%2, %3};\nmov.b64 rb, {%4, %5};\nmov.b64 rc, {%6, %7};\n"
        "fma.rn.f32x2 rd, ra, rb, rc;\nmov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

__device__ __forceinline__ bool last_block_ticket(SolverState* st) {
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(&st->ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    return last != 0;
}

// One element of the ADAM step on s (Alg. 3): g = gsum + mu s, moments, bias-corrected rate,
// projection onto s >= lower.
template <typename T>
__device__ __forceinline__ void adam_s_elem(const TemporalStep<T>& ts, double rate, T gsum, T s, T u0, T v0, T& s1,
                                            T& u1, T& v1) {
    const T g = gsum + (T)ts.mu * s;
    u1 = (T)ts.beta1 * u0 + (T)(1.0 - ts.beta1) * g;
    v1 = (T)ts.beta2 * v0 + (T)(1.0 - ts.beta2) * g * g;
    s1 = s - (T)rate * u1 / (sqrt(v1) + (T)ts.eps);
    if (s1 < (T)ts.lower) s1 = (T)ts.lower;
}

// Run by all threads of the elected last block of a temporal-gradient kernel:
// g = gs + mu s, ADAM step on s with the bias-corrected rate, gs <- 0.
template <typename T>
__device__ void temporal_step_tail(const TemporalStep<T>& ts, T* gs, int R) {
    const double rate = *ts.rate;
    for (int j = threadIdx.x; j < R; j += blockDim.x) {
        T sn, u, v;
        adam_s_elem<T>(ts, rate, __ldcg(gs + j), ts.s[j], ts.u[j], ts.v[j], sn, u, v);
        ts.u[j] = u;
        ts.v[j] = v;
        ts.s[j] = sn;
        gs[j] = T(0);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ts.st->ticket = 0u;
        __threadfence();
    }
}

// Reservoir draw of Alg. 1 at step t (host): j = 1 + floor(u t / 2^32) in
// [1, t] from the Philox block (0, 0, 0, purpose 4 | t); slot j - 1 is
// overwritten when j <= H.
inline uint32_t reservoir_index(uint64_t seed, int64_t t) {
    uint32_t ctr[4] = {0u, 0u, 0u, counter_word3(PUR_RESERVOIR, t)};
    philox4x32_10(ctr, (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32));
    return 1u + bounded_u32(ctr[0], (uint32_t)t);
}

// Hot-row privatisation limits of the sparse kernel.
constexpr int kMaxHot = 64;

// p[0..3] += c (p 16-byte aligned) as one reduction without a returned value (red, not atom: the
// adder never reads the old values, and a returning atomic costs L2-to-SM traffic and a
// scoreboard slot per request).
__device__ __forceinline__ void red_add_f4(float* p, float4 c) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(c.x), "f"(c.y), "f"(c.z), "f"(c.w)
                 : "memory");
}
__device__ __forceinline__ void red_add_f2(float* p, float2 c) {   // p 8-byte aligned
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(c.x), "f"(c.y) : "memory");
}

__device__ __forceinline__ void set_err(int* err, int bits) {
    if (err) atomicOr(err, bits);
}

// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialization may start while the kernel before it in the stream is still
// running; grid_dep_wait() returns once that kernel has completed and its
// writes are visible (at once for a kernel launched without the attribute).
// Everything before the wait may read only data that no kernel of the last
// two in the stream writes, and may write nothing in global memory.
// grid_dep_launch() lets the next kernel start; it is issued after the wait,
// so a kernel that starts early always finds every kernel but its immediate
// predecessor complete.
// A build with SGCP_NO_GRID_DEP defined (the serial profiling build) has neither the instructions
// nor programmatic launches.
#ifndef SGCP_NO_GRID_DEP
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
#else
__device__ __forceinline__ void grid_dep_wait() {}
__device__ __forceinline__ void grid_dep_launch() {}
#endif

}  // namespace sgcp
