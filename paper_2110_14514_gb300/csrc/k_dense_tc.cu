// Dense 3-way fused GCP gradient on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in TMEM), for the BF16 / FP16 MTTKRP precision
// modes (arXiv 2110.14514 Sec. 2.2, eqs. gcp_grad_A / gcp_grad_lambda over
// every entry of a dense slice).
//
// Tile: 128 (i1, i2) rows (8 i1 x 16 i2) x 128 i3 columns.  Per tile
//   M  = KR . A3'        KR[(i1,i2), j] = s_j A1[i1,j] A2[i2,j]; computed as
//                        KR_hi A3_hi' + KR_hi A3_lo' + KR_lo A3_hi' with bf16
//                        hi/lo splits (Henry, Tang, Heinecke, ARITH 2019), so
//                        m keeps ~16 bits and y = df/dm(x, m) stays accurate
//   Y  = df/dm(X, M)     FP32 from TMEM, stored as the MTTKRP operand type
//   T  = Y . A3          -> G1, G2, gs by SIMT reductions (as the FP32 kernel)
//   G3 += Y' . KR        accumulated in TMEM over the block's tiles
// All shared-memory operands use the no-swizzle canonical layout: element
// (r, k) of an (rows x K) tile at (r/8)*SBO + (k/8)*128 + (r%8)*16 + (k%8)*2
// bytes, SBO = K/8 * 128; transposed uses read the same tile MN-major.  A block keeps one i3 block and walks a
// sub-box of n1 x n2 row tiles; G1 / G2 rows accumulate in shared memory and
// G3 in TMEM, and everything is added to global memory once per block.
// Every wait on an mbarrier is bounded; on timeout the kernel records
// ERRB_TIMEOUT in the error word, stops issuing work, and frees its TMEM.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"
#include "sgcp.h"

namespace sgcp {

namespace {

constexpr int kRows = 128;      // (i1, i2) rows per tile
constexpr int kB1 = 8, kB2 = 16;
constexpr int kCols = 128;      // i3 columns per tile
constexpr int kThreads = 256;
constexpr int kTmemCols = 256;  // D1: [0,128), T: [128, 128+R), G3: [192, 192+R)
constexpr int kXld = 132;       // row stride (floats) of the X tile in shared memory: 16-byte aligned, conflict-free
constexpr long kWaitLimit = 1L << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle.  LBO is the byte step between
// core matrices along K, SBO the step along M (or N); this holds for both
// K-major and MN-major operands (checked by measurement on GB300).
__device__ __forceinline__ uint64_t make_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;                        // descriptor version for tcgen05
    return d;
}

// kind::f16 instruction descriptor: D = f32, A = B = (bf16 ? BF16 : F16);
// a_mn / b_mn select MN-major (transposed) operands.
__device__ __forceinline__ uint32_t make_idesc(int M, int N, bool bf16, bool a_mn, bool b_mn) {
    const uint32_t ab = bf16 ? 1u : 0u;
    return (1u << 4) | (ab << 7) | (ab << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of element (r, k) in a K-major canonical tile with K columns
__device__ __forceinline__ uint32_t cano(int r, int k, int K) {
    return (uint32_t)((r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void mma(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 ::"r"(dtmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar)));
}

__device__ __forceinline__ bool wait_phase(uint64_t* mbar, uint32_t phase) {
    uint32_t done = 0;
    for (long it = 0; it < kWaitLimit && !done; ++it) {
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(smem_u32(mbar)), "r"(phase));
    }
    return done != 0;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <bool BF16>
struct Op;
template <>
struct Op<true> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ T cvt(float x) { return __float2bfloat16_rn(x); }
};
template <>
struct Op<false> {
    using T = __half;
    static __device__ __forceinline__ T cvt(float x) { return __float2half_rn(x); }
};

}  // namespace

// Shared-memory plan (bytes), R = rank (multiple of 16, <= 64).  Every tile is
// stored once, K-major canonical in its natural orientation; the GEMMs that
// need it transposed read it through an MN-major descriptor (the core matrices
// of a K-major (rows x K) tile are exactly the core matrices of the MN-major
// (K x rows) view), so no transposed copies are built:
//   KRhi, KRlo   [128 rows][R]  bf16     GEMM1 A (K-major);  GEMM3 B (MN-major, bf16 mode)
//   KR16         [128 rows][R]  fp16     GEMM3 B (MN-major, fp16 mode)
//   A3hi, A3lo   [128 i3][R]    bf16     GEMM1 B (K-major);  GEMM2 B (MN-major, bf16 mode)
//   A316         [128 i3][R]    fp16     GEMM2 B (MN-major, fp16 mode)
//   Yr           [128 rows][128 i3] op   GEMM2 A (K-major);  GEMM3 A (MN-major);
//                                        then reused as Ts [R][128] f32 (T staged for the
//                                        G1 / G2 / gs reductions, rows XOR-swizzled by j)
//   Xs           [128 rows][132] f32     X tile, bulk-copied (TMA) one tile ahead
//   A1t, A1st    [8][64], A2t [16][64], sv [64], acc1 [S1][64], acc2 [S2][64], gsacc [64]  f32
template <bool BF16>
__global__ void __launch_bounds__(kThreads, 1)
    k_dense3_tc(const DenseGradArgs<float> a, int n1, int n2, int nb1, int nb2, int* err) {
    using OT = typename Op<BF16>::T;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ __align__(8) uint64_t mbar_x;
    __shared__ uint32_t tmem_holder;
    __shared__ int abort_flag;
    __shared__ double fred[8];
    if (a.skip && *a.skip) return;
    const int R = a.R;
    const int S1 = kB1 * n1, S2 = kB2 * n2;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = tid & 127, half = tid >> 7;       // TMEM lane of this thread and its column half
    const int64_t I1 = a.dims[0], I2 = a.dims[1], I3 = a.dims[2];
    const int bid = blockIdx.x;
    const int b3 = bid / (nb1 * nb2), rem = bid - b3 * nb1 * nb2;
    const int bb1 = rem / nb2, bb2 = rem - bb1 * nb2;
    const int64_t o1 = (int64_t)bb1 * S1, o2 = (int64_t)bb2 * S2, o3 = (int64_t)b3 * kCols;
    const bool wantG = (a.want & SGCP_WANT_FACTORS) != 0;
    const bool wantS = (a.want & SGCP_WANT_TEMPORAL) != 0;
    const bool wantF = (a.want & SGCP_WANT_LOSS) != 0;
    const float ysc = a.y_scale ? *a.y_scale : 1.0f;
    const float* X = reinterpret_cast<const float*>(a.slice ? a.slice->vals : a.inline_slice.vals);
    // rows of X are 16-byte aligned: bulk copies (else plain loads)
    const bool xtma = (I3 % 4) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;

    unsigned char* p = sm;
    __nv_bfloat16* KRhi = reinterpret_cast<__nv_bfloat16*>(p); p += kRows * R * 2;
    __nv_bfloat16* KRlo = reinterpret_cast<__nv_bfloat16*>(p); p += kRows * R * 2;
    __nv_bfloat16* A3hi = reinterpret_cast<__nv_bfloat16*>(p); p += kCols * R * 2;
    __nv_bfloat16* A3lo = reinterpret_cast<__nv_bfloat16*>(p); p += kCols * R * 2;
    __half* KR16 = reinterpret_cast<__half*>(p); p += BF16 ? 0 : kRows * R * 2;
    __half* A316 = reinterpret_cast<__half*>(p); p += BF16 ? 0 : kCols * R * 2;
    OT* Yr = reinterpret_cast<OT*>(p); p += kRows * kCols * 2;
    float* Ts = reinterpret_cast<float*>(Yr);                       // aliases Yr after GEMM2 / GEMM3
    float* Xs = reinterpret_cast<float*>(p); p += kRows * kXld * 4;
    float* A1t = reinterpret_cast<float*>(p); p += kB1 * 64 * 4;
    float* A1st = reinterpret_cast<float*>(p); p += kB1 * 64 * 4;
    float* A2t = reinterpret_cast<float*>(p); p += kB2 * 64 * 4;
    float* sv = reinterpret_cast<float*>(p); p += 64 * 4;
    float* acc1 = reinterpret_cast<float*>(p); p += S1 * 64 * 4;
    float* acc2 = reinterpret_cast<float*>(p); p += S2 * 64 * 4;
    float* gsacc = reinterpret_cast<float*>(p);

    // ---- set-up: TMEM, mbarrier, accumulators, the block's A3 panels
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        abort_flag = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar_x)), "r"(kRows));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    for (int j = tid; j < 64; j += kThreads) sv[j] = j < R ? a.s[j] : 0.0f;
    for (int i = tid; i < (S1 + S2 + 1) * 64; i += kThreads) acc1[i] = 0.0f;
    __syncthreads();
    // A3 panel: item = (i3 row, 8 consecutive j), 16-byte stores
    for (int i = tid; i < kCols * (R / 8); i += kThreads) {
        const int c = i / (R / 8), j8 = (i - c * (R / 8)) * 8;
        const bool cv = o3 + c < I3;
        uint32_t hi[4], lo[4], h16[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float v0 = cv ? a.A[2][(o3 + c) * R + j8 + 2 * q] : 0.0f;
            const float v1 = cv ? a.A[2][(o3 + c) * R + j8 + 2 * q + 1] : 0.0f;
            const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
            const __nv_bfloat162 l = __floats2bfloat162_rn(v0 - __low2float(h), v1 - __high2float(h));
            const __half2 f = __floats2half2_rn(v0, v1);
            hi[q] = *reinterpret_cast<const uint32_t*>(&h);
            lo[q] = *reinterpret_cast<const uint32_t*>(&l);
            h16[q] = *reinterpret_cast<const uint32_t*>(&f);
        }
        const uint32_t off = cano(c, j8, R);
        *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(A3hi) + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(A3lo) + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        if (!BF16)
            *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(A316) + off) = make_uint4(h16[0], h16[1], h16[2], h16[3]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_holder;
    const uint32_t tD1 = tmem, tT = tmem + 128, tG3 = tmem + 192;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    const uint32_t id_m = make_idesc(128, kCols, true, false, false);
    const uint32_t id_2 = make_idesc(128, R, BF16, false, true);    // A = Y K-major, B = A3 MN-major
    const uint32_t id_3 = make_idesc(128, R, BF16, true, true);     // A = Y' MN-major, B = KR MN-major
    const uint32_t krmt = smem_u32(BF16 ? (const void*)KRhi : (const void*)KR16);
    const uint32_t a3mt = smem_u32(BF16 ? (const void*)A3hi : (const void*)A316);
    uint32_t phase = 0, phase_x = 0;
    int pending_x = 0;                        // bulk copies issued and not yet waited for (uniform)
    float fsum = 0.0f;
    int tiles_done = 0;
    // threads 0..127: each bulk-copies its X row of tile (a1, a2) into Xs; mbar_x counts the 128
    // arrivals and the transferred bytes
    auto issue_x = [&](int64_t a1, int64_t a2) {
        const int64_t ncol = (I3 - o3) < kCols ? (I3 - o3) : kCols;
        const uint32_t rowbytes = (uint32_t)ncol * 4;
        const int r = tid;
        const int64_t i1 = a1 + r / kB2, i2 = a2 + r % kB2;
        if (i1 < I1 && i2 < I2) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&mbar_x)),
                         "r"(rowbytes) : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         ::"r"(smem_u32(Xs + r * kXld)), "l"(X + (i1 * I2 + i2) * I3 + o3), "r"(rowbytes),
                         "r"(smem_u32(&mbar_x))
                         : "memory");
        } else {
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&mbar_x)) : "memory");
        }
    };
    if (xtma && o1 < I1 && o2 < I2) {
        if (tid < kRows) issue_x(o1, o2);
        pending_x = 1;
    }

    for (int t1 = 0; t1 < n1; ++t1) {
        const int64_t i1b = o1 + (int64_t)t1 * kB1;
        if (i1b >= I1) break;
        for (int t2 = 0; t2 < n2; ++t2) {
            const int64_t i2b = o2 + (int64_t)t2 * kB2;
            if (i2b >= I2) break;
            if (abort_flag) break;
            // next tile of this block (for the X prefetch)
            int64_t n1b = i1b, n2b = i2b + kB2;
            if (t2 + 1 >= n2 || n2b >= I2) {
                n1b = i1b + kB1;
                n2b = o2;
                if (t1 + 1 >= n1) n1b = I1;   // none
            }
            // ---- factor rows of the tile and the Khatri-Rao panel KR = (s * A1) (.) A2
            for (int i = tid; i < kB1 * R; i += kThreads) {
                const int r = i / R, j = i - r * R;
                const float v = (i1b + r < I1) ? a.A[0][(i1b + r) * R + j] : 0.0f;
                A1t[r * 64 + j] = v;
                A1st[r * 64 + j] = v * sv[j];
            }
            for (int i = tid; i < kB2 * R; i += kThreads) {
                const int r = i / R, j = i - r * R;
                A2t[r * 64 + j] = (i2b + r < I2) ? a.A[1][(i2b + r) * R + j] : 0.0f;
            }
            __syncthreads();
            for (int i = tid; i < kRows * (R / 8); i += kThreads) {
                const int r = i / (R / 8), j8 = (i - r * (R / 8)) * 8;
                const float* a1 = A1st + (r / kB2) * 64 + j8;
                const float* a2 = A2t + (r % kB2) * 64 + j8;
                uint32_t hi[4], lo[4], h16[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float v0 = a1[2 * q] * a2[2 * q], v1 = a1[2 * q + 1] * a2[2 * q + 1];
                    const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
                    const __nv_bfloat162 l = __floats2bfloat162_rn(v0 - __low2float(h), v1 - __high2float(h));
                    const __half2 f = __floats2half2_rn(v0, v1);
                    hi[q] = *reinterpret_cast<const uint32_t*>(&h);
                    lo[q] = *reinterpret_cast<const uint32_t*>(&l);
                    h16[q] = *reinterpret_cast<const uint32_t*>(&f);
                }
                const uint32_t off = cano(r, j8, R);
                *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(KRhi) + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(KRlo) + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                if (!BF16)
                    *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(KR16) + off) =
                        make_uint4(h16[0], h16[1], h16[2], h16[3]);
            }
            asm volatile("fence.proxy.async.shared::cta;");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;");
            // ---- GEMM1: M = KR A3' in three bf16 products
            if (tid == 0) {
                const uint32_t sboR = (uint32_t)R * 16;
                const uint32_t krh = smem_u32(KRhi), krl = smem_u32(KRlo), a3h = smem_u32(A3hi), a3l = smem_u32(A3lo);
                const uint32_t Aop[3] = {krh, krh, krl}, Bop[3] = {a3h, a3l, a3h};
                for (int sp = 0; sp < 3; ++sp)
                    for (int kk = 0; kk < R / 16; ++kk)
                        mma(tD1, make_desc(Aop[sp] + kk * 256, 128, sboR), make_desc(Bop[sp] + kk * 256, 128, sboR),
                            id_m, (sp > 0 || kk > 0) ? 1u : 0u);
                commit(&mbar);
            }
            if (!wait_phase(&mbar, phase)) {
                if (tid == 0) {
                    abort_flag = 1;
                    set_err(err, ERRB_TIMEOUT);
                }
            }
            phase ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;");
            __syncthreads();
            if (abort_flag) break;
            // ---- Y = df/dm(X, M): thread = TMEM lane (row), half = which 64 columns
            if (xtma) {
                if (!wait_phase(&mbar_x, phase_x)) {
                    if (tid == 0) set_err(err, ERRB_TIMEOUT);
                    abort_flag = 1;
                }
                phase_x ^= 1u;
                pending_x = 0;
            }
            {
                const int r = row;
                const int64_t i1 = i1b + r / kB2, i2 = i2b + r % kB2;
                const bool rv = i1 < I1 && i2 < I2;
                const float* xrow = X + (i1 * I2 + i2) * I3 + o3;
                const float* xs = Xs + r * kXld;
#pragma unroll 1
                for (int c0 = 64 * half; c0 < 64 * half + 64; c0 += 16) {
                    float m[16], x[16];
                    tmem_ld16(tD1 + lane_base + (uint32_t)c0, m);
                    if (xtma) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float4 v = *reinterpret_cast<const float4*>(xs + c0 + 4 * q);
                            x[4 * q] = v.x;
                            x[4 * q + 1] = v.y;
                            x[4 * q + 2] = v.z;
                            x[4 * q + 3] = v.w;
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 16; ++q) x[q] = (rv && o3 + c0 + q < I3) ? __ldg(xrow + c0 + q) : 0.0f;
                    }
                    uint32_t packed[8];
#pragma unroll
                    for (int q = 0; q < 16; q += 2) {
                        float y2[2];
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const bool valid = rv && (o3 + c0 + q + e < I3);
                            float y = 0.0f;
                            if (valid) {
                                y = loss_dfdm<float>(a.loss, x[q + e], m[q + e], a.eps) * ysc;
                                if (wantF) {
                                    float f, yy;
                                    loss_eval<float>(a.loss, x[q + e], m[q + e], a.eps, f, yy);
                                    fsum += f * ysc;
                                }
                            }
                            y2[e] = y;
                        }
                        if (BF16) {
                            const __nv_bfloat162 h = __floats2bfloat162_rn(y2[0], y2[1]);
                            packed[q / 2] = *reinterpret_cast<const uint32_t*>(&h);
                        } else {
                            const __half2 h = __floats2half2_rn(y2[0], y2[1]);
                            packed[q / 2] = *reinterpret_cast<const uint32_t*>(&h);
                        }
                    }
                    unsigned char* yb = reinterpret_cast<unsigned char*>(Yr);
                    *reinterpret_cast<uint4*>(yb + cano(r, c0, kCols)) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
                    *reinterpret_cast<uint4*>(yb + cano(r, c0 + 8, kCols)) = make_uint4(packed[4], packed[5], packed[6], packed[7]);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (abort_flag) break;
            // Xs is consumed: prefetch the next tile's X behind the rest of this tile
            if (xtma && n1b < I1 && n2b < I2) {
                if (tid < kRows) issue_x(n1b, n2b);
                pending_x = 1;
            }
            // ---- GEMM2: T = Y A3 ; GEMM3: G3 += Y' KR
            if (tid == 0) {
                const uint32_t yr = smem_u32(Yr);
                const uint32_t ldR = (uint32_t)R * 16;      // 8-row step of an R-wide tile
                for (int kk = 0; kk < kCols / 16; ++kk)    // K = i3
                    mma(tT, make_desc(yr + kk * 256, 128, 2048), make_desc(a3mt + kk * 2 * ldR, ldR, 128), id_2,
                        kk > 0 ? 1u : 0u);
                if (wantG)
                    for (int kk = 0; kk < kRows / 16; ++kk)   // K = rows
                        mma(tG3, make_desc(yr + kk * 4096, 2048, 128), make_desc(krmt + kk * 2 * ldR, ldR, 128), id_3,
                            (tiles_done > 0 || kk > 0) ? 1u : 0u);
                commit(&mbar);
            }
            if (!wait_phase(&mbar, phase)) {
                if (tid == 0) {
                    abort_flag = 1;
                    set_err(err, ERRB_TIMEOUT);
                }
            }
            phase ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;");
            __syncthreads();
            if (abort_flag) break;
            ++tiles_done;
            // ---- T to shared memory (Ts[j][row], consecutive rows in consecutive words)
            {
                const int cb = (R % 32 == 0) ? (R / 2) * half : (half ? R : 0);
                const int ce = (R % 32 == 0) ? cb + R / 2 : R;
                for (int c0 = cb; c0 < ce; c0 += 16) {
                    float tv[16];
                    tmem_ld16(tT + lane_base + (uint32_t)c0, tv);
#pragma unroll
                    for (int q = 0; q < 16; ++q) Ts[(c0 + q) * 128 + (row ^ ((c0 + q) & 31))] = tv[q];
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            // ---- G1 (and gs) over the 16 i2 rows of each i1; G2 over the 8 i1 rows of each i2
            for (int it = tid; it < kB1 * R; it += kThreads) {
                const int j = it % R, i1l = it / R;
                const float* tr = Ts + j * 128;
                const int sw = j & 31;
                float g1 = 0.0f;
#pragma unroll
                for (int i2l = 0; i2l < kB2; ++i2l) g1 += A2t[i2l * 64 + j] * tr[(i1l * kB2 + i2l) ^ sw];
                if (wantG) acc1[(t1 * kB1 + i1l) * 64 + j] += sv[j] * g1;
                if (wantS) atomicAdd(&gsacc[j], A1t[i1l * 64 + j] * g1);
            }
            if (wantG) {
                for (int it = tid; it < kB2 * R; it += kThreads) {
                    const int j = it % R, i2l = it / R;
                    const float* tr = Ts + j * 128;
                    const int sw = j & 31;
                    float g2 = 0.0f;
#pragma unroll
                    for (int i1l = 0; i1l < kB1; ++i1l) g2 += A1st[i1l * 64 + j] * tr[(i1l * kB2 + i2l) ^ sw];
                    acc2[(t2 * kB2 + i2l) * 64 + j] += g2;
                }
            }
            __syncthreads();
        }
        if (abort_flag) break;
    }

    // ---- an aborted block still lets its own bulk copy land before shared memory is released
    if (pending_x) wait_phase(&mbar_x, phase_x);
    // ---- flush: G3 from TMEM, G1 / G2 / gs from shared memory, the loss
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (wantG && tiles_done > 0 && !abort_flag) {
        const int c = row;                    // i3 row of the G3 accumulator
        const int64_t i3 = o3 + c;
        const int cb = (R % 32 == 0) ? (R / 2) * half : (half ? R : 0);
        const int ce = (R % 32 == 0) ? cb + R / 2 : R;
        for (int j0 = cb; j0 < ce; j0 += 16) {
            float g[16];
            tmem_ld16(tG3 + lane_base + (uint32_t)j0, g);
            if (i3 < I3)
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    if (g[q] != 0.0f) atomicAdd(a.G[2] + i3 * R + j0 + q, g[q]);
        }
    }
    __syncthreads();
    if (wantG) {
        for (int i = tid; i < S1 * R; i += kThreads) {
            const int r = i / R, j = i - r * R;
            const float v = acc1[r * 64 + j];
            if (o1 + r < I1 && v != 0.0f) atomicAdd(a.G[0] + (o1 + r) * R + j, v);
        }
        for (int i = tid; i < S2 * R; i += kThreads) {
            const int r = i / R, j = i - r * R;
            const float v = acc2[r * 64 + j];
            if (o2 + r < I2 && v != 0.0f) atomicAdd(a.G[1] + (o2 + r) * R + j, v);
        }
    }
    if (wantS)
        for (int j = tid; j < R; j += kThreads)
            if (gsacc[j] != 0.0f) atomicAdd(a.gs + j, gsacc[j]);
    if (wantF) {
        double fd = (double)fsum;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) fd += __shfl_xor_sync(SGCP_FULL_MASK, fd, o);
        if (lane == 0) fred[warp] = fd;
        __syncthreads();
        if (tid == 0) {
            double tot = 0.0;
            for (int i = 0; i < kThreads / 32; ++i) tot += fred[i];
            if (tot != 0.0) atomicAdd(a.f, tot);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    if (a.tstep_on && last_block_ticket(a.tstep.st)) temporal_step_tail<float>(a.tstep, a.gs, R);
}

static int tc_num_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

cudaError_t launch_dense_grad_tc(const DenseGradArgs<float>& a, bool bf16, int* err, cudaStream_t st,
                                 int64_t* launches) {
    if (a.ndim != 3 || a.R % 16 != 0 || a.R > 64) return cudaErrorInvalidValue;
    const int64_t I1 = a.dims[0], I2 = a.dims[1], I3 = a.dims[2];
    const int64_t nb3 = (I3 + kCols - 1) / kCols;
    const int64_t t1 = (I1 + kB1 - 1) / kB1, t2 = (I2 + kB2 - 1) / kB2;
    // sub-box of n1 x n2 tiles: minimise (waves x tiles per block), then prefer fewer blocks
    const int64_t sms = tc_num_sms();
    int n1 = 1, n2 = 1;
    int64_t best = -1;
    for (int m1 = 1; m1 <= 4; m1 *= 2)
        for (int m2 = 1; m2 <= 2; m2 *= 2) {
            if (m1 > 1 && (m1 / 2) * kB1 >= I1) continue;
            if (m2 > 1 && (m2 / 2) * kB2 >= I2) continue;
            const int64_t blocks = ((t1 + m1 - 1) / m1) * ((t2 + m2 - 1) / m2) * nb3;
            // tiles on the critical path plus a per-block start-up of about 3/4 of a tile
            // (TMEM, the A3 panel, an unoverlapped first X copy); ties go to more tiles per block
            const int64_t cost = ((blocks + sms - 1) / sms) * (m1 * m2 * 64 + 48) - m1 * m2;
            if (best < 0 || cost < best) {
                best = cost;
                n1 = m1;
                n2 = m2;
            }
        }
    const int nb1 = (int)((t1 + n1 - 1) / n1), nb2 = (int)((t2 + n2 - 1) / n2);
    const int64_t blocks = (int64_t)nb1 * nb2 * nb3;
    const int R = a.R;
    const size_t smem = (size_t)kRows * R * 2 * 2 + (size_t)kCols * R * 2 * 2 +
                        (bf16 ? 0 : (size_t)(kRows + kCols) * R * 2) + (size_t)kRows * kCols * 2 + (size_t)kRows * kXld * 4 +
                        (size_t)(2 * kB1 + kB2 + 1) * 64 * 4 + (size_t)(kB1 * n1 + kB2 * n2 + 1) * 64 * 4 + 1024;
    if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
    if (bf16) {
        cudaFuncSetAttribute(k_dense3_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_dense3_tc<true><<<(unsigned)blocks, kThreads, smem, st>>>(a, n1, n2, nb1, nb2, err);
    } else {
        cudaFuncSetAttribute(k_dense3_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_dense3_tc<false><<<(unsigned)blocks, kThreads, smem, st>>>(a, n1, n2, nb1, nb2, err);
    }
    if (launches) *launches += 1;
    return cudaGetLastError();
}

}  // namespace sgcp
