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
//   T  = Y . A3          -> G1, G2, gs by SIMT reductions (float4 atomics per tile)
//   G3 += Y' . KR        accumulated in TMEM while the i3 block stays the same
// All shared-memory operands use the no-swizzle canonical layout: element
// (r, k) of an (rows x K) tile at (r/8)*SBO + (k/8)*128 + (r%8)*16 + (k%8)*2
// bytes, SBO = K/8 * 128; transposed uses read the same tile MN-major.
//
// Persistent schedule: one block of 512 threads per SM takes a contiguous run
// of tiles (i3 block major, then i1, then i2).  The model product of the next
// tile runs on the tensor core while this tile's loss epilogue, T read-back
// and reductions run on the CUDA cores: two TMEM model accumulators and two
// KR panels alternate, the next X tile arrives by cp.async.bulk and the next
// factor rows by cp.async behind the current tile's work.  Per tile:
//   wait M(t), X(t) -> stage rows(t+1) -> epilogue(t): Y -> copy X(t+1) ->
//   issue T, G3 (t) -> build KR(t+1) -> issue M(t+1) -> wait T -> reductions(t)
// A change of i3 block drains the tensor core first (the A3 panel changes).
// Every wait on an mbarrier is bounded; on timeout the kernel records
// ERRB_TIMEOUT in the error word, stops issuing work, lets its own copies land
// and frees its TMEM.
#include <cstring>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"
#include "sgcp.h"

namespace sgcp {

namespace {

constexpr int kRows = 128;      // (i1, i2) rows per tile
constexpr int kB1 = 8, kB2 = 16;
constexpr int kCols = 128;      // i3 columns per tile
constexpr int kThreads = 512;
constexpr int kStageLd = 68;    // row stride (floats) of the staged factor rows: 16-byte rows, spread banks
constexpr int kXBase = kThreads - kRows;   // first of the threads that copy X rows
constexpr int kKrLo = 32, kKrCnt = kXBase - 32;   // threads that build the next KR panel beside the MMA issue
constexpr int kTmemCols = 512;  // D1 x 2: [0, 256), T: [256, 256 + R), G3: [320, 320 + R)
constexpr int kXBox = 32;       // i3 columns per tensor-map box (128 bytes: one 128-byte swizzle row)
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

// TMEM -> registers, 16 columns of this thread's lane (issue only).
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
}

// Wait for this thread's TMEM loads; the registers are operands so no use of them moves above the wait.
__device__ __forceinline__ void tmem_wait16(uint32_t (&r)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    tmem_ld16_issue(taddr, r);
    tmem_wait16(r);
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


// Shared-memory plan (bytes), R = rank (multiple of 16, <= 64), in this order:
//   KRh[0], KRh[1] [128 rows][R] bf16   GEMM1 A hi (K-major); GEMM3 B (MN-major) in bf16 mode
//                                       (fp16 mode keeps one KRh)
//   KRl            [128 rows][R] bf16   GEMM1 A lo
//   KR3[0], KR3[1] [128 rows][R] fp16   GEMM3 B in fp16 mode
//   A3hi, A3lo     [128 i3][R]   bf16   GEMM1 B (K-major); GEMM2 B (MN-major) in bf16 mode
//   A316           [128 i3][R]   fp16   GEMM2 B in fp16 mode
//   Yr             [128 rows][128 i3] op  GEMM2 A (K-major), GEMM3 A (MN-major);
//                                       then [4][16][68] f32 G2 partials of the T reduction
//   Xs             [4][128 rows][32] f32  X tile: four tensor-map boxes of 32 i3 columns, each row
//                                       of 128 bytes with its 16-byte chunks XOR-swizzled by (row mod 8)
//   stage          [2][24 rows][64] f32 A1 rows (8) and A2 rows (16) of a tile (cp.async)
//   sv [64], gsacc [64] f32
struct TcPlan {
    int KRh0, KRh1, KRl, KR30, KR31, A3hi, A3lo, A316, Yr, Xs, stage, sv, gsacc, total;
};

__host__ __device__ inline TcPlan tc_plan(int R, bool bf16) {
    TcPlan p{};
    const int kr = kRows * R * 2, a3 = kCols * R * 2;
    int o = 0;
    p.KRh0 = o; o += kr;
    p.KRh1 = bf16 ? o : p.KRh0; o += bf16 ? kr : 0;
    p.KRl = o; o += kr;
    p.KR30 = o; o += bf16 ? 0 : kr;
    p.KR31 = o; o += bf16 ? 0 : kr;
    if (bf16) p.KR30 = p.KR31 = -1;
    p.A3hi = o; o += a3;
    p.A3lo = o; o += a3;
    p.A316 = bf16 ? -1 : o; o += bf16 ? 0 : a3;
    p.Yr = o;
    o += kRows * kCols * 2;   // >= 4 * 16 * kStageLd * 4
    o = (o + 1023) & ~1023;
    p.Xs = o; o += kRows * kCols * 4;
    p.stage = o; o += 2 * 24 * kStageLd * 4;
    p.sv = o; o += 64 * 4;
    p.gsacc = o; o += 64 * 4;
    p.total = o;
    return p;
}

template <bool BF16, int LOSS>
__global__ void __launch_bounds__(kThreads, 1)
    k_dense3_tc(const DenseGradArgs<float> a, int t1n, int t2n, int ntiles, int* err) {
    using OT = typename Op<BF16>::T;
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar1, mbar2, mbar_x;
    __shared__ uint32_t tmem_holder;
    __shared__ int abort_flag;
    __shared__ double fred[kThreads / 32];
    if (a.skip && *a.skip) return;
    const int R = a.R;
    const TcPlan P = tc_plan(R, BF16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, cq = warp >> 2;     // TMEM lane quarter and column quarter of this warp
    const int row = 32 * quarter + lane;              // TMEM lane = tile row of this thread
    const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
    const int64_t I1 = a.dims[0], I2 = a.dims[1], I3 = a.dims[2];
    const bool wantG = (a.want & SGCP_WANT_FACTORS) != 0;
    const bool wantS = (a.want & SGCP_WANT_TEMPORAL) != 0;
    const bool wantF = (a.want & SGCP_WANT_LOSS) != 0;
    const bool g23 = wantG || wantS;
    const float ysc = a.y_scale ? *a.y_scale : 1.0f;
    const float* X = reinterpret_cast<const float*>(a.slice ? a.slice->vals : a.inline_slice.vals);
    const bool xtma = a.xmap != nullptr;     // X tiles by TMA from the slice's tensor map
    // this block's run of tiles
    const int tb = (int)((int64_t)blockIdx.x * ntiles / gridDim.x);
    const int te = (int)((int64_t)(blockIdx.x + 1) * ntiles / gridDim.x);

    auto KRhp = [&](int b) { return reinterpret_cast<__nv_bfloat16*>(sm + (b ? P.KRh1 : P.KRh0)); };
    __nv_bfloat16* KRl = reinterpret_cast<__nv_bfloat16*>(sm + P.KRl);
    auto KR3p = [&](int b) { return reinterpret_cast<__half*>(sm + (b ? P.KR31 : P.KR30)); };
    __nv_bfloat16* A3hi = reinterpret_cast<__nv_bfloat16*>(sm + P.A3hi);
    __nv_bfloat16* A3lo = reinterpret_cast<__nv_bfloat16*>(sm + P.A3lo);
    __half* A316 = BF16 ? nullptr : reinterpret_cast<__half*>(sm + P.A316);
    OT* Yr = reinterpret_cast<OT*>(sm + P.Yr);
    float* Xs = reinterpret_cast<float*>(sm + P.Xs);
    float* stage = reinterpret_cast<float*>(sm + P.stage);   // [2][24][64]
    float* sv = reinterpret_cast<float*>(sm + P.sv);
    float* gsacc = reinterpret_cast<float*>(sm + P.gsacc);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        abort_flag = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar1)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar2)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar_x)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    for (int j = tid; j < 64; j += kThreads) {
        sv[j] = j < R ? a.s[j] : 0.0f;
        gsacc[j] = 0.0f;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_holder;
    const uint32_t tT = tmem + 256, tG3 = tmem + 320;
    const uint32_t id_m = make_idesc(128, kCols, true, false, false);
    const uint32_t id_2 = make_idesc(128, R, BF16, false, true);    // A = Y K-major, B = A3 MN-major
    const uint32_t id_3 = make_idesc(128, R, BF16, true, true);     // A = Y' MN-major, B = KR MN-major
    const uint32_t sboR = (uint32_t)R * 16;                         // 8-row step of an R-wide tile

    struct TileIx {
        int b3;
        int64_t i1b, i2b, o3;
    };
    auto decode = [&](int t) {
        TileIx x;
        const int i2t = t % t2n, rest = t / t2n;
        const int i1t = rest % t1n;
        x.b3 = rest / t1n;
        x.i1b = (int64_t)i1t * kB1;
        x.i2b = (int64_t)i2t * kB2;
        x.o3 = (int64_t)x.b3 * kCols;
        return x;
    };
    // A1 (8 rows) and A2 (16 rows) of a tile into stage[buf] by cp.async, zero-filled outside the slice
    auto stage_rows = [&](const TileIx& x, int buf) {
        const int per = R / 4;                    // 16-byte chunks per row
        const int n = 24 * per;
        for (int i = tid; i < n; i += kThreads) {
            const int r = i / per, c = (i - r * per) * 4;
            const bool is1 = r < kB1;
            const int64_t gr = is1 ? x.i1b + r : x.i2b + (r - kB1);
            const bool ok = is1 ? gr < I1 : gr < I2;
            const float* src = (is1 ? a.A[0] : a.A[1]) + (ok ? gr * R + c : 0);
            const uint32_t dst = smem_u32(stage + (buf * 24 + r) * kStageLd + c);
            const uint32_t bytes = ok ? 16u : 0u;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    // A3 panel of an i3 block: item = (i3 row, 8 consecutive j), 16-byte stores
    auto build_a3 = [&](int64_t o3) {
        const int nj = R / 8;
        for (int i = tid; i < kCols * nj; i += kThreads) {
            const int rlo = i & 7, rest = i >> 3;
            const int j8 = (rest % nj) * 8, c = (rest / nj) * 8 + rlo;
            const bool cv = o3 + c < I3;
            float a8[8];
            {
                const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
                const float4* src = reinterpret_cast<const float4*>(a.A[2] + (cv ? (o3 + c) * R + j8 : 0));
                const float4 p0 = cv ? __ldg(src) : z, p1 = cv ? __ldg(src + 1) : z;
                a8[0] = p0.x, a8[1] = p0.y, a8[2] = p0.z, a8[3] = p0.w;
                a8[4] = p1.x, a8[5] = p1.y, a8[6] = p1.z, a8[7] = p1.w;
            }
            uint32_t hi[4], lo[4], h16[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float v0 = a8[2 * q], v1 = a8[2 * q + 1];
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
                *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(A316) + off) =
                    make_uint4(h16[0], h16[1], h16[2], h16[3]);
        }
    };
    // KR panel of a tile from its staged rows: KR = (s A1) (.) A2 as bf16 hi / lo (and fp16).
    // A warp covers 8 consecutive rows x 4 chunks of 8 j, so its 16-byte stores hit distinct banks.
    auto build_kr = [&](int sbuf, int kbuf, int lo, int cnt) {   // by threads lo .. lo + cnt - 1
        if (tid < lo || tid >= lo + cnt) return;
        const float* A1 = stage + sbuf * 24 * kStageLd;
        const float* A2 = A1 + kB1 * kStageLd;
        __nv_bfloat16* kh = KRhp(kbuf);
        const int nj = R / 8;
        for (int i = tid - lo; i < kRows * nj; i += cnt) {
            const int rlo = i & 7, rest = i >> 3;
            const int j8 = (rest % nj) * 8, r = (rest / nj) * 8 + rlo;
            float s8[8], a18[8], a28[8];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float4 sq = *reinterpret_cast<const float4*>(sv + j8 + 4 * h);
                const float4 aq = *reinterpret_cast<const float4*>(A1 + (r / kB2) * kStageLd + j8 + 4 * h);
                const float4 bq = *reinterpret_cast<const float4*>(A2 + (r % kB2) * kStageLd + j8 + 4 * h);
                s8[4 * h] = sq.x, s8[4 * h + 1] = sq.y, s8[4 * h + 2] = sq.z, s8[4 * h + 3] = sq.w;
                a18[4 * h] = aq.x, a18[4 * h + 1] = aq.y, a18[4 * h + 2] = aq.z, a18[4 * h + 3] = aq.w;
                a28[4 * h] = bq.x, a28[4 * h + 1] = bq.y, a28[4 * h + 2] = bq.z, a28[4 * h + 3] = bq.w;
            }
            uint32_t hi[4], lo[4], h16[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float v0 = s8[2 * q] * a18[2 * q] * a28[2 * q];
                const float v1 = s8[2 * q + 1] * a18[2 * q + 1] * a28[2 * q + 1];
                const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
                const __nv_bfloat162 l = __floats2bfloat162_rn(v0 - __low2float(h), v1 - __high2float(h));
                const __half2 f = __floats2half2_rn(v0, v1);
                hi[q] = *reinterpret_cast<const uint32_t*>(&h);
                lo[q] = *reinterpret_cast<const uint32_t*>(&l);
                h16[q] = *reinterpret_cast<const uint32_t*>(&f);
            }
            const uint32_t off = cano(r, j8, R);
            *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(kh) + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(KRl) + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
            if (!BF16)
                *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(KR3p(kbuf)) + off) =
                    make_uint4(h16[0], h16[1], h16[2], h16[3]);
        }
    };
    // operand writes by every thread -> visible to the tensor core
    auto publish_smem = [&]() {
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
    };
    // MMA issue: descriptors formed once per call and stepped by adds (a descriptor's address field
    // counts 16-byte units), loops unrolled, so the issuing thread spends a few instructions per MMA
    auto issue_gemm1 = [&](int dbuf, int kbuf) {
        if (tid == 0) {
            const uint64_t ahd = make_desc(smem_u32(KRhp(kbuf)), 128, sboR), ald = make_desc(smem_u32(KRl), 128, sboR);
            const uint64_t bh = make_desc(smem_u32(A3hi), 128, sboR), bl = make_desc(smem_u32(A3lo), 128, sboR);
            const uint32_t d = tmem + (uint32_t)dbuf * 128;
            const int nk = R >> 4;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                if (kk < nk) mma(d, ahd + 16 * kk, bh + 16 * kk, id_m, kk > 0 ? 1u : 0u);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                if (kk < nk) mma(d, ahd + 16 * kk, bl + 16 * kk, id_m, 1u);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                if (kk < nk) mma(d, ald + 16 * kk, bh + 16 * kk, id_m, 1u);
            commit(&mbar1);
        }
    };
    auto issue_gemm23 = [&](int kbuf, bool g3acc) {
        if (tid == 0) {
            const uint64_t at = make_desc(smem_u32(Yr), 128, 2048);
            const uint64_t bt = make_desc(smem_u32(BF16 ? (const void*)A3hi : (const void*)A316), sboR, 128);
            const uint64_t ag = make_desc(smem_u32(Yr), 2048, 128);
            const uint64_t bg = make_desc(smem_u32(BF16 ? (const void*)KRhp(kbuf) : (const void*)KR3p(kbuf)), sboR, 128);
            const uint64_t stp = (uint64_t)(2 * sboR) >> 4;
#pragma unroll
            for (int kk = 0; kk < kCols / 16; ++kk)
                mma(tT, at + 16 * kk, bt + stp * kk, id_2, kk > 0 ? 1u : 0u);
            if (wantG) {
#pragma unroll
                for (int kk = 0; kk < kRows / 16; ++kk)
                    mma(tG3, ag + 256 * kk, bg + stp * kk, id_3, (g3acc || kk > 0) ? 1u : 0u);
            }
            commit(&mbar2);
        }
    };
    // one thread (kXBase) loads the X tile: four 3D tensor-map boxes of 32 i3 x 16 i2 x 8 i1 floats
    // on mbar_x (64 KB of transactions; boxes reaching past the slice are zero-filled and still count)
    if (xtma && tid == kXBase)
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(a.xmap) : "memory");
    auto issue_x = [&](const TileIx& x) {
        if (tid == kXBase) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&mbar_x)),
                         "r"((uint32_t)(kRows * kCols * 4)) : "memory");
#pragma unroll
            for (int b = 0; b < kCols / kXBox; ++b)
                asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                             " [%0], [%1, {%2, %3, %4}], [%5];"
                             ::"r"(smem_u32(Xs + b * kRows * kXBox)), "l"(a.xmap), "r"((int)(x.o3 + b * kXBox)),
                             "r"((int)x.i2b), "r"((int)x.i1b), "r"(smem_u32(&mbar_x))
                             : "memory");
        }
    };
    auto fail = [&]() {
        if (tid == 0) {
            abort_flag = 1;
            set_err(err, ERRB_TIMEOUT);
        }
    };

    float fsum = 0.0f;
    float gs_acc = 0.0f;                              // gradient of s, column 16 cq + (lane & 15)
    const float s_c = sv[16 * cq + (lane & 15)];
    uint32_t ph1 = 0, ph2 = 0, phx = 0;
    int pending_x = 0;
    bool g3_started = false;
    int b3_open = -1;            // i3 block whose G3 sits in TMEM
    TileIx cur{};
    if (tb < te) {   // the first X tile and factor rows are in flight while the A3 panel is built
        cur = decode(tb);
        if (xtma) {
            issue_x(cur);
            pending_x = 1;
        }
        stage_rows(cur, 0);
        build_a3(cur.o3);
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();
        build_kr(0, 0, 0, kThreads);
        publish_smem();
        issue_gemm1(0, 0);
    }
    for (int t = tb, k = 0; t < te; ++t, ++k) {
        const int cb = k & 1;
        const bool has_next = t + 1 < te;
        const TileIx nxt = has_next ? decode(t + 1) : cur;
        // ---- wait for M(t) and X(t)
        if (!wait_phase(&mbar1, ph1)) fail();
        ph1 ^= 1u;
        if (xtma) {
            if (!wait_phase(&mbar_x, phx)) fail();
            phx ^= 1u;
            pending_x = 0;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        __syncthreads();
        if (abort_flag) break;
        if (has_next) stage_rows(nxt, (k + 1) & 1);
        // ---- epilogue: Y = df/dm(X, M) for columns [32 cq, 32 cq + 32) of this thread's row
        {
            const int64_t i1 = cur.i1b + row / kB2, i2 = cur.i2b + row % kB2;
            const bool rv = i1 < I1 && i2 < I2;
            const bool interior = cur.i1b + kB1 <= I1 && cur.i2b + kB2 <= I2 && cur.o3 + kCols <= I3 && xtma;
            const float* xrow = X + (i1 * I2 + i2) * I3 + cur.o3;
            const int swz = row & 7;     // 128-byte swizzle of this row's 16-byte chunks
            const uint32_t dcol = tmem + (uint32_t)cb * 128 + lane_base;
            unsigned char* yb = reinterpret_cast<unsigned char*>(Yr);
            uint32_t mr[2][16];     // both 16-column halves in flight before one wait
            tmem_ld16_issue(dcol + (uint32_t)(32 * cq), mr[0]);
            tmem_ld16_issue(dcol + (uint32_t)(32 * cq + 16), mr[1]);
            tmem_wait16(mr[0]);
            tmem_wait16(mr[1]);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int c0 = 32 * cq + 16 * h;
                float m[16], x[16], y[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) m[q] = __uint_as_float(mr[h][q]);
                if (xtma) {
                    const float* xb = Xs + (c0 / kXBox) * kRows * kXBox + row * kXBox;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int chunk = ((c0 % kXBox) >> 2) + q;
                        const float4 v = *reinterpret_cast<const float4*>(xb + ((chunk ^ swz) << 2));
                        x[4 * q] = v.x;
                        x[4 * q + 1] = v.y;
                        x[4 * q + 2] = v.z;
                        x[4 * q + 3] = v.w;
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) x[q] = (rv && cur.o3 + c0 + q < I3) ? __ldg(xrow + c0 + q) : 0.0f;
                }
                if (interior) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        y[q] = loss_dfdm<float>(LOSS, x[q], m[q], a.eps) * ysc;
                        if (wantF) {
                            float f, yy;
                            loss_eval<float>(LOSS, x[q], m[q], a.eps, f, yy);
                            fsum += f * ysc;
                        }
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const bool valid = rv && (cur.o3 + c0 + q < I3);
                        y[q] = valid ? loss_dfdm<float>(LOSS, x[q], m[q], a.eps) * ysc : 0.0f;
                        if (wantF && valid) {
                            float f, yy;
                            loss_eval<float>(LOSS, x[q], m[q], a.eps, f, yy);
                            fsum += f * ysc;
                        }
                    }
                }
                if (g23) {
                    uint32_t packed[8];
#pragma unroll
                    for (int q = 0; q < 16; q += 2) {
                        if (BF16) {
                            const __nv_bfloat162 hh = __floats2bfloat162_rn(y[q], y[q + 1]);
                            packed[q / 2] = *reinterpret_cast<const uint32_t*>(&hh);
                        } else {
                            const __half2 hh = __floats2half2_rn(y[q], y[q + 1]);
                            packed[q / 2] = *reinterpret_cast<const uint32_t*>(&hh);
                        }
                    }
                    *reinterpret_cast<uint4*>(yb + cano(row, c0, kCols)) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
                    *reinterpret_cast<uint4*>(yb + cano(row, c0 + 8, kCols)) = make_uint4(packed[4], packed[5], packed[6], packed[7]);
                }
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");   // this thread's rows of the next tile have landed
        publish_smem();
        // ---- three roles side by side (Xs and Y are settled): thread 0 issues T = Y A3 and
        // G3 += Y' KR of this tile, the last 128 threads copy X of the next tile, warps 1 .. 11
        // build the next KR panel (the MMA and copy issue block their threads for ~1-2 K cycles)
        const bool new_b3 = has_next && nxt.b3 != cur.b3;
        if (g23) {
            issue_gemm23(cb, g3_started);
            if (wantG) {
                g3_started = true;
                b3_open = cur.b3;
            }
        }
        if (xtma && has_next) {
            issue_x(nxt);
            pending_x = 1;
        }
        if (has_next && !new_b3) build_kr((k + 1) & 1, (k + 1) & 1, kKrLo, kKrCnt);
        bool t_ready = false;
        auto flush_g3 = [&](int b3) {   // G3 rows of an i3 block: TMEM -> global
            if (16 * cq < R) {
                const int64_t i3 = (int64_t)b3 * kCols + row;
                float g[16];
                tmem_ld16(tG3 + lane_base + (uint32_t)(16 * cq), g);
                if (i3 < I3)
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        red_add_f4(a.G[2] + i3 * R + 16 * cq + 4 * q,
                                   make_float4(g[4 * q], g[4 * q + 1], g[4 * q + 2], g[4 * q + 3]));
            }
        };
        if (new_b3) {   // the A3 panel changes: T and G3 of this tile must be done first
            if (g23) {
                if (!wait_phase(&mbar2, ph2)) fail();
                ph2 ^= 1u;
                asm volatile("tcgen05.fence::after_thread_sync;");
                t_ready = true;
            }
            if (wantG && g3_started) {
                flush_g3(b3_open);
                g3_started = false;
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            build_a3(nxt.o3);
            build_kr((k + 1) & 1, (k + 1) & 1, 0, kThreads);
        }
        if (has_next) publish_smem();   // KR (and A3) of the next tile are in place
        // ---- thread 0 queues the next model product behind T / G3 on the tensor pipe; every warp
        // then reduces its 32 rows x 16 columns of T straight from TMEM (row = 16 i1l + i2l):
        //   G1[i1l] += s * sum_i2l A2[i2l] * T      over the 16 lanes of a half-warp (shuffles)
        //   gs      += sum_i1l A1[i1l] * (sum_i2l A2[i2l] * T)
        //   G2[i2l] += sum_i1l s * A1[i1l] * T      over lane pairs, then the 4 lane quarters in Yr
        if (has_next) issue_gemm1((k + 1) & 1, (k + 1) & 1);
        float* red = reinterpret_cast<float*>(Yr);   // [4 quarters][16 i2l][kStageLd] G2 partials
        if (g23) {
            if (!t_ready) {
                if (!wait_phase(&mbar2, ph2)) fail();
                ph2 ^= 1u;
                asm volatile("tcgen05.fence::after_thread_sync;");
            }
            if (16 * cq < R) {
                const int i1l = row / kB2, i2l = row % kB2;
                const float* A1 = stage + (cb * 24 + i1l) * kStageLd + 16 * cq;
                const float* A2 = stage + (cb * 24 + kB1 + i2l) * kStageLd + 16 * cq;
                float tv[16];
                __syncwarp();   // lane 0 may come from the MMA issue: the TMEM load is warp-wide
                tmem_ld16(tT + lane_base + (uint32_t)(16 * cq), tv);
                float u[16], v[16];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 w2 = *reinterpret_cast<const float4*>(A2 + 4 * q);
                    const float4 w1 = *reinterpret_cast<const float4*>(A1 + 4 * q);
                    const float4 s4 = *reinterpret_cast<const float4*>(sv + 16 * cq + 4 * q);
                    u[4 * q] = w2.x * tv[4 * q], u[4 * q + 1] = w2.y * tv[4 * q + 1];
                    u[4 * q + 2] = w2.z * tv[4 * q + 2], u[4 * q + 3] = w2.w * tv[4 * q + 3];
                    v[4 * q] = s4.x * w1.x * tv[4 * q], v[4 * q + 1] = s4.y * w1.y * tv[4 * q + 1];
                    v[4 * q + 2] = s4.z * w1.z * tv[4 * q + 2], v[4 * q + 3] = s4.w * w1.w * tv[4 * q + 3];
                }
                // reduce-scatter of u over the half-warp: lane ends with column (lane & 15)
                const bool b8 = lane & 8, b4 = lane & 4, b2 = lane & 2, b1 = lane & 1;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float snd = b8 ? u[i] : u[i + 8];
                    u[i] = (b8 ? u[i + 8] : u[i]) + __shfl_xor_sync(SGCP_FULL_MASK, snd, 8);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float snd = b4 ? u[i] : u[i + 4];
                    u[i] = (b4 ? u[i + 4] : u[i]) + __shfl_xor_sync(SGCP_FULL_MASK, snd, 4);
                }
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const float snd = b2 ? u[i] : u[i + 2];
                    u[i] = (b2 ? u[i + 2] : u[i]) + __shfl_xor_sync(SGCP_FULL_MASK, snd, 2);
                }
                {
                    const float snd = b1 ? u[0] : u[1];
                    u[0] = (b1 ? u[1] : u[0]) + __shfl_xor_sync(SGCP_FULL_MASK, snd, 1);
                }
                const int c = lane & 15;
                if (wantS) gs_acc = fmaf(A1[c], u[0], gs_acc);
                if (wantG) {
                    if (cur.i1b + i1l < I1) atomicAdd(a.G[0] + (cur.i1b + i1l) * R + 16 * cq + c, s_c * u[0]);
                    // G2: lanes l and l ^ 16 hold the same i2l; keep 8 columns each, then stage them
                    const bool b16 = lane & 16;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float snd = b16 ? v[i] : v[i + 8];
                        v[i] = (b16 ? v[i + 8] : v[i]) + __shfl_xor_sync(SGCP_FULL_MASK, snd, 16);
                    }
                    float* dst = red + (quarter * kB2 + i2l) * kStageLd + 16 * cq + (b16 ? 8 : 0);
                    *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
                    *reinterpret_cast<float4*>(dst + 4) = make_float4(v[4], v[5], v[6], v[7]);
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        if (g23 && wantG && tid < kB2 * 16) {   // G2 rows of the tile: the 4 quarters' partials
            const int i2l = tid >> 4, c4 = (tid & 15) * 4;
            if (c4 < R && cur.i2b + i2l < I2) {
                float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 w = *reinterpret_cast<const float4*>(red + (q * kB2 + i2l) * kStageLd + c4);
                    g.x += w.x, g.y += w.y, g.z += w.z, g.w += w.w;
                }
                red_add_f4(a.G[1] + (cur.i2b + i2l) * R + c4, g);
            }
        }
        // red (= Yr) is read before the next epilogue writes Y: the barrier at the loop top orders it
        cur = nxt;
    }

    // ---- an aborted block still lets its own copies land before shared memory is released
    if (pending_x) wait_phase(&mbar_x, phx);
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("tcgen05.fence::after_thread_sync;");
    // G3 of the open i3 block: TMEM -> a padded staging copy in Xs (free now; 68-float rows keep
    // the 16-byte stores conflict-free) -> one bulk reduce-add into G^(3) per row, so the blocks
    // sharing an i3 block add whole rows in L2 instead of 16-byte atomics
    if (wantS) {   // lanes l and l ^ 16 hold the same column
        const float g = gs_acc + __shfl_xor_sync(SGCP_FULL_MASK, gs_acc, 16);
        if (lane < 16 && 16 * cq < R && g != 0.0f) atomicAdd(gsacc + 16 * cq + lane, g);
    }
    const bool g3_flush = wantG && g3_started && !abort_flag;
    if (g3_flush && 16 * cq < R) {
        float g[16];
        tmem_ld16(tG3 + lane_base + (uint32_t)(16 * cq), g);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *reinterpret_cast<float4*>(Xs + row * kStageLd + 16 * cq + 4 * q) =
                make_float4(g[4 * q], g[4 * q + 1], g[4 * q + 2], g[4 * q + 3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (g3_flush && tid < kRows) {
        const int64_t i3 = (int64_t)b3_open * kCols + tid;
        if (i3 < I3) {
            asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f32 [%0], [%1], %2;"
                         ::"l"(a.G[2] + i3 * R), "r"(smem_u32(Xs + tid * kStageLd)), "r"((uint32_t)(R * 4))
                         : "memory");
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");   // Xs is read before the block ends
        }
    }
    __syncthreads();
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

template <bool BF16, int LOSS>
static cudaError_t run_tc(const DenseGradArgs<float>& a, int t1n, int t2n, int ntiles, int grid, size_t smem, int* err,
                          cudaStream_t st) {
    cudaFuncSetAttribute(k_dense3_tc<BF16, LOSS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_dense3_tc<BF16, LOSS><<<grid, kThreads, smem, st>>>(a, t1n, t2n, ntiles, err);
    return cudaGetLastError();
}

template <bool BF16>
static cudaError_t run_tc_loss(const DenseGradArgs<float>& a, int t1n, int t2n, int ntiles, int grid, size_t smem,
                               int* err, cudaStream_t st) {
    switch (a.loss) {
        case LOSS_GAUSSIAN: return run_tc<BF16, LOSS_GAUSSIAN>(a, t1n, t2n, ntiles, grid, smem, err, st);
        case LOSS_POISSON: return run_tc<BF16, LOSS_POISSON>(a, t1n, t2n, ntiles, grid, smem, err, st);
        case LOSS_ODDS: return run_tc<BF16, LOSS_ODDS>(a, t1n, t2n, ntiles, grid, smem, err, st);
        case LOSS_LOGIT: return run_tc<BF16, LOSS_LOGIT>(a, t1n, t2n, ntiles, grid, smem, err, st);
        default: return run_tc<BF16, LOSS_IDENTITY_X>(a, t1n, t2n, ntiles, grid, smem, err, st);
    }
}

}  // namespace

namespace {
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        cudaGetLastError();
    }
    return fn;
}

__global__ void k_write_map(unsigned long long* dst, const CUtensorMap m) {
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&m);
    if (threadIdx.x < sizeof(CUtensorMap) / 8) dst[threadIdx.x] = src[threadIdx.x];
}
}  // namespace

bool encode_x_map(void* map128, const float* X, int64_t I1, int64_t I2, int64_t I3) {
    if (I3 % 4 != 0 || (reinterpret_cast<uintptr_t>(X) & 15) != 0 || I1 > 0x7fffffff || I2 > 0x7fffffff ||
        I3 > 0x7fffffff)
        return false;
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)I3, (cuuint64_t)I2, (cuuint64_t)I1};
    const cuuint64_t strides[2] = {(cuuint64_t)I3 * 4, (cuuint64_t)I2 * I3 * 4};   // bytes, dims 1 and 2
    const cuuint32_t box[3] = {(cuuint32_t)kXBox, (cuuint32_t)kB2, (cuuint32_t)kB1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUtensorMap m;
    const CUresult r = fn(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(X), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    memcpy(map128, &m, sizeof(m));
    return true;
}

cudaError_t launch_write_map(void* dst_dev, const void* map128, cudaStream_t st, int64_t* launches) {
    CUtensorMap m;
    memcpy(&m, map128, sizeof(m));
    k_write_map<<<1, 32, 0, st>>>(reinterpret_cast<unsigned long long*>(dst_dev), m);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_dense_grad_tc(const DenseGradArgs<float>& a, bool bf16, int* err, cudaStream_t st,
                                 int64_t* launches) {
    if (a.ndim != 3 || a.R % 16 != 0 || a.R > 64) return cudaErrorInvalidValue;
    const int64_t I1 = a.dims[0], I2 = a.dims[1], I3 = a.dims[2];
    const int64_t nb3 = (I3 + kCols - 1) / kCols;
    const int64_t t1 = (I1 + kB1 - 1) / kB1, t2 = (I2 + kB2 - 1) / kB2;
    const int64_t ntiles = t1 * t2 * nb3;
    if (ntiles > 0x7fffffff || t1 > 0x7fffffff || t2 > 0x7fffffff) return cudaErrorInvalidValue;
    const int grid = (int)(ntiles < tc_num_sms() ? ntiles : tc_num_sms());
    const size_t smem = (size_t)tc_plan(a.R, bf16).total;
    if (launches) *launches += 1;
    if (grid <= 0) return cudaSuccess;
    return bf16 ? run_tc_loss<true>(a, (int)t1, (int)t2, (int)ntiles, grid, smem, err, st)
                : run_tc_loss<false>(a, (int)t1, (int)t2, (int)ntiles, grid, smem, err, st);
}

}  // namespace sgcp
