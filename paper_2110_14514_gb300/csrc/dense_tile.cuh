// Register-tiled dense GCP gradient of one box of a 3-way FP32 slice, run by
// one block of 256 threads: the fused model -> loss derivative -> all-mode
// MTTKRP of eq. gcp_grad_A (k = 1..3) and eq. gcp_grad_lambda, every entry
// of the box taken once with weight 1.
//
// A box is n1 x n2 tiles of 64 (i1, i2) rows (B1 = 2^lb1 values of i1 times
// B2 = 2^(6 - lb1) values of i2) that share one block of 32 i3 columns.  Per tile:
//   KR[row, j] = s_j A1[i1, j] A2[i2, j]        Khatri-Rao panel (both layouts in shared memory)
//   M  = KR . A3'                                model values (64 x 32)
//   Y  = df/dm(X, M)                             loss derivative (Sec. 2.2)
//   T  = Y . A3        -> G1[i1] += s * sum_i2 A2[i2] * T[(i1, i2)]
//                         G2[i2] += sum_i1 (s A1[i1]) * T[(i1, i2)]
//                         gs     += sum_(i1,i2) A1[i1] A2[i2] T[(i1, i2)]
//   G3 += Y' . KR                                (KR carries s)
// The three products run on one 16 x 16 thread grid; each keeps a 4 x 2,
// 4 x RT/16 or 2 x RT/16 register tile and reads its operands from k-major
// shared arrays, one 64- or 128-bit load per operand per k.  A 128-bit load
// takes four shared-memory wavefronts (one per quarter warp) even where lanes
// share addresses, so these tiles issue ~1.5 FMA instructions per wavefront:
// the products are bound by shared-memory wavefronts.  R is padded to RT in
// {16, 32, 48, 64} with zero columns (RT = 48: three single-word loads per
// operand row instead of one vector load).
#pragma once

#include "common.cuh"
#include "sgcp.h"

namespace sgcp {

constexpr int kBoxThreads = 256;
constexpr int kBoxMaxS = 32;   // largest box extent along i1 and along i2 (rows)

// Shared-memory plan (floats) of the box computation for padded rank RT.
template <int RT>
struct TileLayout {
    static constexpr int LDR = RT + 4;             // padded row stride of R-wide panels (16-byte rows)
    static constexpr int A3n = 0;                  // [32][LDR]   A3 rows of the i3 block
    static constexpr int A3t = A3n + 32 * LDR;     // [RT][32]
    static constexpr int KRn = A3t + RT * 32;      // [64][LDR]
    static constexpr int KRt = KRn + 64 * LDR;     // [RT][64]; then T as [64][LDR]
    static constexpr int LDY = 34;                 // Yn row stride: the 4 x 2 tiles' float2 stores hit 2 ways, not 8
    static constexpr int Yn = KRt + 64 * LDR;      // [64][LDY]
    static constexpr int Yt = Yn + 64 * LDY;       // [32][64]
    static constexpr int A1 = Yt + 32 * 64;        // [16][LDR]
    static constexpr int A1s = A1 + 16 * LDR;      // [16][LDR]
    static constexpr int A2 = A1s + 16 * LDR;      // [16][LDR]
    static constexpr int SV = A2 + 16 * LDR;       // [RT]
    static constexpr int ACC1 = SV + RT;           // [32][RT]
    static constexpr int ACC2 = ACC1 + kBoxMaxS * RT;   // [32][RT]
    static constexpr int GSB = ACC2 + kBoxMaxS * RT;    // [2][RT]: the box's gradient of s, per warp parity
    static constexpr int RED = GSB + 2 * RT;            // 8 doubles
    static constexpr int TOTAL = RED + 16;
    static_assert(RT * 64 <= 64 * LDR, "T fits the KRt region");
    static_assert(RED % 2 == 0 && A3t % 4 == 0 && KRn % 4 == 0 && KRt % 4 == 0 && Yn % 4 == 0 && Yt % 4 == 0 &&
                      A1 % 4 == 0 && A1s % 4 == 0 && A2 % 4 == 0 && GSB % 4 == 0,
                  "16-byte aligned regions");
};

struct BoxGeom {
    int R, loss;
    float eps;
    int I1, I2, I3;
    int lb1;              // B1 = 2^lb1 i1 rows per tile (2..4), B2 = 2^(6 - lb1)
    int n1, n2;           // tiles per box along i1 and i2 (B1 n1 <= 32, B2 n2 <= 32)
    int o1, o2, o3;       // box origin (i3 block of 32 columns)
    const float* A1;
    const float* A2;
    const float* A3;
    const float* s;
    const float* X;       // dense slice, C order
    float* G1;
    float* G2;
    float* G3;
    float* gs;
    double* f;
    float ysc;            // multiplies every y and f (1 unless a caller scales the loss)
};

template <int N>
__device__ __forceinline__ void lds_vec(float (&d)[N], const float* p);
template <>
__device__ __forceinline__ void lds_vec<1>(float (&d)[1], const float* p) {
    d[0] = *p;
}
template <>
__device__ __forceinline__ void lds_vec<3>(float (&d)[3], const float* p) {   // 4-byte aligned: three words
    d[0] = p[0];
    d[1] = p[1];
    d[2] = p[2];
}
template <>
__device__ __forceinline__ void lds_vec<2>(float (&d)[2], const float* p) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    d[0] = v.x;
    d[1] = v.y;
}
template <>
__device__ __forceinline__ void lds_vec<4>(float (&d)[4], const float* p) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    d[0] = v.x;
    d[1] = v.y;
    d[2] = v.z;
    d[3] = v.w;
}

template <int N>
__device__ __forceinline__ void sts_vec(float* p, const float (&d)[N]);
template <>
__device__ __forceinline__ void sts_vec<1>(float* p, const float (&d)[1]) {
    *p = d[0];
}
template <>
__device__ __forceinline__ void sts_vec<3>(float* p, const float (&d)[3]) {
    p[0] = d[0];
    p[1] = d[1];
    p[2] = d[2];
}
template <>
__device__ __forceinline__ void sts_vec<2>(float* p, const float (&d)[2]) {
    *reinterpret_cast<float2*>(p) = make_float2(d[0], d[1]);
}
template <>
__device__ __forceinline__ void sts_vec<4>(float* p, const float (&d)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(d[0], d[1], d[2], d[3]);
}

// Block-wide double sum of v (blockDim.x == kBoxThreads); result in thread 0.
__device__ __forceinline__ double box_block_sum(double v, double* red) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(SGCP_FULL_MASK, v, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kBoxThreads / 32; ++i) tot += red[i];
    return tot;
}

// want: SGCP_WANT_* bits (factor gradients, gradient of s, loss), any combination.
// Factor, s and slice reads go through L2 (ld.global.cg) for the factors and s,
// which a persistent caller may have rewritten from another SM, and through the
// read-only path for X, which no kernel writes while it is read.
//
// SPLIT (factor-gradient tiles): T and G3 run side by side on the two halves of
// the block instead of one after the other on all of it -- warps 0-3 form T on
// 8 x TN register tiles, warps 4-7 accumulate G3 on 4 x TN register tiles -- so
// the two products issue about 2.7 and 2 FMAs per shared-memory wavefront
// (8 x 4 / 12 and 4 x 4 / 8 at RT = 64) instead of 2 and 1.33; tiles without
// factor gradients keep the 256-thread T.
template <int RT, bool SPLIT = false>
__device__ void dense_box(const BoxGeom& g, int want, float* sm) {
    using L = TileLayout<RT>;
    constexpr int LDR = L::LDR;
    constexpr int TN = RT / 16;   // j values per thread in T and G3
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // 16 x 16 thread grid; a warp covers 8 x 4 of it, so per-k operand reads are contiguous
    const int g0 = (tid & 7) + 8 * (warp & 1);
    const int g1 = ((tid >> 3) & 3) + 4 * (warp >> 1);
    const int R = g.R;
    const int lb1 = g.lb1, lb2 = 6 - lb1, B1 = 1 << lb1, B2 = 1 << lb2;
    const int I1 = g.I1, I2 = g.I2, I3 = g.I3;
    float* A3n = sm + L::A3n;
    float* A3t = sm + L::A3t;
    float* KRn = sm + L::KRn;
    float* KRt = sm + L::KRt;
    float* Ts = sm + L::KRt;
    float* Yn = sm + L::Yn;
    float* Yt = sm + L::Yt;
    float* A1t = sm + L::A1;
    float* A1s = sm + L::A1s;
    float* A2t = sm + L::A2;
    float* sv = sm + L::SV;
    float* acc1 = sm + L::ACC1;
    float* acc2 = sm + L::ACC2;
    double* red = reinterpret_cast<double*>(sm + L::RED);
    const bool wantF = (want & SGCP_WANT_LOSS) != 0, wantS = (want & SGCP_WANT_TEMPORAL) != 0;
    const bool wantG = (want & SGCP_WANT_FACTORS) != 0, wantY = wantG || wantS;
    const float ysc = g.ysc;

    for (int i = tid; i < 32 * RT; i += kBoxThreads) {   // lanes along j: coalesced rows of A3
        const int c = i / RT, j = i - c * RT;
        A3n[c * LDR + j] = (j < R && g.o3 + c < I3) ? __ldcg(g.A3 + (int64_t)(g.o3 + c) * R + j) : 0.f;
    }
    float* gsb = sm + L::GSB;
    for (int j = tid; j < RT; j += kBoxThreads) sv[j] = j < R ? __ldcg(g.s + j) : 0.f;
    if (wantG)
        for (int i = tid; i < 2 * kBoxMaxS * RT; i += kBoxThreads) acc1[i] = 0.f;   // acc1, acc2 adjacent
    __syncthreads();
    for (int i = tid; i < 32 * RT; i += kBoxThreads) {   // lanes along c: conflict-free transposed stores
        const int j = i >> 5, c = i & 31;
        A3t[j * 32 + c] = A3n[c * LDR + j];
    }

    constexpr int G3C = SPLIT ? 4 : 2;   // i3 columns per thread in G3
    float g3[G3C][TN];
#pragma unroll
    for (int c = 0; c < G3C; ++c)
#pragma unroll
        for (int q = 0; q < TN; ++q) g3[c][q] = 0.f;
    float gsv[TN];   // this thread's share of the box's gradient of s, columns TN g1 ..
#pragma unroll
    for (int q = 0; q < TN; ++q) gsv[q] = 0.f;
    float fsum = 0.f;

    for (int t1 = 0; t1 < g.n1; ++t1) {
        const int i1b = g.o1 + t1 * B1;
        if (i1b >= I1) break;
        for (int t2 = 0; t2 < g.n2; ++t2) {
            const int i2b = g.o2 + t2 * B2;
            if (i2b >= I2) break;
            __syncthreads();   // the previous tile is done with every panel
            for (int i = tid; i < B1 * RT; i += kBoxThreads) {
                const int r = i / RT, j = i - r * RT;
                const float v = (j < R && i1b + r < I1) ? __ldcg(g.A1 + (int64_t)(i1b + r) * R + j) : 0.f;
                A1t[r * LDR + j] = v;
                A1s[r * LDR + j] = v * sv[j];
            }
            for (int i = tid; i < B2 * RT; i += kBoxThreads) {
                const int r = i / RT, j = i - r * RT;
                A2t[r * LDR + j] = (j < R && i2b + r < I2) ? __ldcg(g.A2 + (int64_t)(i2b + r) * R + j) : 0.f;
            }
            for (int i = tid; i < 64 * 32; i += kBoxThreads) {   // a warp reads 32 consecutive i3: 128 bytes
                const int row = i >> 5, col = i & 31;
                const int i1 = i1b + (row >> lb2), i2 = i2b + (row & (B2 - 1)), i3 = g.o3 + col;
                Yn[row * L::LDY + col] = (g.X && i1 < I1 && i2 < I2 && i3 < I3)
                                             ? __ldg(g.X + ((int64_t)i1 * I2 + i2) * I3 + i3)
                                             : 0.f;   // X == nullptr: the all-zero slice
            }
            __syncthreads();
            // Khatri-Rao panel, natural layout (lanes along j; only G3 reads it) and k-major layout
            // (lanes along rows)
            if (wantG)
                for (int i = tid; i < 64 * (RT / 4); i += kBoxThreads) {
                    const int row = i / (RT / 4), j0 = (i - row * (RT / 4)) * 4;
                    float a[4], b[4], p[4];
                    lds_vec<4>(a, A1s + (row >> lb2) * LDR + j0);
                    lds_vec<4>(b, A2t + (row & (B2 - 1)) * LDR + j0);
#pragma unroll
                    for (int q = 0; q < 4; ++q) p[q] = a[q] * b[q];
                    sts_vec<4>(KRn + row * LDR + j0, p);
                }
            for (int i = tid; i < RT * 16; i += kBoxThreads) {   // rows r0 .. r0 + 3 share one i1 (B2 >= 4)
                const int j = i >> 4, r0 = (i & 15) * 4;
                const float a = A1s[(r0 >> lb2) * LDR + j];
                const float* b = A2t + (r0 & (B2 - 1)) * LDR + j;
                float p[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) p[q] = a * b[q * LDR];
                sts_vec<4>(KRt + j * 64 + r0, p);
            }
            __syncthreads();
            // M = KR . A3' on rows 4 g0 .. 4 g0 + 3, columns 2 g1, 2 g1 + 1
            float m[4][2];
#pragma unroll
            for (int i = 0; i < 4; ++i) m[i][0] = m[i][1] = 0.f;
#pragma unroll 4
            for (int j = 0; j < RT; ++j) {
                float a[4], c[2];
                lds_vec<4>(a, KRt + j * 64 + 4 * g0);
                lds_vec<2>(c, A3t + j * 32 + 2 * g1);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    m[i][0] = fmaf(a[i], c[0], m[i][0]);
                    m[i][1] = fmaf(a[i], c[1], m[i][1]);
                }
            }
            float y[4][2];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int row = 4 * g0 + i, col = 2 * g1 + c;
                    const int i1 = i1b + (row >> lb2), i2 = i2b + (row & (B2 - 1)), i3 = g.o3 + col;
                    const bool valid = i1 < I1 && i2 < I2 && i3 < I3;
                    const float x = Yn[row * L::LDY + col];
                    if (wantF) {
                        float f, yy;
                        loss_eval<float>(g.loss, x, m[i][c], g.eps, f, yy);
                        if (valid) fsum += f * ysc;
                        y[i][c] = valid ? yy * ysc : 0.f;
                    } else {
                        y[i][c] = valid ? loss_dfdm<float>(g.loss, x, m[i][c], g.eps) * ysc : 0.f;
                    }
                }
            if (!wantY) continue;
            if (wantG)   // Y row-major: only G3 reads it
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float v[2] = {y[i][0], y[i][1]};
                    sts_vec<2>(Yn + (4 * g0 + i) * L::LDY + 2 * g1, v);
                }
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const float v[4] = {y[0][c], y[1][c], y[2][c], y[3][c]};
                sts_vec<4>(Yt + (2 * g1 + c) * 64 + 4 * g0, v);
            }
            __syncthreads();
            if (SPLIT && wantG) {
                if (warp < 4) {
                    // T = Y . A3 on rows 8 u0 .. 8 u0 + 7, j = TN u1 ..; a quarter warp covers two u0 and
                    // four u1, so its Yt and A3 vectors fall on distinct banks (one wavefront each)
                    const int u0 = 2 * (lane >> 3) + (lane & 1), u1 = 4 * warp + ((lane >> 1) & 3);
                    float tv[8][TN];
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int q = 0; q < TN; ++q) tv[i][q] = 0.f;
#pragma unroll 4
                    for (int c = 0; c < 32; ++c) {
                        float a[4], a2[4], b[TN];
                        lds_vec<4>(a, Yt + c * 64 + 8 * u0);
                        lds_vec<4>(a2, Yt + c * 64 + 8 * u0 + 4);
                        lds_vec<TN>(b, A3n + c * LDR + TN * u1);
#pragma unroll
                        for (int q = 0; q < TN; ++q) {
#pragma unroll
                            for (int i = 0; i < 4; ++i) tv[i][q] = fmaf(a[i], b[q], tv[i][q]);
#pragma unroll
                            for (int i = 0; i < 4; ++i) tv[4 + i][q] = fmaf(a2[i], b[q], tv[4 + i][q]);
                        }
                    }
                    if (wantS) {   // rows 8 u0 .. 8 u0 + 3 share one i1, rows 8 u0 + 4 .. + 7 another (B2 >= 4)
                        float a1lo[TN], a1hi[TN];
                        lds_vec<TN>(a1lo, A1t + ((8 * u0) >> lb2) * LDR + TN * u1);
                        lds_vec<TN>(a1hi, A1t + ((8 * u0 + 4) >> lb2) * LDR + TN * u1);
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            float a2[TN];
                            lds_vec<TN>(a2, A2t + ((8 * u0 + i) & (B2 - 1)) * LDR + TN * u1);
#pragma unroll
                            for (int q = 0; q < TN; ++q)
                                gsv[q] = fmaf((i < 4 ? a1lo[q] : a1hi[q]) * a2[q], tv[i][q], gsv[q]);
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 8; ++i) sts_vec<TN>(Ts + (8 * u0 + i) * LDR + TN * u1, tv[i]);   // KRt is free now
                } else {
                    // G3 += Y' . KR on columns 4 v0 .. 4 v0 + 3, j = TN v1 ..
                    const int v0 = lane & 7, v1 = 4 * (warp - 4) + (lane >> 3);
#pragma unroll 4
                    for (int r = 0; r < 64; ++r) {
                        float a[2], a2[2], b[TN];
                        lds_vec<2>(a, Yn + r * L::LDY + 4 * v0);
                        lds_vec<2>(a2, Yn + r * L::LDY + 4 * v0 + 2);
                        lds_vec<TN>(b, KRn + r * LDR + TN * v1);
#pragma unroll
                        for (int q = 0; q < TN; ++q) {
                            g3[0][q] = fmaf(a[0], b[q], g3[0][q]);
                            g3[1][q] = fmaf(a[1], b[q], g3[1][q]);
                            g3[G3C - 2][q] = fmaf(a2[0], b[q], g3[G3C - 2][q]);
                            g3[G3C - 1][q] = fmaf(a2[1], b[q], g3[G3C - 1][q]);
                        }
                    }
                }
            } else {
                // T = Y . A3 on rows 4 g0 .., j = TN g1 ..
                float tv[4][TN];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int q = 0; q < TN; ++q) tv[i][q] = 0.f;
#pragma unroll 4
                for (int c = 0; c < 32; ++c) {
                    float a[4], b[TN];
                    lds_vec<4>(a, Yt + c * 64 + 4 * g0);
                    lds_vec<TN>(b, A3n + c * LDR + TN * g1);
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int q = 0; q < TN; ++q) tv[i][q] = fmaf(a[i], b[q], tv[i][q]);
                }
                if (!SPLIT && wantG) {   // G3 += Y' . KR on columns 2 g0 .., j = TN g1 ..
#pragma unroll 4
                    for (int r = 0; r < 64; ++r) {
                        float a[2], b[TN];
                        lds_vec<2>(a, Yn + r * L::LDY + 2 * g0);
                        lds_vec<TN>(b, KRn + r * LDR + TN * g1);
#pragma unroll
                        for (int c = 0; c < 2; ++c)
#pragma unroll
                            for (int q = 0; q < TN; ++q) g3[c][q] = fmaf(a[c], b[q], g3[c][q]);
                    }
                }
                if (wantS) {   // g_s[j] += sum over this thread's rows of A1[i1][j] A2[i2][j] T[row][j]
                    const int row0 = 4 * g0, i1l = row0 >> lb2, i2l = row0 & (B2 - 1);   // B2 >= 4: one i1
                    float a1[TN];
                    lds_vec<TN>(a1, A1t + i1l * LDR + TN * g1);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        float a2[TN];
                        lds_vec<TN>(a2, A2t + (i2l + i) * LDR + TN * g1);
#pragma unroll
                        for (int q = 0; q < TN; ++q) gsv[q] = fmaf(a1[q] * a2[q], tv[i][q], gsv[q]);
                    }
                }
                if (!wantG) continue;
#pragma unroll
                for (int i = 0; i < 4; ++i) sts_vec<TN>(Ts + (4 * g0 + i) * LDR + TN * g1, tv[i]);   // KRt is free now
            }
            __syncthreads();
            {
                for (int i = tid; i < B1 * RT; i += kBoxThreads) {
                    const int il = i / RT, j = i - il * RT;
                    float acc = 0.f;
                    for (int i2l = 0; i2l < B2; ++i2l) acc = fmaf(A2t[i2l * LDR + j], Ts[(il * B2 + i2l) * LDR + j], acc);
                    acc1[(t1 * B1 + il) * RT + j] += sv[j] * acc;
                }
                for (int i = tid; i < B2 * RT; i += kBoxThreads) {
                    const int il = i / RT, j = i - il * RT;
                    float acc = 0.f;
                    for (int i1l = 0; i1l < B1; ++i1l) acc = fmaf(A1s[i1l * LDR + j], Ts[(i1l * B2 + il) * LDR + j], acc);
                    acc2[(t2 * B2 + il) * RT + j] += acc;
                }
            }
        }
    }
    __syncthreads();
    if (wantG) {   // the box's rows, four columns per 16-byte reduction (R % 4 == 0: rows stay 16-byte aligned)
        const int S1 = B1 * g.n1, S2 = B2 * g.n2, Q = R / 4;
        const bool vec = ((reinterpret_cast<uintptr_t>(g.G1) | reinterpret_cast<uintptr_t>(g.G2) |
                           reinterpret_cast<uintptr_t>(g.G3)) & 15) == 0;
        auto add4 = [&](float* dst, float4 v) {
            if (v.x == 0.f && v.y == 0.f && v.z == 0.f && v.w == 0.f) return;
            if (vec) {
                red_add_f4(dst, v);
            } else {
                atomicAdd(dst, v.x), atomicAdd(dst + 1, v.y), atomicAdd(dst + 2, v.z), atomicAdd(dst + 3, v.w);
            }
        };
        for (int i = tid; i < S1 * Q; i += kBoxThreads) {
            const int r = i / Q, j = 4 * (i - r * Q);
            if (g.o1 + r < I1) add4(g.G1 + (int64_t)(g.o1 + r) * R + j, *reinterpret_cast<const float4*>(acc1 + r * RT + j));
        }
        for (int i = tid; i < S2 * Q; i += kBoxThreads) {
            const int r = i / Q, j = 4 * (i - r * Q);
            if (g.o2 + r < I2) add4(g.G2 + (int64_t)(g.o2 + r) * R + j, *reinterpret_cast<const float4*>(acc2 + r * RT + j));
        }
        // G3 rows of this thread: 2 g0 .. (256-thread G3) or, in the split, 4 v0 .. on warps 4-7
        const bool g3_mine = !SPLIT || warp >= 4;
        const int c0 = SPLIT ? 4 * (lane & 7) : 2 * g0;
        const int j = SPLIT ? TN * (4 * (warp - 4) + (lane >> 3)) : TN * g1;   // TN consecutive columns
#pragma unroll
        for (int c = 0; c < G3C; ++c) {
            const int i3 = g.o3 + c0 + c;
            if (!g3_mine || i3 >= I3) continue;
            if constexpr (TN == 4) {
                if (j < R) add4(g.G3 + (int64_t)i3 * R + j, make_float4(g3[c][0], g3[c][1], g3[c][2], g3[c][3]));
            } else {
#pragma unroll
                for (int q = 0; q < TN; ++q)
                    if (j + q < R && g3[c][q] != 0.f) atomicAdd(g.G3 + (int64_t)i3 * R + j + q, g3[c][q]);
            }
        }
    }
    if (wantS) {
        // 256-thread T: over the 16 row groups g0 (8 lanes of a warp, then the warp pair warp & 1);
        // split T: over the 8 row groups u0 of a warp (lane bits 0, 3 and 4), warps 0-3 only
        const bool split = SPLIT && wantG;
#pragma unroll
        for (int q = 0; q < TN; ++q) {
            float v = gsv[q];
            if (split) {
                v += __shfl_xor_sync(SGCP_FULL_MASK, v, 1);
                v += __shfl_xor_sync(SGCP_FULL_MASK, v, 8);
                v += __shfl_xor_sync(SGCP_FULL_MASK, v, 16);
                if (warp < 4 && (lane & 0x19) == 0) gsb[TN * (4 * warp + ((lane >> 1) & 3)) + q] = v;
            } else {
                v += __shfl_xor_sync(SGCP_FULL_MASK, v, 1);
                v += __shfl_xor_sync(SGCP_FULL_MASK, v, 2);
                v += __shfl_xor_sync(SGCP_FULL_MASK, v, 4);
                if ((tid & 7) == 0) gsb[(warp & 1) * RT + TN * g1 + q] = v;
            }
        }
        __syncthreads();
        if (tid < R) {
            const float v = gsb[tid] + (split ? 0.f : gsb[RT + tid]);
            if (v != 0.f) atomicAdd(g.gs + tid, v);
        }
    }
    if (wantF) {
        const double tot = box_block_sum((double)fsum, red);
        if (tid == 0 && tot != 0.0) atomicAdd(g.f, tot);
    }
}

// Padded rank for R (R <= 64, R % 4 == 0).
__host__ __device__ inline int box_rt(int R) { return R <= 16 ? 16 : (R <= 32 ? 32 : (R <= 48 ? 48 : 64)); }

// Dispatch on the padded rank.
template <bool SPLIT = false>
__device__ __forceinline__ void dense_box_any(const BoxGeom& g, int want, float* sm) {
    if (g.R <= 16) dense_box<16, SPLIT>(g, want, sm);
    else if (g.R <= 32) dense_box<32, SPLIT>(g, want, sm);
    else if (g.R <= 48) dense_box<48, SPLIT>(g, want, sm);
    else dense_box<64, SPLIT>(g, want, sm);
}

constexpr int kBoxSmemFloats = TileLayout<64>::TOTAL;

}  // namespace sgcp
