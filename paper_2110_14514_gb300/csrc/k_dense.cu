// Dense-slice fused GCP gradient on CUDA cores (FP32 / FP64), every entry of
// the slice taken once with weight 1 (exact gradient and loss).
//
// Algebra (3-way, slice X of I1 x I2 x I3 in C order; 2-way slices run with a
// unit middle mode whose factor is all ones):  for a tile of 32 (i1,i2) rows
// x 32 i3 columns,
//   KR[(i1,i2), j] = s_j A1[i1,j] A2[i2,j]                (Khatri-Rao panel in shared memory)
//   M  = KR . A3'                                        (model values, eq. CP_model)
//   Y  = df/dm(X, M)                                     (Sec. 2.2)
//   T  = Y . A3          -> G1[i1] += s * sum_i2 A2[i2] * T[(i1,i2)]
//                           G2[i2] += sum_i1 (s*A1[i1]) * T[(i1,i2)]
//                           gs     += sum_(i1,i2) A1[i1] * A2[i2] * T[(i1,i2)]
//   G3 += Y' . KR
// which is eq. gcp_grad_A for k = 1..3 and eq. gcp_grad_lambda, with the
// partial contraction T shared by modes 1 and 2 (6R flops per entry instead
// of 8R).  A block walks a sub-box of n1 x n2 tiles that share one i3 block,
// keeps the sub-box's G rows in shared memory / registers and adds them to
// global memory once, so the global atomics per entry are
// (S1 + S2 + 32) R / (S1 S2 32).
#include "dense_tile.cuh"
#include "internal.h"
#include "sgcp.h"

namespace sgcp {

// FP32 3-way slices with R <= 64 run the register-tiled box of dense_tile.cuh:
// one block per box of n1 x n2 tiles of 64 (i1, i2) rows sharing 32 i3 columns.
template <int RT>
__global__ void __launch_bounds__(kBoxThreads, 2) k_dense3_box(const DenseGradArgs<float> a, int lb1, int n1, int n2,
                                                                int nb1, int nb2) {
    extern __shared__ __align__(16) float box_sm[];
    if (a.skip && *a.skip) return;
    const int bid = blockIdx.x;
    const int b3 = bid / (nb1 * nb2), rem = bid - b3 * nb1 * nb2;
    const int bb1 = rem / nb2, bb2 = rem - bb1 * nb2;
    const int R = a.R;
    BoxGeom g;
    g.R = R;
    g.loss = a.loss;
    g.eps = a.eps;
    g.I1 = (int)a.dims[0];
    g.I2 = (int)a.dims[1];
    g.I3 = (int)a.dims[2];
    g.lb1 = lb1;
    g.n1 = n1;
    g.n2 = n2;
    g.o1 = bb1 * (1 << lb1) * n1;
    g.o2 = bb2 * (64 >> lb1) * n2;
    g.o3 = b3 * 32;
    g.A1 = a.A[0];
    g.A2 = a.A[1];
    g.A3 = a.A[2];
    g.s = a.s;
    g.X = reinterpret_cast<const float*>(a.slice ? a.slice->vals : a.inline_slice.vals);
    g.G1 = a.G[0];
    g.G2 = a.G[1];
    g.G3 = a.G[2];
    g.gs = a.gs;
    g.f = a.f;
    g.ysc = a.y_scale ? *a.y_scale : 1.0f;
    dense_box<RT, true>(g, a.want, box_sm);
    if (a.tstep_on && last_block_ticket(a.tstep.st)) temporal_step_tail<float>(a.tstep, a.gs, R);
}

static int box_num_sms();

template <int RT>
static cudaError_t run_box(const DenseGradArgs<float>& a, cudaStream_t st) {
    const int64_t I1 = a.dims[0], I2 = a.dims[1], I3 = a.dims[2];
    const int lb1 = 3;                      // 8 i1 x 8 i2 rows per tile
    const int64_t nb3 = (I3 + 31) / 32;
    // the largest boxes (fewest G1 / G2 reductions) that still give six blocks per SM (three
    // waves of two): measured at 256^3, R = 64, boxes of 8 x 4 tiles' rows (1024 blocks) ran the
    // factor gradient in 320 us against 347 us for 32 x 32 rows (512 blocks) and 379 us for 8 x 8
    int n1 = 1, n2 = 1;
    auto nblocks = [&](int m1, int m2) { return ((I1 + 8 * m1 - 1) / (8 * m1)) * ((I2 + 8 * m2 - 1) / (8 * m2)) * nb3; };
    const int64_t target = 6 * box_num_sms();
    for (;;) {
        bool grew = false;
        if (8 * n1 * 2 <= kBoxMaxS && 8 * n1 < I1 && nblocks(n1 * 2, n2) >= target) { n1 *= 2; grew = true; }
        if (8 * n2 * 2 <= kBoxMaxS && 8 * n2 < I2 && nblocks(n1, n2 * 2) >= target) { n2 *= 2; grew = true; }
        if (!grew) break;
    }
    const int nb1 = (int)((I1 + 8 * n1 - 1) / (8 * n1)), nb2 = (int)((I2 + 8 * n2 - 1) / (8 * n2));
    const int64_t blocks = (int64_t)nb1 * nb2 * nb3;
    if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
    const size_t smem = (size_t)TileLayout<RT>::TOTAL * sizeof(float);
    cudaFuncSetAttribute(k_dense3_box<RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_dense3_box<RT><<<(unsigned)blocks, kBoxThreads, smem, st>>>(a, lb1, n1, n2, nb1, nb2);
    return cudaGetLastError();
}

template <typename T, int B1, int B2, int RMAX>
struct DenseCfg {
    static constexpr int TR = B1 * B2;   // 32 rows per tile
    static constexpr int TC = 32;        // i3 columns per tile
    static constexpr int LD = RMAX + 1;  // padded leading dimension of R-wide panels
    static constexpr int NC = (RMAX + 15) / 16;   // columns j per thread in the T / G3 products
};

template <typename T, int B1, int B2, int RMAX>
__global__ void __launch_bounds__(256) k_dense3(const DenseGradArgs<T> a, int n1, int n2, int nb1, int nb2) {
    using C = DenseCfg<T, B1, B2, RMAX>;
    static_assert(B1 * B2 == 32, "tile rows");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (a.skip && *a.skip) return;
    const int R = a.R;
    const int S1 = B1 * n1, S2 = B2 * n2;
    T* A3s = reinterpret_cast<T*>(smem_raw);          // [32][LD]
    T* KR = A3s + C::TC * C::LD;                      // [32][LD]
    T* Ts = KR + C::TR * C::LD;                       // [32][LD]
    T* Ys = Ts + C::TR * C::LD;                       // [32][33]
    T* A1t = Ys + C::TR * 33;                         // [B1][RMAX]
    T* A1st = A1t + B1 * RMAX;                        // [B1][RMAX]
    T* A2t = A1st + B1 * RMAX;                        // [B2][RMAX]
    T* sv = A2t + B2 * RMAX;                          // [RMAX]
    T* acc1 = sv + RMAX;                              // [S1][RMAX]
    T* acc2 = acc1 + S1 * RMAX;                       // [S2][RMAX]
    double* fred = reinterpret_cast<double*>(acc2 + S2 * RMAX);   // float offset is even: 8-byte aligned

    const int64_t I1 = a.dims[0], I2 = a.dims[1], I3 = a.dims[2];
    const bool dummy2 = (a.ndim == 2);   // 2-way slice: middle mode of size 1, factor all ones
    const int bid = blockIdx.x;
    const int b3 = bid / (nb1 * nb2), rem = bid - b3 * nb1 * nb2;
    const int bb1 = rem / nb2, bb2 = rem - bb1 * nb2;
    const int64_t o1 = (int64_t)bb1 * S1, o2 = (int64_t)bb2 * S2, o3 = (int64_t)b3 * C::TC;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const bool wantG = (a.want & SGCP_WANT_FACTORS) != 0;
    const bool wantS = (a.want & SGCP_WANT_TEMPORAL) != 0;
    const bool wantF = (a.want & SGCP_WANT_LOSS) != 0;
    const T ysc = a.y_scale ? *a.y_scale : T(1);
    const T* X = reinterpret_cast<const T*>(a.slice ? a.slice->vals : a.inline_slice.vals);

    for (int i = tid; i < C::TC * C::LD; i += 256) {
        const int r = i / C::LD, j = i - r * C::LD;
        A3s[i] = (j < R && o3 + r < I3) ? a.A[2][(o3 + r) * R + j] : T(0);
    }
    for (int j = tid; j < RMAX; j += 256) sv[j] = j < R ? a.s[j] : T(0);
    for (int i = tid; i < (S1 + S2) * RMAX; i += 256) acc1[i] = T(0);

    T g3[2][C::NC];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < C::NC; ++c) g3[r][c] = T(0);
    T gsr = T(0);     // thread tid < R owns gs[tid]
    T fsum = T(0);    // per-thread loss partial; reduced in double below

    for (int t1 = 0; t1 < n1; ++t1) {
        const int64_t i1b = o1 + (int64_t)t1 * B1;
        if (i1b >= I1) break;
        for (int t2 = 0; t2 < n2; ++t2) {
            const int64_t i2b = o2 + (int64_t)t2 * B2;
            if (i2b >= I2) break;
            __syncthreads();   // previous tile done with the panels
            for (int i = tid; i < B1 * RMAX; i += 256) {
                const int r = i / RMAX, j = i - r * RMAX;
                const T v = (j < R && i1b + r < I1) ? a.A[0][(i1b + r) * R + j] : T(0);
                A1t[i] = v;
                A1st[i] = v * sv[j];
            }
            for (int i = tid; i < B2 * RMAX; i += 256) {
                const int r = i / RMAX, j = i - r * RMAX;
                A2t[i] = (j < R && i2b + r < I2) ? (dummy2 ? T(1) : a.A[1][(i2b + r) * R + j]) : T(0);
            }
            for (int i = tid; i < C::TR * C::TC; i += 256) {
                const int row = i >> 5, col = i & 31;
                const int64_t i1 = i1b + row / B2, i2 = i2b + row % B2, i3 = o3 + col;
                Ys[row * 33 + col] = (X && i1 < I1 && i2 < I2 && i3 < I3) ? X[(i1 * I2 + i2) * I3 + i3] : T(0);
            }
            __syncthreads();
            for (int i = tid; i < C::TR * RMAX; i += 256) {
                const int row = i / RMAX, j = i - row * RMAX;
                KR[row * C::LD + j] = A1st[(row / B2) * RMAX + j] * A2t[(row % B2) * RMAX + j];
            }
            __syncthreads();
            // M and Y: thread owns rows {ty, ty+16} x cols {tx, tx+16}
            {
                T m[2][2] = {{T(0), T(0)}, {T(0), T(0)}};
                for (int j = 0; j < R; ++j) {
                    const T k0 = KR[ty * C::LD + j], k1 = KR[(ty + 16) * C::LD + j];
                    const T c0 = A3s[tx * C::LD + j], c1 = A3s[(tx + 16) * C::LD + j];
                    m[0][0] += k0 * c0;
                    m[0][1] += k0 * c1;
                    m[1][0] += k1 * c0;
                    m[1][1] += k1 * c1;
                }
#pragma unroll
                for (int rr = 0; rr < 2; ++rr)
#pragma unroll
                    for (int cc = 0; cc < 2; ++cc) {
                        const int row = ty + 16 * rr, col = tx + 16 * cc;
                        const int64_t i1 = i1b + row / B2, i2 = i2b + row % B2, i3 = o3 + col;
                        const bool valid = i1 < I1 && i2 < I2 && i3 < I3;
                        T f, y;
                        loss_eval<T>(a.loss, Ys[row * 33 + col], m[rr][cc], a.eps, f, y);
                        if (valid && wantF) fsum += f * ysc;
                        Ys[row * 33 + col] = valid ? y * ysc : T(0);
                    }
            }
            __syncthreads();
            if (wantG || wantS) {
                // T = Y . A3 (rows {ty, ty+16}, cols tx + 16c) and G3 += Y' . KR
                T tv[2][C::NC];
#pragma unroll
                for (int r = 0; r < 2; ++r)
#pragma unroll
                    for (int c = 0; c < C::NC; ++c) tv[r][c] = T(0);
                for (int k = 0; k < 32; ++k) {
                    const T y0 = Ys[ty * 33 + k], y1 = Ys[(ty + 16) * 33 + k];
                    const T z0 = Ys[k * 33 + ty], z1 = Ys[k * 33 + ty + 16];
#pragma unroll
                    for (int c = 0; c < C::NC; ++c) {
                        const int j = tx + 16 * c;
                        const T a3 = A3s[k * C::LD + j];
                        const T kr = KR[k * C::LD + j];
                        tv[0][c] += y0 * a3;
                        tv[1][c] += y1 * a3;
                        g3[0][c] += z0 * kr;
                        g3[1][c] += z1 * kr;
                    }
                }
#pragma unroll
                for (int r = 0; r < 2; ++r)
#pragma unroll
                    for (int c = 0; c < C::NC; ++c) Ts[(ty + 16 * r) * C::LD + tx + 16 * c] = tv[r][c];
                __syncthreads();
                if (wantG) {
                    for (int i = tid; i < B1 * R; i += 256) {
                        const int il = i / R, j = i - il * R;
                        T acc = T(0);
#pragma unroll
                        for (int i2l = 0; i2l < B2; ++i2l) acc += A2t[i2l * RMAX + j] * Ts[(il * B2 + i2l) * C::LD + j];
                        acc1[(t1 * B1 + il) * RMAX + j] += sv[j] * acc;
                    }
                    if (!dummy2) {
                        for (int i = tid; i < B2 * R; i += 256) {
                            const int il = i / R, j = i - il * R;
                            T acc = T(0);
#pragma unroll
                            for (int i1l = 0; i1l < B1; ++i1l) acc += A1st[i1l * RMAX + j] * Ts[(i1l * B2 + il) * C::LD + j];
                            acc2[(t2 * B2 + il) * RMAX + j] += acc;
                        }
                    }
                }
                if (wantS && tid < R) {
                    T acc = T(0);
                    for (int row = 0; row < C::TR; ++row)
                        acc += A1t[(row / B2) * RMAX + tid] * A2t[(row % B2) * RMAX + tid] * Ts[row * C::LD + tid];
                    gsr += acc;
                }
            }
        }
    }
    __syncthreads();
    if (wantG) {
        for (int i = tid; i < S1 * R; i += 256) {
            const int r = i / R, j = i - r * R;
            const T v = acc1[r * RMAX + j];
            if (o1 + r < I1 && v != T(0)) atomicAdd(a.G[0] + (o1 + r) * R + j, v);
        }
        if (!dummy2) {
            for (int i = tid; i < S2 * R; i += 256) {
                const int r = i / R, j = i - r * R;
                const T v = acc2[r * RMAX + j];
                if (o2 + r < I2 && v != T(0)) atomicAdd(a.G[1] + (o2 + r) * R + j, v);
            }
        }
        T* G3 = dummy2 ? a.G[1] : a.G[2];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < C::NC; ++c) {
                const int64_t i3 = o3 + ty + 16 * r;
                const int j = tx + 16 * c;
                if (i3 < I3 && j < R && g3[r][c] != T(0)) atomicAdd(G3 + i3 * R + j, g3[r][c]);  // KR carries s
            }
    }
    if (wantS && tid < R && gsr != T(0)) atomicAdd(a.gs + tid, gsr);
    if (wantF) {
        double fd = (double)fsum;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) fd += __shfl_xor_sync(SGCP_FULL_MASK, fd, off);
        if ((tid & 31) == 0) fred[tid >> 5] = fd;
        __syncthreads();
        if (tid == 0) {
            double tot = 0.0;
            for (int i = 0; i < 8; ++i) tot += fred[i];
            if (tot != 0.0) atomicAdd(a.f, tot);
        }
    }
    // temporal solver: the last block applies the ADAM step to s (Alg. 3)
    if (a.tstep_on && last_block_ticket(a.tstep.st)) temporal_step_tail<T>(a.tstep, a.gs, R);
}

static int dense_num_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

template <typename T, int B1, int B2, int RMAX>
static cudaError_t run_dense(const DenseGradArgs<T>& a, cudaStream_t st) {
    using C = DenseCfg<T, B1, B2, RMAX>;
    const int64_t I1 = a.dims[0], I2 = a.dims[1], I3 = a.dims[2];
    const int64_t nb3 = (I3 + C::TC - 1) / C::TC;
    // Choose the sub-box (S1 = B1 n1, S2 = B2 n2): as large as possible (fewer
    // global atomics) while keeping at least two blocks per SM busy.
    const int maxS = (RMAX >= 128 || sizeof(T) == 8) ? 16 : 32;
    int n1 = 1, n2 = 1;
    auto nblocks = [&](int m1, int m2) {
        return ((I1 + B1 * m1 - 1) / (B1 * m1)) * ((I2 + B2 * m2 - 1) / (B2 * m2)) * nb3;
    };
    const int64_t target = 2 * dense_num_sms();
    for (;;) {
        bool grew = false;
        if (B1 * n1 * 2 <= maxS && B1 * n1 < I1 && nblocks(n1 * 2, n2) >= target) { n1 *= 2; grew = true; }
        if (B2 * n2 * 2 <= maxS && B2 * n2 < I2 && nblocks(n1, n2 * 2) >= target) { n2 *= 2; grew = true; }
        if (!grew) break;
    }
    const int S1 = B1 * n1, S2 = B2 * n2;
    const int nb1 = (int)((I1 + S1 - 1) / S1), nb2 = (int)((I2 + S2 - 1) / S2);
    const int64_t blocks = (int64_t)nb1 * nb2 * nb3;
    const size_t elems = (size_t)C::TC * C::LD + 2 * (size_t)C::TR * C::LD + (size_t)C::TR * 33 +
                         (size_t)(2 * B1 + B2 + 1) * RMAX + (size_t)(S1 + S2) * RMAX + 2;
    const size_t smem = elems * sizeof(T) + 8 * sizeof(double) + 16;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_dense3<T, B1, B2, RMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
    k_dense3<T, B1, B2, RMAX><<<(unsigned)blocks, 256, smem, st>>>(a, n1, n2, nb1, nb2);
    return cudaGetLastError();
}

template <typename T, int B1, int B2>
static cudaError_t dense_rank(const DenseGradArgs<T>& a, cudaStream_t st) {
    if (a.R <= 16) return run_dense<T, B1, B2, 16>(a, st);
    if (a.R <= 32) return run_dense<T, B1, B2, 32>(a, st);
    if (a.R <= 64) return run_dense<T, B1, B2, 64>(a, st);
    return cudaErrorInvalidValue;
}

static int box_num_sms() { return dense_num_sms(); }

template <typename T>
static bool dense_box_path(const DenseGradArgs<T>&, cudaStream_t, cudaError_t*) {
    return false;
}
template <>
bool dense_box_path<float>(const DenseGradArgs<float>& a, cudaStream_t st, cudaError_t* e) {
    if (a.ndim != 3 || a.R > 64) return false;
    *e = a.R <= 16 ? run_box<16>(a, st)
                   : (a.R <= 32 ? run_box<32>(a, st) : (a.R <= 48 ? run_box<48>(a, st) : run_box<64>(a, st)));
    return true;
}

template <typename T>
cudaError_t launch_dense_grad(const DenseGradArgs<T>& a, cudaStream_t st, int64_t* launches) {
    if (launches) *launches += 1;
    {
        cudaError_t e = cudaSuccess;
        if (dense_box_path<T>(a, st, &e)) return e;
    }
    if (a.ndim == 2) {
        // (I1, I2) viewed as (I1, 1, I2): rows are i1 only, columns i2.
        DenseGradArgs<T> b = a;
        b.dims[2] = a.dims[1];
        b.dims[1] = 1;
        b.A[2] = a.A[1];
        b.A[1] = nullptr;
        b.G[2] = nullptr;
        return dense_rank<T, 32, 1>(b, st);
    }
    if (a.ndim == 3) return dense_rank<T, 4, 8>(a, st);
    return cudaErrorInvalidValue;
}

template cudaError_t launch_dense_grad<float>(const DenseGradArgs<float>&, cudaStream_t, int64_t*);
template cudaError_t launch_dense_grad<double>(const DenseGradArgs<double>&, cudaStream_t, int64_t*);

}  // namespace sgcp
