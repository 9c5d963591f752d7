// Solver kernels of OnlineGCP (arXiv 2110.14514 Sec. 4.2-4.4): Gram matrices,
// history-penalty coefficients, the fused history + regularisation + ADAM row
// update of the factor matrices (eq. spatial_gcp_grad, Alg. 2, Alg. 4), the
// temporal-weight ADAM step (Alg. 3), per-epoch accept / rollback, the
// objective's history and regularisation terms (Alg. 5), the history weight
// matrix S_H and the Gaussian least-squares temporal solve (Sec. 5).
//
// History algebra used here.  With Gamma_k = *_{n != k} A^(n)'A^(n),
// Gammabar_k = *_{n != k} Abar^(n)'A^(n) and S_H = sum_h w_h s_h s_h', the
// per-h loop of eq. spatial_gcp_grad collapses because
// diag(s_h) B diag(s_h) = B * (s_h s_h'):
//   sum_h w_h (A Gamma_h-term - Abar Gammabar_h-term)
//     = A (Gamma_k * S_H) - Abar (Gammabar_k * S_H)
//     = D (Gamma_k * S_H) + Abar ((Gamma_k - Gammabar_k) * S_H),   D = A - Abar,
// and Gamma_k - Gammabar_k is summed from differences E_n = D^(n)'A^(n)
// (telescoping over the Hadamard factors) so nothing cancels when A ~ Abar.
#include <type_traits>

#include <cooperative_groups.h>

#include "internal.h"
#include "sgcp.h"

namespace cg = cooperative_groups;

namespace sgcp {

// ---------------------------------------------------------------------------
// Gram matrices Gram(U, V)[l][m] = sum_r U[r][l] V[r][m], U, V in {A, Abar, D}.
// grid = (blocks per mode, ndim, npairs).  Each block writes the partial sum
// over its rows (element type T); k_gram_reduce adds the partials in double.
// No atomics, so results do not depend on scheduling.
// ---------------------------------------------------------------------------
constexpr int kGramStage = 32;   // rows staged in shared memory at a time
constexpr int kGramMaxBlocks = 512;

void gram_geometry(int64_t max_dim, int* nblk, int64_t* rows_per_block) {
    int64_t rpb = 64;
    int64_t nb = (max_dim + rpb - 1) / rpb;
    if (nb > kGramMaxBlocks) {
        nb = kGramMaxBlocks;
        rpb = (max_dim + nb - 1) / nb;
        rpb = (rpb + kGramStage - 1) / kGramStage * kGramStage;
        nb = (max_dim + rpb - 1) / rpb;
    }
    *nblk = (int)(nb < 1 ? 1 : nb);
    *rows_per_block = rpb;
}

template <typename T, int TPT>
__global__ void __launch_bounds__(256) k_gram(const GramArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (a.skip && *a.skip) return;
    const int k = blockIdx.y, pr = blockIdx.z, R = a.R;
    const int64_t I = a.dims[k];
    const int64_t r0 = (int64_t)blockIdx.x * a.rows_per_block;
    if (r0 >= I) return;
    const int64_t r1 = min(r0 + a.rows_per_block, I);
    const T* A = a.A + a.row_off[k] * R;
    const T* Ab = a.Abar + a.row_off[k] * R;
    const int su = a.sel_u[pr], svv = a.sel_v[pr];
    T* Us = reinterpret_cast<T*>(smem_raw);          // [stage][R]
    T* Vs = Us + kGramStage * R;                      // [stage][R]
    T* red = Vs + kGramStage * R;                     // [groups][R*R]
    const int tq = R / 4;                 // 4x4 output tiles per dimension
    const int tiles = tq * tq;
    const int tpg = tiles >= 256 ? 256 : tiles;       // threads per row group
    const int groups = 256 / tpg;
    const int tid = threadIdx.x;
    const int grp = tid / tpg;
    T acc[TPT][4][4];
#pragma unroll
    for (int t = 0; t < TPT; ++t)
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[t][x][y] = T(0);
    for (int64_t base = r0; base < r1; base += kGramStage) {
        const int nr = (int)min((int64_t)kGramStage, r1 - base);
        __syncthreads();
        for (int i = tid; i < nr * R; i += blockDim.x) {
            Us[i] = gsel(su, A, Ab, base * R + i);
            Vs[i] = gsel(svv, A, Ab, base * R + i);
        }
        __syncthreads();
        if (grp < groups) {
#pragma unroll
            for (int t = 0; t < TPT; ++t) {
                const int tile = (tiles >= 256) ? tid + 256 * t : tid % tiles;
                if (tile >= tiles) continue;
                const int tl = tile / tq, tm = tile % tq;
                for (int r = grp; r < nr; r += groups) {
                    T u[4], v[4];
#pragma unroll
                    for (int x = 0; x < 4; ++x) {
                        u[x] = Us[r * R + tl * 4 + x];
                        v[x] = Vs[r * R + tm * 4 + x];
                    }
#pragma unroll
                    for (int x = 0; x < 4; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) acc[t][x][y] += u[x] * v[y];
                }
            }
        }
    }
    __syncthreads();
    for (int i = tid; i < groups * R * R; i += blockDim.x) red[i] = T(0);
    __syncthreads();
    if (grp < groups) {
#pragma unroll
        for (int t = 0; t < TPT; ++t) {
            const int tile = (tiles >= 256) ? tid + 256 * t : tid % tiles;
            if (tile >= tiles) continue;
            const int tl = tile / tq, tm = tile % tq;
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) red[grp * R * R + (tl * 4 + x) * R + tm * 4 + y] = acc[t][x][y];
        }
    }
    __syncthreads();
    T* out = a.part + (((int64_t)pr * a.ndim + k) * a.nblk + blockIdx.x) * R * R;
    for (int i = tid; i < R * R; i += blockDim.x) {
        T sum = T(0);
        for (int g = 0; g < groups; ++g) sum += red[g * R * R + i];
        out[i] = sum;
    }
}

// grams[p][k][i] = sum over the blocks of mode k of the partials: one warp
// per output, lanes stride over the partials, double accumulation.
template <typename T>
__global__ void k_gram_reduce(const GramArgs<T> a) {
    if (a.skip && *a.skip) return;
    const int k = blockIdx.y, pr = blockIdx.z, RR = a.R * a.R;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= RR) return;
    const int nb = (int)((a.dims[k] + a.rows_per_block - 1) / a.rows_per_block);
    const T* part = a.part + ((int64_t)pr * a.ndim + k) * a.nblk * RR + i;
    T sum = T(0);
    for (int b = lane; b < nb; b += 32) sum += part[(int64_t)b * RR];
    double ds = (double)sum;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ds += __shfl_xor_sync(SGCP_FULL_MASK, ds, off);
    if (lane == 0) a.out[((int64_t)pr * a.ndim + k) * RR + i] = ds;
}

template <typename T>
cudaError_t launch_gram(const GramArgs<T>& a, int64_t, cudaStream_t st, int64_t* launches) {
    const int tiles = (a.R / 4) * (a.R / 4);
    const int groups = tiles >= 256 ? 1 : 256 / tiles;
    const size_t smem = 2 * kGramStage * a.R * sizeof(T) + (size_t)groups * a.R * a.R * sizeof(T);
    dim3 grid((unsigned)a.nblk, a.ndim, a.npairs);
    if (tiles <= 256) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_gram<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_gram<T, 1><<<grid, 256, smem, st>>>(a);
    } else {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_gram<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_gram<T, 4><<<grid, 256, smem, st>>>(a);
    }
    dim3 rgrid((unsigned)((a.R * a.R + 7) / 8), a.ndim, a.npairs);
    k_gram_reduce<T><<<rgrid, 256, 0, st>>>(a);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// B_k = Gamma_k * S_H and C_k = (Gamma_k - Gammabar_k) * S_H  (float outputs)
// grams = [pairs][ndim][R][R]: P_n = A'A at pair 0, E_n = D'A at pair e_pair.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_hist_coeffs(int ndim, int R, const double* grams, int e_pair, const double* SH,
                              const int32_t* hist_len, T* B, T* C, const int32_t* skip) {
    if (skip && *skip) return;
    const int RR = R * R;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= RR) return;
    hist_coeff_elem<T>(ndim, RR, grams, grams + (int64_t)e_pair * ndim * RR, SH, i, *hist_len > 0, B, C);
}

template <typename T>
cudaError_t launch_hist_coeffs(int ndim, int R, const double* grams, int e_pair, const double* SH,
                               const int32_t* hist_len, T* B, T* C, const int32_t* skip, cudaStream_t st,
                               int64_t* launches) {
    k_hist_coeffs<T><<<(R * R + 127) / 128, 128, 0, st>>>(ndim, R, grams, e_pair, SH, hist_len, B, C, skip);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Factor row update: g = G + lambda a + d B_k + abar C_k; ADAM step (Alg. 2)
// with the bias-corrected rate of iteration i (written by k_epoch_begin);
// projection a <- max(a, l); G <- 0 for the next gradient.
// ---------------------------------------------------------------------------
// Warp-per-row layout: LPR = min(R, 32) lanes per row (a template parameter so
// the matrix-vector loops unroll), lane l holds columns l, l + 32, ... of its
// row; the products with B_k, C_k take the row entries by shuffle and the
// coefficients through L1.
template <typename T, int LPR, int VPL>
__global__ void __launch_bounds__(256) k_factor_update(const FactorUpdateArgs<T> a) {
    if (a.skip && *a.skip) return;
    constexpr int RPW = 32 / LPR;              // rows per warp
    const int R = a.R, RR = R * R;
    const bool hist = a.B != nullptr && *a.hist_len > 0;
    const T at = (T)*a.rate;
    const T b1 = (T)a.beta1, b2 = (T)a.beta2, c1 = (T)(1.0 - a.beta1), c2 = (T)(1.0 - a.beta2);
    const T lam = (T)a.lam, eps = (T)a.eps, lower = (T)a.lower;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane / LPR, l0 = lane % LPR;
    const int64_t wglobal = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t rb = wglobal * RPW; rb < a.nrows; rb += wstride * RPW) {
        const int64_t row = rb + sub;
        const bool act = row < a.nrows;
        int k = 0;
#pragma unroll
        for (int q = 1; q < 4; ++q)
            if (q < a.ndim && row >= a.row_off[q]) k = q;
        T av[VPL], dv[VPL], bv[VPL], g[VPL], uo[VPL], vo[VPL];
#pragma unroll
        for (int c = 0; c < VPL; ++c) {
            const int j = l0 + 32 * c;
            const bool on = act && j < R;
            const int64_t idx = row * R + j;
            av[c] = on ? a.A[idx] : T(0);
            bv[c] = on ? a.Abar[idx] : T(0);
            g[c] = on ? a.G[idx] : T(0);
            uo[c] = on ? a.u[idx] : T(0);
            vo[c] = on ? a.v[idx] : T(0);
            dv[c] = av[c] - bv[c];
            g[c] += lam * av[c];
        }
        if (hist) {
            const T* Bk = a.B + (int64_t)k * RR;
            const T* Ck = a.C + (int64_t)k * RR;
            T sb[VPL], sc[VPL];
#pragma unroll
            for (int c = 0; c < VPL; ++c) sb[c] = sc[c] = T(0);
#pragma unroll
            for (int lc = 0; lc < VPL; ++lc) {
#pragma unroll
                for (int ll = 0; ll < LPR; ++ll) {
                    const int l = ll + 32 * lc;
                    const T dl = __shfl_sync(SGCP_FULL_MASK, dv[lc], ll, LPR);
                    const T bl = __shfl_sync(SGCP_FULL_MASK, bv[lc], ll, LPR);
                    if (l < R) {
#pragma unroll
                        for (int c = 0; c < VPL; ++c) {
                            const int j = l0 + 32 * c;
                            if (j < R) {
                                sb[c] += dl * __ldg(Bk + l * R + j);
                                sc[c] += bl * __ldg(Ck + l * R + j);
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < VPL; ++c) g[c] += sb[c] + sc[c];
        }
#pragma unroll
        for (int c = 0; c < VPL; ++c) {
            const int j = l0 + 32 * c;
            if (!act || j >= R) continue;
            const int64_t idx = row * R + j;
            if (a.grad_only) {
                a.G[idx] = g[c];
                continue;
            }
            const T u = b1 * uo[c] + c1 * g[c];
            const T v = b2 * vo[c] + c2 * g[c] * g[c];
            T an = av[c] - at * u / (sqrt(v) + eps);
            if (an < lower) an = lower;
            a.u[idx] = u;
            a.v[idx] = v;
            a.A[idx] = an;
            a.G[idx] = T(0);
        }
    }
}

static int solver_num_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// FP32, R <= 32, history terms possible.  A block owns up to kFuBlockRows rows of one mode and
// stages B_k and C_k in shared memory; each warp updates 8 rows at once with lane j on column j:
// the rows' d = a - abar and abar are staged per warp and read as 16-byte broadcasts, B_k[l][j]
// and C_k[l][j] as conflict-free pairs, two-wide FMAs.  Every global request of the block is
// issued before the first use.  With gacc set the block also keeps its updated rows and their d
// in shared memory and sums its share of the Grams A'A and D'A (4 x 4 register tiles), added
// into gacc with 16-byte float atomics (GB300's FP64 atomics are far slower); the next update
// (gprev) forms B_k, C_k for its own mode from those sums at its start instead of reading them,
// and its last block clears the buffer, so no kernel between two updates touches the Grams.
constexpr int kFuBlockRows = 64;
constexpr int kFuGroup = kFuBlockRows / 8;   // rows a warp updates (all at once)
constexpr int kFuWarps = 8;

__host__ __device__ inline int64_t fu_blocks_of_mode(const FactorUpdateArgs<float>& a, int k, int64_t* beg,
                                                     int64_t* end) {
    *beg = a.row_off[k];
    *end = k + 1 < a.ndim ? a.row_off[k + 1] : a.nrows;
    return (*end - *beg + kFuBlockRows - 1) / kFuBlockRows;
}

__global__ void __launch_bounds__(256, 2) k_factor_update_rows(const FactorUpdateArgs<float> a) {
    __shared__ __align__(16) float2 sBk[16][32], sCk[16][32];   // [l / 2][j] = (X[l][j], X[l + 1][j])
    __shared__ __align__(16) float sD[kFuWarps][kFuGroup][32], sAb[kFuWarps][kFuGroup][32];
    // dynamic: a, G, u, v of the warp's rows while B / C apply; with gacc the updated rows and d
    extern __shared__ __align__(16) float fu_dyn[];
    float(*sRow)[kFuWarps][kFuGroup][32] = reinterpret_cast<float(*)[kFuWarps][kFuGroup][32]>(fu_dyn);
    float(*sA)[32] = reinterpret_cast<float(*)[32]>(fu_dyn + 4 * kFuBlockRows * 32);
    float(*sDn)[32] = reinterpret_cast<float(*)[32]>(fu_dyn + 5 * kFuBlockRows * 32);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int R = a.R, j = lane;
    const bool on = j < R;
    const bool step = !a.grad_only;
    const bool gram = a.gacc != nullptr && step;
    // this block's mode and rows (no memory access)
    int k = -1;
    int64_t b0 = 0, b1 = 0;
    {
        int64_t b = blockIdx.x;
        for (int m = 0; m < a.ndim && k < 0; ++m) {
            int64_t beg, end;
            const int64_t nb = fu_blocks_of_mode(a, m, &beg, &end);
            if (b < nb) {
                k = m;
                b0 = beg + b * kFuBlockRows;
                b1 = b0 + kFuBlockRows < end ? b0 + kFuBlockRows : end;
            } else {
                b -= nb;
            }
        }
    }
    if (k < 0) return;   // the grid is sized from the same geometry
    const int RR = R * R;
    const int nrows = (int)(b1 - b0);
    // Up to grid_dep_wait() the block reads what the gradient kernel before it leaves alone (the
    // history length, the rate, the coefficients or the previous update's Gram sums, the rows of
    // A, Abar, u and v) and forms the history term of every row; G and the skip flag come after
    // the wait.  The requests of each phase are issued before any of them is used.
    const int32_t hlen = a.B != nullptr ? *a.hist_len : 0;
    const double rate = *a.rate;
    // B_k, C_k entries i = tid + 256 q of the padded 32 x 32 tiles: read (an epoch's first update),
    // or formed here from the previous update's Gram sums (P_n = A'A, E_n = D'A of every mode)
    float bco[4], cco[4];
    float gp[4][4], ge[4][4], gsh[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = threadIdx.x + 256 * q, l = i >> 5, m = i & 31;
        const bool in = a.B != nullptr && l < R && m < R;
        const int e = l * R + m;
        bco[q] = in && !a.gprev ? __ldg(a.B + (int64_t)k * RR + e) : 0.0f;
        cco[q] = in && !a.gprev ? __ldg(a.C + (int64_t)k * RR + e) : 0.0f;
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            const bool ld = in && a.gprev && n < a.ndim;
            gp[q][n] = ld ? __ldcg(a.gprev + (int64_t)n * RR + e) : 0.0f;
            ge[q][n] = ld ? __ldcg(a.gprev + ((int64_t)a.ndim + n) * RR + e) : 0.0f;
        }
        gsh[q] = in && a.gprev ? (float)__ldcg(a.SH + e) : 0.0f;
    }
    // the block's rows through 32-bit offsets from its first row
    float* Ab = a.A + b0 * R;
    const float* Abarb = a.Abar + b0 * R;
    float* Gb = a.G + b0 * R;
    float* ub = a.u + b0 * R;
    float* vb = a.v + b0 * R;
    const int g0 = warp * kFuGroup;   // this warp's rows of the block
    float av[kFuGroup], uv[kFuGroup], vv[kFuGroup], xbv[kFuGroup];
#pragma unroll
    for (int r = 0; r < kFuGroup; ++r) {
        const bool act = on && g0 + r < nrows;
        const int o = act ? (g0 + r) * R + j : 0;
        av[r] = act ? Ab[o] : 0.0f;
        xbv[r] = act ? Abarb[o] : 0.0f;
        uv[r] = act && step ? ub[o] : 0.0f;
        vv[r] = act && step ? vb[o] : 0.0f;
    }
    const bool hist = hlen > 0;
    if (a.gprev)   // B_k = Gamma_k * S_H, C_k = (Gamma_k - Gammabar_k) * S_H of this block's mode
#pragma unroll
        for (int q = 0; q < 4; ++q) hist_coeff_k<float>(a.ndim, k, gp[q], ge[q], gsh[q], bco[q], cco[q]);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = threadIdx.x + 256 * q, l = i >> 5, m = i & 31;
        reinterpret_cast<float*>(&sBk[l >> 1][m])[l & 1] = hist ? bco[q] : 0.0f;
        reinterpret_cast<float*>(&sCk[l >> 1][m])[l & 1] = hist ? cco[q] : 0.0f;
    }
    const float at = (float)rate;
    const float b1c = (float)a.beta1, b2c = (float)a.beta2, c1 = (float)(1.0 - a.beta1), c2 = (float)(1.0 - a.beta2);
    const float lam = (float)a.lam, eps = (float)a.eps, lower = (float)a.lower;
#pragma unroll
    for (int r = 0; r < kFuGroup; ++r) {
        sD[warp][r][lane] = av[r] - xbv[r];   // zero outside the rank and the block's rows
        sAb[warp][r][lane] = xbv[r];
        sRow[0][warp][r][lane] = av[r];       // parked in shared memory: the matrix products
        sRow[2][warp][r][lane] = uv[r];       // below then run without them in registers
        sRow[3][warp][r][lane] = vv[r];
    }
    __syncthreads();   // B_k, C_k and every warp's rows are staged
    // (d B_k + abar C_k)[j] in two interleaved partial sums (even and odd l), packed FMAs
    float2 acc[kFuGroup];
#pragma unroll
    for (int r = 0; r < kFuGroup; ++r) acc[r] = make_float2(0.f, 0.f);
    if (hist) {
#pragma unroll 1
        for (int l4 = 0; l4 < R; l4 += 4) {
            const float2 bp0 = sBk[l4 >> 1][j], bp1 = sBk[(l4 >> 1) + 1][j];
            const float2 cp0 = sCk[l4 >> 1][j], cp1 = sCk[(l4 >> 1) + 1][j];
#pragma unroll
            for (int r = 0; r < kFuGroup; ++r) {
                const float4 d = *reinterpret_cast<const float4*>(&sD[warp][r][l4]);
                const float4 x = *reinterpret_cast<const float4*>(&sAb[warp][r][l4]);
                acc[r] = fma2(make_float2(d.x, d.y), bp0, acc[r]);
                acc[r] = fma2(make_float2(d.z, d.w), bp1, acc[r]);
                acc[r] = fma2(make_float2(x.x, x.y), cp0, acc[r]);
                acc[r] = fma2(make_float2(x.z, x.w), cp1, acc[r]);
            }
        }
    }
    grid_dep_wait();   // the gradient kernel's G is complete and visible from here
    grid_dep_launch();
    if (a.skip && *a.skip) return;   // the solver has finished: nothing is written
    float gv[kFuGroup];
#pragma unroll
    for (int r = 0; r < kFuGroup; ++r) {
        const bool act = on && g0 + r < nrows;
        gv[r] = act ? Gb[(g0 + r) * R + j] : 0.0f;
    }
#pragma unroll
    for (int r = 0; r < kFuGroup; ++r) {
        const bool act = on && g0 + r < nrows;
        float an = 0.0f;
        if (act) {
            const int o = (g0 + r) * R + j;
            const float x = sRow[0][warp][r][lane];
            const float g = gv[r] + lam * x + (acc[r].x + acc[r].y);
            if (!step) {
                Gb[o] = g;
            } else {
                const float u = b1c * sRow[2][warp][r][lane] + c1 * g;
                const float v = b2c * sRow[3][warp][r][lane] + c2 * g * g;
                an = x - at * u / (sqrtf(v) + eps);
                if (an < lower) an = lower;
                ub[o] = u;
                vb[o] = v;
                Ab[o] = an;
                Gb[o] = 0.0f;
            }
        }
        if (gram) {
            sA[g0 + r][lane] = an;
            sDn[g0 + r][lane] = act ? an - sAb[warp][r][lane] : 0.0f;
        }
    }
    if (gram) {

        // ---- Grams of the block's updated rows.  Thread = 4 x 4 tile (l4, m4) of A'A and of D'A over
        // one quarter of the rows; pairs (x_l, x_l+1) * (a_m, a_m+1) give the diagonal entries of a
        // 2 x 2 block and (x_l, x_l+1) * (a_m+1, a_m) the off-diagonal ones, two packed FMAs each.
        __syncthreads();
        const int tq = R >> 2, part = threadIdx.x >> 6, tile = threadIdx.x & 63;
        const int l4 = (tile / 8) * 4, m4 = (tile % 8) * 4;
        float2 pd[4], po[4], ed[4], eo[4];   // [2 x 2 block (lb, mb)]: diagonal, off-diagonal
#pragma unroll
        for (int q = 0; q < 4; ++q) pd[q] = po[q] = ed[q] = eo[q] = make_float2(0.f, 0.f);
        const bool tile_on = tile / 8 < tq && tile % 8 < tq;
        if (tile_on) {
            const int rb = part * (kFuBlockRows / 4), re = min(nrows, rb + kFuBlockRows / 4);
#pragma unroll 2
            for (int r = rb; r < re; ++r) {
                const float4 al = *reinterpret_cast<const float4*>(&sA[r][l4]);
                const float4 dl = *reinterpret_cast<const float4*>(&sDn[r][l4]);
                const float4 am = *reinterpret_cast<const float4*>(&sA[r][m4]);
                const float2 al0 = make_float2(al.x, al.y), al1 = make_float2(al.z, al.w);
                const float2 dl0 = make_float2(dl.x, dl.y), dl1 = make_float2(dl.z, dl.w);
                const float2 am0 = make_float2(am.x, am.y), am1 = make_float2(am.z, am.w);
                const float2 as0 = make_float2(am.y, am.x), as1 = make_float2(am.w, am.z);
                pd[0] = fma2(al0, am0, pd[0]), po[0] = fma2(al0, as0, po[0]);
                pd[1] = fma2(al0, am1, pd[1]), po[1] = fma2(al0, as1, po[1]);
                pd[2] = fma2(al1, am0, pd[2]), po[2] = fma2(al1, as0, po[2]);
                pd[3] = fma2(al1, am1, pd[3]), po[3] = fma2(al1, as1, po[3]);
                ed[0] = fma2(dl0, am0, ed[0]), eo[0] = fma2(dl0, as0, eo[0]);
                ed[1] = fma2(dl0, am1, ed[1]), eo[1] = fma2(dl0, as1, eo[1]);
                ed[2] = fma2(dl1, am0, ed[2]), eo[2] = fma2(dl1, as0, eo[2]);
                ed[3] = fma2(dl1, am1, ed[3]), eo[3] = fma2(dl1, as1, eo[3]);
            }
        }
        // quarters 1..3 meet quarter 0 in shared memory (the parked rows' planes are free now), then
        // one float4 atomic per row of the tile
        float2* hs = reinterpret_cast<float2*>(&sRow[0][0][0][0]);   // [3 parts][16 values][64 tiles]
        if (tile_on && part > 0)                                      // consecutive tiles, consecutive words
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float2* hp = hs + (part - 1) * 16 * 64;
                hp[q * 64 + tile] = pd[q];
                hp[(4 + q) * 64 + tile] = po[q];
                hp[(8 + q) * 64 + tile] = ed[q];
                hp[(12 + q) * 64 + tile] = eo[q];
            }
        __syncthreads();
        if (tile_on && part == 0) {
#pragma unroll
            for (int p2 = 0; p2 < 3; ++p2)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float2* hp = hs + p2 * 16 * 64;
                    const float2 a0 = hp[q * 64 + tile];
                    const float2 a1 = hp[(4 + q) * 64 + tile];
                    const float2 a2 = hp[(8 + q) * 64 + tile];
                    const float2 a3 = hp[(12 + q) * 64 + tile];
                    pd[q].x += a0.x, pd[q].y += a0.y, po[q].x += a1.x, po[q].y += a1.y;
                    ed[q].x += a2.x, ed[q].y += a2.y, eo[q].x += a3.x, eo[q].y += a3.y;
                }
            // block (lb, mb) = q: rows l4 + 2 lb + {0, 1}, columns m4 + 2 mb + {0, 1}
            float P4[4][4], E4[4][4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int lb = q >> 1, mb = q & 1;
                P4[2 * lb][2 * mb] = pd[q].x, P4[2 * lb + 1][2 * mb + 1] = pd[q].y;
                P4[2 * lb][2 * mb + 1] = po[q].x, P4[2 * lb + 1][2 * mb] = po[q].y;
                E4[2 * lb][2 * mb] = ed[q].x, E4[2 * lb + 1][2 * mb + 1] = ed[q].y;
                E4[2 * lb][2 * mb + 1] = eo[q].x, E4[2 * lb + 1][2 * mb] = eo[q].y;
            }
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                float* P = a.gacc + (int64_t)k * RR + (l4 + x) * R + m4;
                float* E = a.gacc + ((int64_t)a.ndim + k) * RR + (l4 + x) * R + m4;
                red_add_f4(P, make_float4(P4[x][0], P4[x][1], P4[x][2], P4[x][3]));
                red_add_f4(E, make_float4(E4[x][0], E4[x][1], E4[x][2], E4[x][3]));
            }
        }
    }
    if (a.gzero && last_block_ticket(a.tk)) {   // every block has read gprev: clear it for reuse
        for (int i = threadIdx.x; i < 2 * a.ndim * RR; i += blockDim.x) a.gzero[i] = 0.0f;
        if (threadIdx.x == 0) {
            a.tk->ticket = 0u;
            __threadfence();
        }
    }
}

// Launches k_factor_update_rows when it applies (FP32, R <= 32, history coefficients present);
// false leaves the update to the warp-per-row kernel.
template <typename T>
static bool factor_update_rows(const FactorUpdateArgs<T>& a, cudaStream_t st, cudaError_t* err) {
    if constexpr (std::is_same<T, float>::value) {
        if (a.R > 32 || a.B == nullptr) return false;
        int64_t blocks = 0;
        for (int k = 0; k < a.ndim; ++k) {
            int64_t beg, end;
            blocks += fu_blocks_of_mode(a, k, &beg, &end);
        }
        if (blocks < 1 || blocks > 0x7fffffff) return false;
        const size_t smem = (a.gacc ? 6 : 4) * kFuBlockRows * 32 * sizeof(float);
        cudaFuncSetAttribute(k_factor_update_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (a.overlap) {
            *err = launch_after_prev(k_factor_update_rows, dim3((unsigned)blocks), dim3(32 * kFuWarps), smem, st, a);
        } else {
            k_factor_update_rows<<<(int)blocks, 32 * kFuWarps, smem, st>>>(a);
            *err = cudaGetLastError();
        }
        return true;
    } else {
        (void)a, (void)st, (void)err;
        return false;
    }
}

template <typename T>
cudaError_t launch_factor_update(const FactorUpdateArgs<T>& a, cudaStream_t st, int64_t* launches) {
    if (a.R > 128) return cudaErrorInvalidValue;
    {
        cudaError_t e = cudaSuccess;
        if (factor_update_rows(a, st, &e)) {
            if (launches) *launches += 1;
            return e;
        }
    }
    const int LPR = a.R < 32 ? a.R : 32;
    const int rows_per_block = 8 * (32 / LPR);
    // one row group per warp, every row in flight at once
    const int64_t want = (a.nrows + rows_per_block - 1) / rows_per_block;
    const int blocks = (int)(want < 1 ? 1 : (want > 0x7fffffff ? 0x7fffffff : want));
    const int vpl = (a.R + 31) / 32;
    if (LPR == 4) k_factor_update<T, 4, 1><<<blocks, 256, 0, st>>>(a);
    else if (LPR == 8) k_factor_update<T, 8, 1><<<blocks, 256, 0, st>>>(a);
    else if (LPR == 16) k_factor_update<T, 16, 1><<<blocks, 256, 0, st>>>(a);
    else if (LPR == 32 && vpl == 1) k_factor_update<T, 32, 1><<<blocks, 256, 0, st>>>(a);
    else if (vpl == 2) k_factor_update<T, 32, 2><<<blocks, 256, 0, st>>>(a);
    else if (vpl == 3) k_factor_update<T, 32, 3><<<blocks, 256, 0, st>>>(a);
    else k_factor_update<T, 32, 4><<<blocks, 256, 0, st>>>(a);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Solver bookkeeping
// ---------------------------------------------------------------------------
__global__ void k_solver_init(SolverState* st, double alpha, int reset_counter) {
    solver_init_state(st, alpha, reset_counter);
}

cudaError_t launch_solver_init(SolverState* st, double alpha, int reset_counter, cudaStream_t stream,
                               int64_t* launches) {
    k_solver_init<<<1, 1, 0, stream>>>(st, alpha, reset_counter);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

// Alg. 3/4 loop test "while F > tol": once it fails, every later kernel of
// the solver call is skipped through st->done.
__global__ void k_epoch_begin(SolverState* st, double tol, double* rates, int tau, double beta1, double beta2,
                              float* zero, int nzero) {
    for (int i = threadIdx.x; i < nzero; i += blockDim.x) zero[i] = 0.0f;
    epoch_begin_block(st, tol, rates, tau, beta1, beta2);
}

cudaError_t launch_epoch_begin(SolverState* st, double tol, double* rates, int tau, double beta1, double beta2,
                               cudaStream_t stream, int64_t* launches, float* zero, int nzero) {
    k_epoch_begin<<<1, 128, 0, stream>>>(st, tol, rates, tau, beta1, beta2, zero, zero ? nzero : 0);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

// Alg. 2 Update(passed) with passed = (F_new <= F_old) and F_new finite.
template <typename T>
__global__ void k_epoch_end(SolverState* st, int64_t n, T* a, T* u, T* v, T* a_o, T* u_o, T* v_o, int tau,
                            double decay, double beta1, double beta2) {
    if (st->done) return;
    const bool passed = epoch_passed(st);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        epoch_end_elem(passed, i, a, u, v, a_o, u_o, v_o);
    if (last_block_ticket(st) && threadIdx.x == 0) {
        epoch_end_state(st, passed, tau, decay, beta1, beta2);
        st->ticket = 0u;
        __threadfence();
    }
}

template <typename T>
cudaError_t launch_epoch_end(SolverState* st, int64_t n, T* a, T* u, T* v, T* a_o, T* u_o, T* v_o, int tau,
                             double decay, double beta1, double beta2, cudaStream_t stream, int64_t* launches) {
    int64_t want = (n + 255) / 256;
    const int64_t cap = 4LL * solver_num_sms();
    const int blocks = (int)(want < 1 ? 1 : (want > cap ? cap : want));
    k_epoch_end<T><<<blocks, 256, 0, stream>>>(st, n, a, u, v, a_o, u_o, v_o, tau, decay, beta1, beta2);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

// ADAM Init (with the checkpoint set to the starting point); zero_a also sets a <- 0 first.
template <typename T>
__global__ void k_adam_reset(int64_t n, const T* a, T* u, T* v, T* a_o, T* u_o, T* v_o, int zero_a, T* a_zero) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (zero_a) a_zero[i] = T(0);
        u[i] = T(0);
        v[i] = T(0);
        u_o[i] = T(0);
        v_o[i] = T(0);
        a_o[i] = zero_a ? T(0) : a[i];
    }
}

template <typename T>
cudaError_t launch_adam_reset(int64_t n, const T* a, T* u, T* v, T* a_o, T* u_o, T* v_o, int zero_a, T* a_zero,
                              cudaStream_t stream, int64_t* launches) {
    int64_t want = (n + 255) / 256;
    const int64_t cap = 4LL * solver_num_sms();
    const int blocks = (int)(want < 1 ? 1 : (want > cap ? cap : want));
    k_adam_reset<T><<<blocks, 256, 0, stream>>>(n, a, u, v, a_o, u_o, v_o, zero_a, a_zero);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Objective terms
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_obj_finish_w(SolverState* st, const T* s, int R, double mu, int set_cur, int* err,
                               const int32_t* skip) {
    if (skip && *skip) return;
    double ss = 0.0;
    for (int j = 0; j < R; ++j) ss += (double)s[j] * (double)s[j];
    const double F = st->F_new + 0.5 * mu * ss;
    st->F_new = F;
    if (!isfinite(F)) set_err(err, ERRB_NUMERIC);
    if (set_cur) st->F_cur = F;
}

template <typename T>
cudaError_t launch_obj_finish_w(SolverState* st, const T* s, int R, double mu, int set_cur, int* err,
                                const int32_t* skip, cudaStream_t stream, int64_t* launches) {
    k_obj_finish_w<T><<<1, 1, 0, stream>>>(st, s, R, mu, set_cur, err, skip);
    if (launches) *launches += 1;
    return cudaGetLastError();
}


// S_H = sum_{h in window} w theta^(t-h) s_h s_h' (one block).  The window is taken in rounds of
// kShSlots slots: each slot's weight w theta^(t-h) is formed once per round (not once per entry)
// and its s_h row staged in shared memory; every entry adds the slots in window order, carrying
// its sum in S_H across rounds, so the result equals the slot-by-slot sum of history_SH_elem.
constexpr int kShSlots = 32;
template <typename T>
__global__ void __launch_bounds__(256) k_history_SH(int R, const T* s_hist, const int64_t* h_dev,
                                                    const int32_t* hist_len, const SliceDesc* slice, double w,
                                                    double theta, double* SH) {
    __shared__ double wh[kShSlots];
    __shared__ T sh[kShSlots * 128];   // R <= 128
    const int n = *hist_len;
    const int64_t t = slice->t;
    const int RR = R * R;
    if (n <= 0) {
        for (int i = threadIdx.x; i < RR; i += blockDim.x) SH[i] = 0.0;
        return;
    }
    for (int h0 = 0; h0 < n; h0 += kShSlots) {
        const int hn = n - h0 < kShSlots ? n - h0 : kShSlots;
        __syncthreads();   // the previous round's slots are no longer read
        if (threadIdx.x < hn) wh[threadIdx.x] = w * pow(theta, (double)(t - __ldcg(h_dev + h0 + threadIdx.x)));
        for (int e = threadIdx.x; e < hn * R; e += blockDim.x) sh[e] = __ldcg(s_hist + (int64_t)h0 * R + e);
        __syncthreads();
        for (int i = threadIdx.x; i < RR; i += blockDim.x) {
            const int l = i / R, m = i - l * R;
            double acc = h0 == 0 ? 0.0 : SH[i];
            for (int h = 0; h < hn; ++h) acc += wh[h] * (double)sh[h * R + l] * (double)sh[h * R + m];
            SH[i] = acc;
        }
    }
}

template <typename T>
cudaError_t launch_history_SH(int R, const T* s_hist, const int64_t* h_dev, const int32_t* hist_len,
                              const SliceDesc* slice, double w, double theta, double* SH, cudaStream_t stream,
                              int64_t* launches) {
    k_history_SH<T><<<1, 256, 0, stream>>>(R, s_hist, h_dev, hist_len, slice, w, theta, SH);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Least-squares temporal solve (one block, Cholesky in double).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_lsq_solve(int ndim, int R, const double* P, const T* rhs, double mu, double lower, T* s,
                            double* Mw, int* err) {
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    for (int i = threadIdx.x; i < R * R; i += blockDim.x) {
        double g = 1.0;
        for (int n = 0; n < ndim; ++n) g *= P[(int64_t)n * R * R + i];
        if (i / R == i % R) g += 0.5 * mu;
        Mw[i] = g;
    }
    __syncthreads();
    // in-place lower Cholesky factor, column by column
    for (int c = 0; c < R; ++c) {
        if (threadIdx.x == 0) {
            double d = Mw[c * R + c];
            for (int k = 0; k < c; ++k) d -= Mw[c * R + k] * Mw[c * R + k];
            if (!(d > 0.0)) {
                bad = 1;
                d = 1.0;
            }
            Mw[c * R + c] = sqrt(d);
        }
        __syncthreads();
        for (int r = c + 1 + threadIdx.x; r < R; r += blockDim.x) {
            double v = Mw[r * R + c];
            for (int k = 0; k < c; ++k) v -= Mw[r * R + k] * Mw[c * R + k];
            Mw[r * R + c] = v / Mw[c * R + c];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double* y = Mw + R * R;
        for (int r = 0; r < R; ++r) {
            double v = (double)rhs[r];
            for (int k = 0; k < r; ++k) v -= Mw[r * R + k] * y[k];
            y[r] = v / Mw[r * R + r];
        }
        for (int r = R - 1; r >= 0; --r) {
            double v = y[r];
            for (int k = r + 1; k < R; ++k) v -= Mw[k * R + r] * y[k];
            y[r] = v / Mw[r * R + r];
        }
        for (int r = 0; r < R; ++r) {
            double v = y[r];
            if (v < lower) v = lower;
            s[r] = (T)v;
        }
        if (bad) set_err(err, ERRB_SOLVE);
    }
}

template <typename T>
cudaError_t launch_lsq_solve(int ndim, int R, const double* P, const T* rhs, double mu, double lower, T* s,
                             double* work, int* err, cudaStream_t stream, int64_t* launches) {
    k_lsq_solve<T><<<1, 128, 0, stream>>>(ndim, R, P, rhs, mu, lower, s, work, err);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

__global__ void k_write_desc(SliceDesc* dst, SliceDesc val) { *dst = val; }

cudaError_t launch_write_desc(SliceDesc* dst, SliceDesc val, cudaStream_t stream, int64_t* launches) {
    k_write_desc<<<1, 1, 0, stream>>>(dst, val);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

template <typename T>
__global__ void k_hist_update(int R, T* s_hist, int64_t* h_dev, int32_t* hist_len, int slot, int64_t t, int len,
                              const T* s) {
    for (int j = threadIdx.x; j < R; j += blockDim.x) s_hist[(int64_t)slot * R + j] = s[j];
    if (threadIdx.x == 0) {
        h_dev[slot] = t;
        *hist_len = len;
    }
}

template <typename T>
cudaError_t launch_hist_update(int R, T* s_hist, int64_t* h_dev, int32_t* hist_len, int slot, int64_t t, int len,
                               const T* s, cudaStream_t stream, int64_t* launches) {
    k_hist_update<T><<<1, 128, 0, stream>>>(R, s_hist, h_dev, hist_len, slot, t, len, s);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Projected L-BFGS on the device (Nocedal & Wright, "Numerical Optimization",
// Alg. 7.4 two-loop recursion; backtracking Armijo line search on the
// projected point).  The vectors are the concatenated factor matrices
// (n = sum I_k R elements, L2-resident for the dense workloads).  The
// recursion, the Armijo test and the pair update each run as one cluster of
// kLbCluster CTAs (one per SM): a pass over the vectors is spread over the
// cluster's threads, and every dot product is reduced per CTA and then across
// the cluster through distributed shared memory, in a fixed order, so that
// every CTA holds the same value and no scalar leaves the device.  One CTA
// alone was limited to ~15 GB/s by its outstanding loads (~40 us per pass at
// n = 49152).
// ---------------------------------------------------------------------------
constexpr int kLbThreads = 1024;
constexpr int kLbCluster = 8;
constexpr int kLbUnroll = 8;

// Sum of v over the whole cluster, returned to every thread of every CTA (same value, same
// order everywhere).  red: 32 doubles, part: 1 double, both in shared memory.
__device__ double lb_cluster_sum(double v, double* red, double* part) {
    cg::cluster_group cl = cg::this_cluster();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(SGCP_FULL_MASK, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        *part = t;
    }
    cl.sync();
    double tot = 0.0;
    for (unsigned r = 0; r < cl.num_blocks(); ++r) tot += *cl.map_shared_rank(part, r);
    cl.sync();   // every CTA has read every part before any part is written again
    return tot;
}

// First element and stride of this thread in a cluster-wide pass.
__device__ __forceinline__ int64_t lb_first() {
    return (int64_t)cg::this_cluster().block_rank() * blockDim.x + threadIdx.x;
}
__device__ __forceinline__ int64_t lb_stride() { return (int64_t)kLbCluster * blockDim.x; }
__device__ __forceinline__ bool lb_leader() { return cg::this_cluster().block_rank() == 0 && threadIdx.x == 0; }

// pd <- c x + pd (x == nullptr: pd <- c pd), returning w'pd of the updated pd.  A thread's
// kLbUnroll elements are loaded before the first store (the pointers do not alias).  Products
// are summed per thread in T (double runs at ~1/64 of the float rate on GB300) and across
// threads in double.
template <typename T>
__device__ double lb_axpy_dot(int64_t n, double* red, double* part, T c, const T* __restrict__ x,
                              T* __restrict__ pd, const T* __restrict__ w) {
    T acc = T(0);
    const int64_t S = lb_stride();
    for (int64_t base = lb_first(); base < n; base += kLbUnroll * S) {
        T xv[kLbUnroll], pv[kLbUnroll], wv[kLbUnroll];
#pragma unroll
        for (int u = 0; u < kLbUnroll; ++u) {
            const int64_t i = base + u * S;
            const bool in = i < n;
            xv[u] = (in && x) ? x[i] : T(0);
            pv[u] = in ? pd[i] : T(0);
            wv[u] = in ? w[i] : T(0);
        }
#pragma unroll
        for (int u = 0; u < kLbUnroll; ++u) {
            const int64_t i = base + u * S;
            const T v = x ? c * xv[u] + pv[u] : c * pv[u];
            if (i < n) pd[i] = v;
            acc += wv[u] * v;
        }
    }
    return lb_cluster_sum((double)acc, red, part);
}

// pd <- g, returning w'g.
template <typename T>
__device__ double lb_copy_dot(int64_t n, double* red, double* part, const T* __restrict__ g, T* __restrict__ pd,
                              const T* __restrict__ w) {
    T acc = T(0);
    const int64_t S = lb_stride();
    for (int64_t base = lb_first(); base < n; base += kLbUnroll * S) {
        T gv[kLbUnroll], wv[kLbUnroll];
#pragma unroll
        for (int u = 0; u < kLbUnroll; ++u) {
            const int64_t i = base + u * S;
            gv[u] = i < n ? g[i] : T(0);
            wv[u] = i < n ? w[i] : T(0);
        }
#pragma unroll
        for (int u = 0; u < kLbUnroll; ++u) {
            const int64_t i = base + u * S;
            if (i < n) pd[i] = gv[u];
            acc += wv[u] * gv[u];
        }
    }
    return lb_cluster_sum((double)acc, red, part);
}

template <typename T>
__global__ void __cluster_dims__(kLbCluster, 1, 1) __launch_bounds__(kLbThreads) k_lbfgs_begin(const LbfgsArgs<T> a) {
    for (int64_t i = lb_first(); i < a.n; i += lb_stride()) {
        a.x[i] = a.A[i];
        a.g[i] = a.G[i];
    }
    if (lb_leader()) {
        LbfgsState* ls = a.ls;
        ls->F = a.sf->F_new;
        ls->npairs = 0;
        ls->done = 0;
        ls->iters = 0;
        ls->evals = 1;
        ls->accepted = 0;
        ls->trial = 0;
        ls->gamma = 1.0;
    }
}

template <typename T>
cudaError_t launch_lbfgs_begin(const LbfgsArgs<T>& a, cudaStream_t st, int64_t* launches) {
    k_lbfgs_begin<T><<<kLbCluster, kLbThreads, 0, st>>>(a);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

// pd <- H g by the two-loop recursion over the stored pairs, newest first then oldest first,
// with H_0 = gamma I (gamma = s'y / y'y of the newest pair, 1 / ||g|| without pairs).  Each
// update of pd shares its pass with the dot product that the next step needs.
template <typename T>
__global__ void __cluster_dims__(kLbCluster, 1, 1) __launch_bounds__(kLbThreads)
    k_lbfgs_direction(const LbfgsArgs<T> a) {
    __shared__ double red[32];
    __shared__ double part;
    __shared__ double alpha[kLbfgsSlots];   // the same values in every CTA
    const LbfgsState* ls = a.ls;
    if (ls->done) return;
    const int np = ls->npairs;
    T* pd = a.pd;
    const T* g = a.g;
    // first loop, newest pair first: q <- q - alpha_k y_k with alpha_k = rho_k s_k'q
    double dot = lb_copy_dot<T>(a.n, red, &part, g, pd, np > 0 ? a.S[ls->order[np - 1]] : g);
    for (int q = np - 1; q >= 0; --q) {
        const int sl = ls->order[q];
        const double al = ls->rho[sl] * dot;
        if (threadIdx.x == 0) alpha[sl] = al;
        const T* y = a.Y[sl];
        const T* sn = q > 0 ? a.S[ls->order[q - 1]] : y;   // (the last step's dot is not used)
        dot = lb_axpy_dot<T>(a.n, red, &part, (T)(-al), y, pd, sn);
    }
    // r = gamma q (gamma = 1 / ||g|| without pairs: dot = g'g then); the same pass forms
    // y_oldest' r for the second loop
    const double gamma = np > 0 ? ls->gamma : 1.0 / fmax(sqrt(dot), 1e-300);
    dot = lb_axpy_dot<T>(a.n, red, &part, (T)gamma, nullptr, pd, np > 0 ? a.Y[ls->order[0]] : g);
    // (alpha[] was written before the cluster barriers of the passes above)
    // second loop, oldest pair first: r <- r + (alpha_k - rho_k y_k'r) s_k
    for (int q = 0; q < np; ++q) {
        const int sl = ls->order[q];
        const T* sv = a.S[sl];
        dot = lb_axpy_dot<T>(a.n, red, &part, (T)(alpha[sl] - ls->rho[sl] * dot), sv, pd,
                             q + 1 < np ? a.Y[ls->order[q + 1]] : sv);
    }
    if (lb_leader()) {
        LbfgsState* lw = a.ls;
        lw->step = 1.0;
        lw->trial = 0;
        lw->accepted = 0;
    }
}

template <typename T>
cudaError_t launch_lbfgs_direction(const LbfgsArgs<T>& a, cudaStream_t st, int64_t* launches) {
    k_lbfgs_direction<T><<<kLbCluster, kLbThreads, 0, st>>>(a);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

template <typename T>
__global__ void k_lbfgs_trial(const LbfgsArgs<T> a) {
    if (a.ls->done) return;
    const T step = (T)a.ls->step;    // a power of two: exact in either type
    const T lower = (T)a.lower;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        const T v = a.x[i] - step * a.pd[i];
        a.A[i] = v < lower ? lower : v;
    }
}

template <typename T>
cudaError_t launch_lbfgs_trial(const LbfgsArgs<T>& a, cudaStream_t st, int64_t* launches) {
    int64_t want = (a.n + 255) / 256;
    const int64_t cap = 4LL * solver_num_sms();
    const int blocks = (int)(want < 1 ? 1 : (want > cap ? cap : want));
    k_lbfgs_trial<T><<<blocks, 256, 0, st>>>(a);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

// Armijo condition on the projected trial point: F(a+) <= F(x) + 1e-4 g'(a+ - x).  A rejected
// trial halves the step and sets the handle of the line search's WHILE node to 1 (another trial)
// while fewer than 30 trials were made; an accepted or last trial sets it to 0.
template <typename T>
__global__ void __cluster_dims__(kLbCluster, 1, 1) __launch_bounds__(kLbThreads)
    k_lbfgs_armijo(const LbfgsArgs<T> a, cudaGraphConditionalHandle h) {
    __shared__ double red[32];
    __shared__ double part;
    if (a.ls->done) return;   // the solve has stopped: the handle keeps its launch value 0
    T acc = T(0);
    const int64_t S = lb_stride();
    for (int64_t base = lb_first(); base < a.n; base += kLbUnroll * S) {
        T gv[kLbUnroll], dv[kLbUnroll];
#pragma unroll
        for (int u = 0; u < kLbUnroll; ++u) {
            const int64_t i = base + u * S;
            const bool in = i < a.n;
            gv[u] = in ? a.g[i] : T(0);
            dv[u] = in ? a.A[i] - a.x[i] : T(0);
        }
#pragma unroll
        for (int u = 0; u < kLbUnroll; ++u) acc += gv[u] * dv[u];
    }
    const double gd = lb_cluster_sum((double)acc, red, &part);
    if (lb_leader()) {
        LbfgsState* ls = a.ls;
        const double Fn = a.sf->F_new;
        ls->evals += 1;
        if (Fn <= ls->F + 1e-4 * gd) {
            ls->accepted = 1;
            cudaGraphSetConditional(h, 0u);
        } else {
            ls->step *= 0.5;
            ls->trial += 1;
            cudaGraphSetConditional(h, ls->trial < 30 ? 1u : 0u);
        }
    }
}

template <typename T>
cudaError_t launch_lbfgs_armijo(const LbfgsArgs<T>& a, cudaGraphConditionalHandle h, cudaStream_t st,
                                int64_t* launches) {
    k_lbfgs_armijo<T><<<kLbCluster, kLbThreads, 0, st>>>(a, h);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

// After a line search: on acceptance store s = a+ - x, y = g(a+) - g in a free slot (kept when
// s'y > 1e-12 ||s|| ||y||; the oldest pair leaves when m are stored) and move to a+; without an
// acceptable step restore A <- x and stop the solve.
template <typename T>
__global__ void __cluster_dims__(kLbCluster, 1, 1) __launch_bounds__(kLbThreads) k_lbfgs_update(const LbfgsArgs<T> a) {
    __shared__ double red[32];
    __shared__ double part;
    const LbfgsState* ls = a.ls;
    // every CTA reads the state before the leader may write it (the barrier below), so that all
    // CTAs take the same branches and meet at the same cluster barriers
    const int done = ls->done, accepted = ls->accepted, np = ls->npairs;
    int sl = 0;                  // the first slot not holding a stored pair (same in every thread)
    for (bool used = true; used;) {
        used = false;
        for (int q = 0; q < np; ++q) used = used || ls->order[q] == sl;
        if (used) ++sl;
    }
    cg::this_cluster().sync();
    if (done) return;
    if (!accepted) {
        for (int64_t i = lb_first(); i < a.n; i += lb_stride()) a.A[i] = a.x[i];
        if (lb_leader()) a.ls->done = 1;
        return;
    }
    T* sv = a.S[sl];
    T* yv = a.Y[sl];
    T sy = T(0), ss = T(0), yy = T(0);
    const int64_t S = lb_stride();
    for (int64_t i = lb_first(); i < a.n; i += S) {
        const T An = a.A[i], Gn = a.G[i];
        const T si = An - a.x[i], yi = Gn - a.g[i];
        sv[i] = si;
        yv[i] = yi;
        a.x[i] = An;
        a.g[i] = Gn;
        sy += si * yi;
        ss += si * si;
        yy += yi * yi;
    }
    const double sy_c = lb_cluster_sum((double)sy, red, &part);
    const double ss_c = lb_cluster_sum((double)ss, red, &part);
    const double yy_c = lb_cluster_sum((double)yy, red, &part);
    if (lb_leader()) {
        LbfgsState* lw = a.ls;
        if (sy_c > 1e-12 * sqrt(ss_c) * sqrt(yy_c)) {
            int n2 = np;
            if (n2 == a.m) {
                for (int q = 1; q < n2; ++q) lw->order[q - 1] = lw->order[q];
                n2 -= 1;
            }
            lw->order[n2] = sl;
            lw->npairs = n2 + 1;
            lw->rho[sl] = 1.0 / sy_c;
            lw->gamma = sy_c / yy_c;
        }
        lw->F = a.sf->F_new;
        lw->iters += 1;
    }
}

template <typename T>
cudaError_t launch_lbfgs_update(const LbfgsArgs<T>& a, cudaStream_t st, int64_t* launches) {
    k_lbfgs_update<T><<<kLbCluster, kLbThreads, 0, st>>>(a);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

__global__ void k_lbfgs_finish(const LbfgsState* ls, SolverState* sf) {
    sf->F_cur = ls->F;
    sf->epoch = ls->iters;
    sf->evals = ls->evals;
    sf->accept = 0u;
    sf->done = 0;
}

cudaError_t launch_lbfgs_finish(LbfgsState* ls, SolverState* sf, cudaStream_t st, int64_t* launches) {
    k_lbfgs_finish<<<1, 1, 0, st>>>(ls, sf);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

// Objective finish of the warm start's stacked problem: F_new += lambda/2 ||W||^2 over every
// factor matrix of the stack (one 8-CTA cluster; per-thread sums in T, the rest in double).
template <typename T>
__global__ void __cluster_dims__(kLbCluster, 1, 1) __launch_bounds__(kLbThreads)
    k_reg_objective(SolverState* st, const T* W, int64_t n, double lam, int set_cur, int* err, const int32_t* skip) {
    __shared__ double red[32];
    __shared__ double part;
    if (skip && *skip) return;
    T acc = T(0);
    for (int64_t i = lb_first(); i < n; i += lb_stride()) acc += W[i] * W[i];
    const double ss = lb_cluster_sum((double)acc, red, &part);
    if (lb_leader()) {
        const double F = st->F_new + 0.5 * lam * ss;
        st->F_new = F;
        if (!isfinite(F)) set_err(err, ERRB_NUMERIC);
        if (set_cur) st->F_cur = F;
    }
}

template <typename T>
cudaError_t launch_reg_objective(SolverState* st, const T* W, int64_t n, double lam, int set_cur, int* err,
                                 const int32_t* skip, cudaStream_t stream, int64_t* launches) {
    k_reg_objective<T><<<kLbCluster, kLbThreads, 0, stream>>>(st, W, n, lam, set_cur, err, skip);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

// Factor solver's objective terms beyond the sampled loss: F_new += 1/2 sum_h w_h ||Mbar_h - M_h||^2
// (eq. gcp_stream_objective, telescoped Gram form: sum over entries (l, m) of S_H[l][m] times
// sum_{k, kk} prod_n Gram_n(which(k, n), which(kk, n))[l][m]) + lambda/2 sum_n ||A^(n)||^2.  One
// 8-CTA cluster: a work item is one (entry, k, kk) triple, whose ndim Gram entries are independent
// loads, so each thread has a few loads in flight instead of one block walking every product of every
// entry; the per-thread sums are reduced across the cluster in a fixed order.
__global__ void __cluster_dims__(kLbCluster, 1, 1) __launch_bounds__(kLbThreads)
    k_obj_finish_f(SolverState* st, int ndim, int R, const double* grams, const double* SH, const int32_t* hist_len,
                   double lam, int set_cur, int* err, const int32_t* skip) {
    __shared__ double red[32];
    __shared__ double part;
    if (skip && *skip) return;   // the same flag for every CTA of the cluster
    const bool hist = *hist_len > 0;
    const int RR = R * R, D2 = ndim * ndim;
    double acc = 0.0, reg = 0.0;
    for (int64_t it = lb_first(); it < (int64_t)RR * D2; it += lb_stride()) {
        const int i = (int)(it / D2), kp = (int)(it - (int64_t)i * D2);
        const int k = kp / ndim, kk = kp - k * ndim;
        const int l = i / R, m = i - l * R;
        if (hist) {
            double prod = 1.0;
#pragma unroll 4
            for (int n = 0; n < ndim; ++n) prod *= gram_entry(grams, ndim, R, n, which_mat(k, n), which_mat(kk, n), l, m);
            acc += __ldcg(SH + i) * prod;
        }
        if (kp == 0 && l == m)
            for (int n = 0; n < ndim; ++n) reg += __ldcg(grams + (int64_t)n * RR + i);
    }
    const double tot = lb_cluster_sum(0.5 * acc + 0.5 * lam * reg, red, &part);
    if (lb_leader()) {
        const double F = __ldcg(&st->F_new) + tot;
        st->F_new = F;
        if (!isfinite(F)) set_err(err, ERRB_NUMERIC);
        if (set_cur) st->F_cur = F;
    }
}

cudaError_t launch_obj_finish_f(SolverState* st, int ndim, int R, const double* grams, const double* SH,
                                const int32_t* hist_len, double lam, int set_cur, int* err, const int32_t* skip,
                                cudaStream_t stream, int64_t* launches) {
    k_obj_finish_f<<<kLbCluster, kLbThreads, 0, stream>>>(st, ndim, R, grams, SH, hist_len, lam, set_cur, err, skip);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

// Stored-slice history (eq. gcp_stream_problem_1), at the start of a step: window slot j is
// active when j < |window|; its weight w_j = w theta^(t - h_j) becomes the y_scale of its launches,
// its descriptor's draw base t * per_step keeps its samples distinct from every other step's,
// and its skip flag is set when it is inactive.
template <typename T>
__global__ void k_hist_slots_begin(SliceDesc* desc, T* wts, int32_t* skip, const int32_t* hist_len,
                                   const int64_t* h_dev, const SliceDesc* cur, double w, double theta, int H,
                                   uint32_t per_step) {
    const int n = *hist_len;
    const int64_t t = cur->t;
    for (int j = threadIdx.x; j < H; j += blockDim.x) {
        const bool on = j < n;
        wts[j] = on ? (T)(w * pow(theta, (double)(t - h_dev[j]))) : T(0);
        skip[j] = on ? 0 : 1;
        desc[j].draw_base = (uint32_t)((uint64_t)t * per_step);
    }
}

template <typename T>
cudaError_t launch_hist_slots_begin(SliceDesc* desc, T* wts, int32_t* skip, const int32_t* hist_len,
                                    const int64_t* h_dev, const SliceDesc* cur, double w, double theta, int H,
                                    uint32_t per_step, cudaStream_t st, int64_t* launches) {
    k_hist_slots_begin<T><<<1, 128, 0, st>>>(desc, wts, skip, hist_len, h_dev, cur, w, theta, H, per_step);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

// After each epoch test of the factor solver: a slot also skips once the solver has finished.
__global__ void k_hist_slots_skip(int32_t* skip, const int32_t* hist_len, const int32_t* done, int H) {
    const int n = *hist_len, d = *done;
    for (int j = threadIdx.x; j < H; j += blockDim.x) skip[j] = (j >= n || d) ? 1 : 0;
}

cudaError_t launch_hist_slots_skip(int32_t* skip, const int32_t* hist_len, const int32_t* done, int H,
                                   cudaStream_t st, int64_t* launches) {
    k_hist_slots_skip<<<1, 128, 0, st>>>(skip, hist_len, done, H);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

template <typename T>
__global__ void k_copy(T* dst, const T* src, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

template <typename T>
cudaError_t launch_copy(T* dst, const T* src, int64_t n, cudaStream_t stream, int64_t* launches) {
    int64_t want = (n + 255) / 256;
    const int64_t cap = 4LL * solver_num_sms();
    const int blocks = (int)(want < 1 ? 1 : (want > cap ? cap : want));
    k_copy<T><<<blocks, 256, 0, stream>>>(dst, src, n);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

#define SGCP_INST(T)                                                                                                  \
    template cudaError_t launch_gram<T>(const GramArgs<T>&, int64_t, cudaStream_t, int64_t*);                        \
    template cudaError_t launch_hist_coeffs<T>(int, int, const double*, int, const double*, const int32_t*, T*, T*,  \
                                               const int32_t*, cudaStream_t, int64_t*);                              \
    template cudaError_t launch_factor_update<T>(const FactorUpdateArgs<T>&, cudaStream_t, int64_t*);                \
    template cudaError_t launch_epoch_end<T>(SolverState*, int64_t, T*, T*, T*, T*, T*, T*, int, double, double,     \
                                             double, cudaStream_t, int64_t*);                                         \
    template cudaError_t launch_adam_reset<T>(int64_t, const T*, T*, T*, T*, T*, T*, int, T*, cudaStream_t,          \
                                              int64_t*);                                                              \
    template cudaError_t launch_obj_finish_w<T>(SolverState*, const T*, int, double, int, int*, const int32_t*,      \
                                                cudaStream_t, int64_t*);                                              \
    template cudaError_t launch_history_SH<T>(int, const T*, const int64_t*, const int32_t*, const SliceDesc*,       \
                                              double, double, double*, cudaStream_t, int64_t*);                      \
    template cudaError_t launch_lsq_solve<T>(int, int, const double*, const T*, double, double, T*, double*, int*,   \
                                             cudaStream_t, int64_t*);                                                 \
    template cudaError_t launch_copy<T>(T*, const T*, int64_t, cudaStream_t, int64_t*);                          \
    template cudaError_t launch_hist_slots_begin<T>(SliceDesc*, T*, int32_t*, const int32_t*, const int64_t*,     \
                                                    const SliceDesc*, double, double, int, uint32_t, cudaStream_t, \
                                                    int64_t*);                                                       \
    template cudaError_t launch_reg_objective<T>(SolverState*, const T*, int64_t, double, int, int*, const int32_t*, \
                                                 cudaStream_t, int64_t*);                                            \
    template cudaError_t launch_lbfgs_begin<T>(const LbfgsArgs<T>&, cudaStream_t, int64_t*);                      \
    template cudaError_t launch_lbfgs_direction<T>(const LbfgsArgs<T>&, cudaStream_t, int64_t*);                  \
    template cudaError_t launch_lbfgs_trial<T>(const LbfgsArgs<T>&, cudaStream_t, int64_t*);                      \
    template cudaError_t launch_lbfgs_armijo<T>(const LbfgsArgs<T>&, cudaGraphConditionalHandle, cudaStream_t,     \
                                                int64_t*);                                                           \
    template cudaError_t launch_lbfgs_update<T>(const LbfgsArgs<T>&, cudaStream_t, int64_t*);                     \
    template cudaError_t launch_hist_update<T>(int, T*, int64_t*, int32_t*, int, int64_t, int, const T*,            \
                                               cudaStream_t, int64_t*);

SGCP_INST(float)
SGCP_INST(double)

}  // namespace sgcp
