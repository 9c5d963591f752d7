// Evaluation metrics of arXiv 2110.14514 Sec. 6: the pieces of the exact
// reconstruction loss (||X||_F^2; the all-entries model term comes from the
// dense loss kernels run on the all-zero slice) and the K-tensor score of
// Sec. 6.1, the congruence (Tomasi and Bro) between two K-tensors' rank-one
// components: Q[r][c] = prod_k |cos(a_r^(k), b_c^(k))|, and the mean of Q over
// the best matching of components (all R! matchings for R <= 8, greedy
// otherwise).
#include "internal.h"

namespace sgcp {

static int score_num_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// *out += sum_i x_i^2: per-thread sums in T, block sums in double, one double atomic per block.
template <typename T>
__global__ void __launch_bounds__(256) k_sum_squares(const T* __restrict__ x, int64_t n, double* out) {
    __shared__ double red[8];
    T acc = T(0);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += x[i] * x[i];
    double v = (double)acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(SGCP_FULL_MASK, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        if (t != 0.0) atomicAdd(out, t);
    }
}

template <typename T>
cudaError_t launch_sum_squares(const T* x, int64_t n, double* out, cudaStream_t st, int64_t* launches) {
    if (n <= 0) return cudaSuccess;
    const int64_t want = (n + 255) / 256;
    const int64_t cap = 4LL * score_num_sms();
    k_sum_squares<T><<<(int)(want < cap ? want : cap), 256, 0, st>>>(x, n, out);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

constexpr int kScoreMaxModes = 8;
constexpr int kScoreMaxR = 128;

struct ScoreMats {
    const void* A[kScoreMaxModes];
    const void* B[kScoreMaxModes];
    int64_t dims[kScoreMaxModes];
};

// Block (r, k): row r of the cross-Gram C_k = A_k' B_k (thread c owns column c; the A_k[i][r]
// read is a broadcast, the B_k[i][c] reads are one row per warp), and the squared norms of
// column r of A_k and of B_k.  Sums in double.
template <typename T>
__global__ void k_cong_cross(ScoreMats m, int R, double* C, double* na, double* nb) {
    const int r = blockIdx.x, k = blockIdx.y, c = threadIdx.x;
    const T* A = (const T*)m.A[k];
    const T* B = (const T*)m.B[k];
    const int64_t I = m.dims[k];
    double acc = 0.0, aa = 0.0, bb = 0.0;
    if (c < R) {
        for (int64_t i = 0; i < I; ++i) {
            const double ar = (double)A[i * R + r];
            const double bc = (double)B[i * R + c];
            acc += ar * bc;
            if (c == 0) aa += ar * ar;
            if (c == r) bb += (double)B[i * R + r] * (double)B[i * R + r];
        }
        C[((int64_t)k * R + r) * R + c] = acc;
        if (c == 0) na[k * R + r] = aa;
        if (c == r) nb[k * R + r] = bb;
    }
}

// One block: Q from the cross-Grams, then the matching.  Q in dynamic shared memory (R * R doubles).
__global__ void __launch_bounds__(1024) k_cong_match(int nm, int R, const double* C, const double* na, const double* nb,
                                                     double* score, int32_t* perm) {
    extern __shared__ __align__(16) double Q[];
    __shared__ double bv[32];
    __shared__ long long bi[32];
    __shared__ int used_r[kScoreMaxR], used_c[kScoreMaxR];
    __shared__ double best_v;
    __shared__ long long best_i;
    const int RR = R * R;
    for (int i = threadIdx.x; i < RR; i += blockDim.x) {
        const int r = i / R, c = i - r * R;
        double q = 1.0;
        for (int k = 0; k < nm; ++k) {
            const double den = sqrt(na[k * R + r]) * sqrt(nb[k * R + c]);
            q *= den > 0.0 ? fabs(C[((int64_t)k * R + r) * R + c]) / den : 0.0;
        }
        Q[i] = q;
    }
    for (int i = threadIdx.x; i < R; i += blockDim.x) used_r[i] = used_c[i] = 0;
    __syncthreads();
    // block argmax of (value, index): the larger value wins, equal values go to the smaller index
    auto argmax = [&](double v, long long idx) {
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double v2 = __shfl_xor_sync(SGCP_FULL_MASK, v, o);
            const long long i2 = __shfl_xor_sync(SGCP_FULL_MASK, idx, o);
            if (v2 > v || (v2 == v && i2 < idx)) {
                v = v2;
                idx = i2;
            }
        }
        if (lane == 0) {
            bv[w] = v;
            bi[w] = idx;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double v0 = bv[0];
            long long i0 = bi[0];
            for (int j = 1; j < (int)(blockDim.x >> 5); ++j)
                if (bv[j] > v0 || (bv[j] == v0 && bi[j] < i0)) {
                    v0 = bv[j];
                    i0 = bi[j];
                }
            best_v = v0;
            best_i = i0;
        }
        __syncthreads();
    };
    if (R <= 8) {
        // every matching, in lexicographic order of the permutation (index p in factorial base)
        long long nperm = 1;
        for (int i = 2; i <= R; ++i) nperm *= i;
        double v = -1.0;
        long long vi = 0x7fffffffffffffffLL;
        for (long long p = threadIdx.x; p < nperm; p += blockDim.x) {
            bool taken[8] = {false, false, false, false, false, false, false, false};
            long long rest = p, f = nperm;
            double tot = 0.0;
            for (int r = 0; r < R; ++r) {
                f /= (R - r);
                int d = (int)(rest / f);
                rest -= d * f;
                int c = 0;
                for (;; ++c)
                    if (!taken[c] && d-- == 0) break;
                taken[c] = true;
                tot += Q[r * R + c];
            }
            if (tot > v) {   // p increases within a thread: equal sums keep the first
                v = tot;
                vi = p;
            }
        }
        argmax(v, vi);
        if (threadIdx.x == 0) {
            long long rest = best_i, f = nperm;
            bool taken[8] = {false, false, false, false, false, false, false, false};
            for (int r = 0; r < R; ++r) {
                f /= (R - r);
                int d = (int)(rest / f);
                rest -= d * f;
                int c = 0;
                for (;; ++c)
                    if (!taken[c] && d-- == 0) break;
                taken[c] = true;
                perm[r] = c;
            }
            *score = best_v / R;
        }
        return;
    }
    // greedy: R rounds, each takes the largest entry among unused rows and columns
    double tot = 0.0;
    for (int round = 0; round < R; ++round) {
        double v = -1.0;
        long long vi = 0x7fffffffffffffffLL;
        for (int i = threadIdx.x; i < RR; i += blockDim.x) {
            const int r = i / R, c = i - r * R;
            if (!used_r[r] && !used_c[c] && Q[i] > v) {
                v = Q[i];
                vi = i;
            }
        }
        argmax(v, vi);
        if (threadIdx.x == 0) {
            const int r = (int)(best_i / R), c = (int)(best_i - (long long)r * R);
            used_r[r] = 1;
            used_c[c] = 1;
            perm[r] = c;
            tot += best_v;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *score = tot / R;
}

template <typename T>
cudaError_t launch_congruence(int nm, int R, const int64_t* dims, const T* const* A, const T* const* B, double* C,
                              double* na, double* nb, double* score, int32_t* perm, cudaStream_t st) {
    if (nm < 1 || nm > kScoreMaxModes || R < 1 || R > kScoreMaxR) return cudaErrorInvalidValue;
    ScoreMats m{};
    for (int k = 0; k < nm; ++k) {
        m.A[k] = A[k];
        m.B[k] = B[k];
        m.dims[k] = dims[k];
    }
    k_cong_cross<T><<<dim3(R, nm), (R + 31) / 32 * 32, 0, st>>>(m, R, C, na, nb);
    const size_t smem = (size_t)R * R * sizeof(double);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_cong_match, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_cong_match<<<1, 1024, smem, st>>>(nm, R, C, na, nb, score, perm);
    return cudaGetLastError();
}

template cudaError_t launch_sum_squares<float>(const float*, int64_t, double*, cudaStream_t, int64_t*);
template cudaError_t launch_sum_squares<double>(const double*, int64_t, double*, cudaStream_t, int64_t*);
template cudaError_t launch_congruence<float>(int, int, const int64_t*, const float* const*, const float* const*,
                                              double*, double*, double*, double*, int32_t*, cudaStream_t);
template cudaError_t launch_congruence<double>(int, int, const int64_t*, const double* const*, const double* const*,
                                               double*, double*, double*, double*, int32_t*, cudaStream_t);

}  // namespace sgcp
