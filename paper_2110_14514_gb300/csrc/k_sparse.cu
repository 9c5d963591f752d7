// Sparse-slice kernels: slice ingest (nonzero hash + hot rows) and the fused
// stratified-sample -> Kruskal model -> loss derivative -> all-mode MTTKRP
// kernel (arXiv 2110.14514 Sec. 4.3, Alg. 5 / Alg. 6; Sec. 2.2 eqs.
// gcp_grad_A, gcp_grad_lambda).
//
// Layout of the fused kernel: a warp owns chunks of 32 consecutive sample
// slots.  In phase 1 every lane draws one sample (Philox counter -> COO entry
// for a nonzero sample, bounded rejection against the nonzero hash for a zero
// sample).  In phase 2 the warp walks its 32 samples SPW at a time: a group of
// G = R/4 lanes handles one sample, each lane holding four consecutive rank
// components j, so every factor-row gather is one 16-byte load per lane and
// a 128-byte row for R = 32.  m is reduced with xor shuffles inside the
// group, y = w df/dm(x, m) stays in registers (the sampled gradient tensor Y~
// is never stored), and every mode's row contribution y s * prod_{n != k}
// a^(n) is added with a 16-byte vector atomic -- or, for the few rows that
// most nonzeros hit (Zipf-like modes), into a per-block shared-memory
// accumulator flushed once at the end.
#include "internal.h"
#include "sgcp.h"

namespace sgcp {

static constexpr unsigned long long kEmpty = ~0ull;

__device__ __forceinline__ unsigned long long hash_home(unsigned long long key, int hlog2) {
    return (key * 0x9E3779B97F4A7C15ull) >> (64 - hlog2);
}

__device__ __forceinline__ bool hash_contains(const unsigned long long* __restrict__ keys, int hlog2,
                                              unsigned long long key) {
    const unsigned long long mask = (1ull << hlog2) - 1ull;
    unsigned long long h = hash_home(key, hlog2);
    for (unsigned long long probe = 0; probe <= mask; ++probe) {
        const unsigned long long k = __ldg(keys + h);
        if (k == key) return true;
        if (k == kEmpty) return false;
        h = (h + 1ull) & mask;
    }
    return false;
}

// Per-draw constants shared by all threads.
struct DrawSizes {
    int64_t p_eff, total;
    float w_nz, w_z;
};

__device__ __forceinline__ DrawSizes draw_sizes(const SparseGradArgs& a, const SliceDesc& sd) {
    DrawSizes z;
    const int64_t eta = sd.nnz;
    int64_t omega = 1;
    for (int k = 0; k < a.ndim; ++k) omega *= a.dims[k];
    const int64_t zeta = omega - eta;
    int64_t q_eff;
    if (a.all_nnz) {
        z.p_eff = eta;
        q_eff = 0;
    } else {
        z.p_eff = eta > 0 ? a.p : 0;
        q_eff = zeta > 0 ? a.q : 0;   // a slice without zeros drops its zero stratum
    }
    z.total = z.p_eff + q_eff;
    z.w_nz = a.all_nnz ? 1.0f : (z.p_eff ? (float)((double)eta / (double)z.p_eff) : 0.0f);
    z.w_z = q_eff ? (float)((double)zeta / (double)q_eff) : 0.0f;
    return z;
}

// Draw sample slot c (Alg. 6 with the counter layout (slot, attempt, draw, purpose<<24 | t)).
// Error bits (a bad coordinate, an exhausted zero-sample search) are ORed into errb.
template <int D>
__device__ __forceinline__ void gen_sample(const SparseGradArgs& a, const SliceDesc& sd, const DrawSizes& z,
                                           int64_t c, int (&ci)[D], float& x, float& w, int& attempt, bool& ok,
                                           int& errb) {
    ok = false;
    x = 0.0f;
    w = 0.0f;
    attempt = -1;
#pragma unroll
    for (int k = 0; k < D; ++k) ci[k] = 0;
    if (c >= z.total) return;
    const float* vals = (const float*)sd.vals;
    const uint32_t draw = a.draw + sd.draw_base;
    if (a.all_nnz || c < z.p_eff) {
        int64_t e = c;
        if (!a.all_nnz) {
            uint32_t ctr[4] = {(uint32_t)c, 0u, draw, counter_word3(a.pur_nz, sd.t)};
            philox4x32_10(ctr, a.key0, a.key1);
            e = bounded_u32(ctr[0], (uint32_t)sd.nnz);
        }
        // The caller's coordinates are checked before any row is touched: an out-of-range
        // entry latches ERRB_COORD and the sample is dropped (no gather, no scatter).
        bool inb = true;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            ci[k] = __ldg(sd.idx + e * D + k);
            inb = inb && ci[k] >= 0 && (int64_t)ci[k] < a.dims[k];
        }
        if (!inb) {
#pragma unroll
            for (int k = 0; k < D; ++k) ci[k] = 0;
            errb |= ERRB_COORD;
            return;
        }
        x = __ldg(vals + e);
        w = z.w_nz;
        ok = true;
        return;
    }
    const uint32_t cz = (uint32_t)(c - z.p_eff);
    const uint32_t w3 = counter_word3(a.pur_z, sd.t);
    const unsigned long long* hk = sd.hkeys ? sd.hkeys : a.hkeys;   // a stored slice's own hash
    const int hl = sd.hkeys ? sd.hlog2 : a.hlog2;
    for (int att = 0; att < a.cap; ++att) {
        uint32_t ctr[4] = {cz, (uint32_t)att, draw, w3};
        philox4x32_10(ctr, a.key0, a.key1);
        unsigned long long key = 0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            ci[k] = (int)bounded_u32(ctr[k], (uint32_t)a.dims[k]);
            key = key * (unsigned long long)a.dims[k] + (unsigned long long)ci[k];
        }
        if (!hash_contains(hk, hl, key)) {
            w = z.w_z;
            attempt = att;
            ok = true;
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < D; ++k) ci[k] = 0;
    errb |= ERRB_SAMPLING;
}

__device__ __forceinline__ float4 f4mul(float4 a, float4 b) {
    return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w);
}
__device__ __forceinline__ float4 f4scale(float4 a, float s) { return make_float4(a.x * s, a.y * s, a.z * s, a.w * s); }

// Hot-row accumulator layout: slot row of RP floats with column j of slot s
// stored at (j + s) mod RP, so that samples with different hot slots that a
// warp scatters in the same instruction fall in different shared-memory banks.
__device__ __forceinline__ int hot_pos(int k, int slot, int nhot, int RP, int j) {
    return (k * nhot + slot) * RP + ((j + slot) & (RP - 1));
}

// CPL = columns per lane (a multiple of 4): G = RP / CPL lanes share one
// sample, SPW = 32 / G samples per warp step.  Wider lanes amortise the
// per-sample scalar work (record load, loss derivative, reduction) over more
// columns.
// Three 256-thread blocks per SM where the register budget allows it without
// spilling much (<= 3 modes, <= 8 columns per lane): the kernel is bound by the
// latency of its L2 row gathers, and a third block cut the R = 32 factor
// gradient from 39.5 to 32.1 us on GB300.
template <int D, int RP, int CPL, bool WG = true>
__global__ void __launch_bounds__(256, (D <= 3 && CPL <= 8) ? 3 : 2) k_sparse_grad(const SparseGradArgs a) {
    constexpr int G = RP / CPL;      // lanes per sample
    constexpr int SPW = 32 / G;      // samples per warp step
    constexpr int NR = 32 / SPW;     // steps per chunk of 32 samples
    constexpr int NV = CPL / 4;      // float4 per lane per row
    constexpr int RS = (2 * D + 2 + 3) / 4 * 4;   // words per staged sample record
    extern __shared__ __align__(16) float smem[];
    __shared__ __align__(16) int srec[8 * 32 * RS];   // 8 warps x 32 records
    __shared__ DrawSizes zs;
    __shared__ __align__(16) float spend[RP];           // s after a deferred step
    // Up to grid_dep_wait() the kernel reads only the slice (its descriptor, COO arrays, nonzero
    // hash and hot-row tables, none of which a kernel of a solve writes) and writes only shared
    // memory: the set-up and the first chunk's draw overlap the previous kernel of the solve.
    const SliceDesc sd = a.slice ? *a.slice : a.inline_slice;
    const bool wantG = WG && (a.want & SGCP_WANT_FACTORS) != 0;
    const bool wantS = (a.want & SGCP_WANT_TEMPORAL) != 0;
    const bool wantF = (a.want & SGCP_WANT_LOSS) != 0;
    const int nhot = wantG ? a.nhot : 0;
    const int R = a.R;

    float* hacc = smem;                                  // [D][nhot][RP]
    float* gsb = smem + D * nhot * RP;                   // [RP]
    double* fb = (double*)(gsb + RP);                    // [8]
    for (int i = threadIdx.x; i < D * nhot * RP + RP; i += blockDim.x) smem[i] = 0.0f;
    if (threadIdx.x < 8) fb[threadIdx.x] = 0.0;
    if (threadIdx.x == 0) zs = draw_sizes(a, sd);        // the double divisions, once per block
    __syncthreads();
    const DrawSizes z = zs;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane / G, gl = lane % G;
    const int j0 = gl * CPL;
    int* wrec = srec + warp * 32 * RS;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 sv[NV];
    bool vact[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) vact[v] = j0 + 4 * v < R;
    float4 gsl[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) gsl[v] = zero4;
    float fl = 0.0f;        // per-lane loss partial (a few samples); reduced in double below

    const int64_t nchunks = (z.total + 31) / 32;
    const int wpb = blockDim.x >> 5;
    const int64_t stride = (int64_t)gridDim.x * wpb;
    int64_t ch = (int64_t)blockIdx.x * wpb + warp;

    // Software pipeline: the sample of the next chunk (Philox, COO / hash and
    // hot-table loads) is drawn while the current chunk's rows are processed.
    int ci[D], hs[D];
    float x = 0.0f, w = 0.0f;
    int att, errb = 0;
    bool ok = false;
    auto draw = [&](int64_t c) {
        gen_sample<D>(a, sd, z, c * 32 + lane, ci, x, w, att, ok, errb);
#pragma unroll
        for (int k = 0; k < D; ++k) hs[k] = (nhot && ok) ? __ldg(a.hot[k] + ci[k]) : -1;
    };
    if (ch < nchunks) draw(ch);

    grid_dep_wait();     // the previous kernel's s, factors, outputs and flags are visible from here
    grid_dep_launch();
    if (a.skip && *a.skip) return;   // uniform over the grid: the solver has finished
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.zero_n; i += gridDim.x * blockDim.x) a.zero_buf[i] = 0.0f;
    if (a.pend_on) {   // the previous kernel's ADAM step on s, formed by every block for its own use
        const TemporalStep<float>& ps = a.pend;
        const double rate = a.pend_apply ? __ldcg(ps.rate) : 0.0;
        for (int j = threadIdx.x; j < R; j += blockDim.x) {   // one element per thread
            float s1 = __ldcg(ps.s + j), u1 = __ldcg(ps.u + j), v1 = __ldcg(ps.v + j);
            if (a.pend_apply) adam_s_elem<float>(ps, rate, __ldcg(a.pend_g + j), s1, u1, v1, s1, u1, v1);
            spend[j] = s1;
            if (blockIdx.x == 0) {
                a.pend_s_out[j] = s1;
                a.pend_u_out[j] = u1;
                a.pend_v_out[j] = v1;
            }
        }
        __syncthreads();
#pragma unroll
        for (int v = 0; v < NV; ++v) sv[v] = vact[v] ? *reinterpret_cast<const float4*>(spend + j0 + 4 * v) : zero4;
    } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) sv[v] = vact[v] ? *reinterpret_cast<const float4*>(a.s + j0 + 4 * v) : zero4;
    }
    const float ysc = a.y_scale ? *a.y_scale : 1.0f;

    for (; ch < nchunks; ch += stride) {
        // stage the 32 records of this chunk: [coords | hot slots | x | w], w == 0 marks an empty slot
        __syncwarp();
        {
            int* rec = wrec + lane * RS;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                rec[k] = ci[k];
                rec[D + k] = hs[k];
            }
            rec[2 * D] = __float_as_int(x);
            rec[2 * D + 1] = __float_as_int(ok ? w : 0.0f);
        }
        __syncwarp();
        if (ch + stride < nchunks) draw(ch + stride);

#pragma unroll 1
        for (int r = 0; r < NR; ++r) {
            const int src = r * SPW + grp;
            int rv[RS];
#pragma unroll
            for (int q = 0; q < RS / 4; ++q) {
                const int4 v4 = *reinterpret_cast<const int4*>(wrec + src * RS + 4 * q);
                rv[4 * q + 0] = v4.x;
                rv[4 * q + 1] = v4.y;
                rv[4 * q + 2] = v4.z;
                rv[4 * q + 3] = v4.w;
            }
            const float xj = __int_as_float(rv[2 * D]);
            const float wj = __int_as_float(rv[2 * D + 1]);
            const bool okj = wj != 0.0f;
            uint32_t off[D];
#pragma unroll
            for (int k = 0; k < D; ++k) off[k] = (uint32_t)rv[k] * (uint32_t)R + (uint32_t)j0;
            float4 av[D][NV];
#pragma unroll
            for (int k = 0; k < D; ++k)
#pragma unroll
                for (int v = 0; v < NV; ++v)
                    av[k][v] = vact[v] ? __ldg(reinterpret_cast<const float4*>(a.A[k] + off[k] + 4 * v)) : zero4;
            float mp = 0.0f;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                float4 pr = sv[v];
#pragma unroll
                for (int k = 0; k < D; ++k) pr = f4mul(pr, av[k][v]);
                mp += (pr.x + pr.y) + (pr.z + pr.w);
            }
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) mp += __shfl_xor_sync(SGCP_FULL_MASK, mp, o);
            const float y = loss_dfdm<float>(a.loss, xj, mp, a.eps);
            const float yw = okj ? y * wj * ysc : 0.0f;
            if (wantF && gl == 0 && okj) {
                float f, yy;
                loss_eval<float>(a.loss, xj, mp, a.eps, f, yy);
                if (a.f_minus_zero) {
                    float f0;
                    loss_eval<float>(a.loss, 0.0f, mp, a.eps, f0, yy);
                    f -= f0;
                }
                fl += wj * f * ysc;
            }
            if (wantS) {
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    float4 t = av[0][v];
#pragma unroll
                    for (int k = 1; k < D; ++k) t = f4mul(t, av[k][v]);
                    gsl[v].x += yw * t.x;
                    gsl[v].y += yw * t.y;
                    gsl[v].z += yw * t.z;
                    gsl[v].w += yw * t.w;
                }
            }
            if (wantG && okj) {
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const int hj = rv[D + k];
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        if (!vact[v]) continue;
                        float4 c = f4scale(sv[v], yw);
#pragma unroll
                        for (int n = 0; n < D; ++n)
                            if (n != k) c = f4mul(c, av[n][v]);
                        if (hj >= 0) {
                            const int jj = j0 + 4 * v;
                            atomicAdd(hacc + hot_pos(k, hj, nhot, RP, jj + 0), c.x);
                            atomicAdd(hacc + hot_pos(k, hj, nhot, RP, jj + 1), c.y);
                            atomicAdd(hacc + hot_pos(k, hj, nhot, RP, jj + 2), c.z);
                            atomicAdd(hacc + hot_pos(k, hj, nhot, RP, jj + 3), c.w);
                        } else {
                            red_add_f4(a.G[k] + off[k] + 4 * v, c);
                        }
                    }
                }
            }
        }
    }

    if (errb) set_err(a.err, errb);
    // temporal gradient: reduce over the groups of the warp, then the block
    if (wantS) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
#pragma unroll
            for (int o = G; o < 32; o <<= 1) {
                gsl[v].x += __shfl_xor_sync(SGCP_FULL_MASK, gsl[v].x, o);
                gsl[v].y += __shfl_xor_sync(SGCP_FULL_MASK, gsl[v].y, o);
                gsl[v].z += __shfl_xor_sync(SGCP_FULL_MASK, gsl[v].z, o);
                gsl[v].w += __shfl_xor_sync(SGCP_FULL_MASK, gsl[v].w, o);
            }
            if (grp == 0 && vact[v]) {
                atomicAdd(gsb + j0 + 4 * v + 0, gsl[v].x);
                atomicAdd(gsb + j0 + 4 * v + 1, gsl[v].y);
                atomicAdd(gsb + j0 + 4 * v + 2, gsl[v].z);
                atomicAdd(gsb + j0 + 4 * v + 3, gsl[v].w);
            }
        }
    }
    if (wantF) {
        double fd = (double)fl;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) fd += __shfl_xor_sync(SGCP_FULL_MASK, fd, o);
        if (lane == 0) fb[warp] = fd;
    }
    __syncthreads();
    if (nhot) {   // one 16-byte reduction per four columns of a hot row (the rows are R-aligned, R % 4 == 0)
        constexpr int QPR = RP / 4;
        for (int i = threadIdx.x; i < D * nhot * QPR; i += blockDim.x) {
            const int k = i / (nhot * QPR), rem = i - k * nhot * QPR;
            const int slot = rem / QPR, j = (rem - slot * QPR) * 4;
            if (j >= R) continue;
            const float4 t = make_float4(hacc[hot_pos(k, slot, nhot, RP, j)], hacc[hot_pos(k, slot, nhot, RP, j + 1)],
                                         hacc[hot_pos(k, slot, nhot, RP, j + 2)], hacc[hot_pos(k, slot, nhot, RP, j + 3)]);
            const int row = a.hot_rows[k * kMaxHot + slot];
            if (row >= 0 && (t.x != 0.f || t.y != 0.f || t.z != 0.f || t.w != 0.f))
                red_add_f4(a.G[k] + (int64_t)row * R + j, t);
        }
    }
    if (wantS) {
        for (int j = threadIdx.x; j < R; j += blockDim.x)
            if (gsb[j] != 0.0f) atomicAdd(a.gs + j, gsb[j]);
    }
    if (wantF && threadIdx.x == 0) {
        double tot = 0.0;
        for (int i = 0; i < wpb; ++i) tot += fb[i];
        if (tot != 0.0) atomicAdd(a.f, tot);
    }
    // temporal solver: the last block applies the ADAM step to s (Alg. 3)
    if (a.tstep_on && last_block_ticket(a.tstep.st)) temporal_step_tail<float>(a.tstep, a.gs, R);
}

template <int D>
__global__ void k_sample_coords(const SparseGradArgs a) {
    const SliceDesc sd = a.slice ? *a.slice : a.inline_slice;
    const DrawSizes z = draw_sizes(a, sd);
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < z.total; c += (int64_t)gridDim.x * blockDim.x) {
        int ci[D];
        float x, w;
        int att, errb = 0;
        bool ok;
        gen_sample<D>(a, sd, z, c, ci, x, w, att, ok, errb);
        if (errb) set_err(a.err, errb);
#pragma unroll
        for (int k = 0; k < D; ++k) a.coords_out[c * D + k] = ok ? ci[k] : -1;
        if (a.attempt_out) a.attempt_out[c] = att;
    }
}

// ---------------------------------------------------------------------------
// Ingest: validate coordinates, insert linear keys into the hash, and count a
// strided subsample of nonzeros per row for the hot-row choice.
// ---------------------------------------------------------------------------
template <int D>
__global__ void k_ingest(const IngestArgs a) {
    const SliceDesc sd = a.slice;
    const unsigned long long mask = (1ull << a.hlog2) - 1ull;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < sd.nnz; e += (int64_t)gridDim.x * blockDim.x) {
        int c[D];
        bool bad = false;
        unsigned long long key = 0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            c[k] = sd.idx[e * D + k];
            if (c[k] < 0 || (int64_t)c[k] >= a.dims[k]) bad = true;
            key = key * (unsigned long long)a.dims[k] + (unsigned long long)(unsigned)c[k];
        }
        if (bad) {
            set_err(a.err, ERRB_COORD);
            continue;
        }
        unsigned long long h = hash_home(key, a.hlog2);
        for (unsigned long long probe = 0;; ++probe) {
            if (probe > mask) {
                set_err(a.err, ERRB_HASH);
                break;
            }
            const unsigned long long prev = atomicCAS(a.hkeys + h, kEmpty, key);
            if (prev == kEmpty) break;
            if (prev == key) {
                set_err(a.err, ERRB_DUP);
                break;
            }
            h = (h + 1ull) & mask;
        }
        if (e % a.sub_stride == 0) {
#pragma unroll
            for (int k = 0; k < D; ++k) atomicAdd(a.counts + a.row_off[k] + c[k], 1);
        }
    }
}

__device__ int block_sum_int(int v, int* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(SGCP_FULL_MASK, v, off);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    int tot = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += red[i];
    return tot;
}

__device__ int block_max_int(int v, int* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = max(v, __shfl_xor_sync(SGCP_FULL_MASK, v, off));
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    int m = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = max(m, red[i]);
    return m;
}

// One block per mode: the nhot rows with the largest subsample counts (at
// least kMinHot) get a shared-memory accumulator slot in the fused kernel.
__global__ void k_hot_select(const IngestArgs a) {
    constexpr int kMinHot = 4;
    __shared__ int red[32];
    __shared__ int nslot;
    const int k = blockIdx.x;
    const int64_t I = a.dims[k];
    const int32_t* cnt = a.counts + a.row_off[k];
    int mx = 0;
    for (int64_t r = threadIdx.x; r < I; r += blockDim.x) mx = max(mx, cnt[r]);
    mx = block_max_int(mx, red);
    int lo = kMinHot, hi = max(mx + 1, kMinHot);
    while (lo < hi) {
        const int mid = lo + (hi - lo) / 2;
        int n = 0;
        for (int64_t r = threadIdx.x; r < I; r += blockDim.x) n += cnt[r] >= mid;
        n = block_sum_int(n, red);
        if (n <= a.nhot) hi = mid;
        else lo = mid + 1;
    }
    if (threadIdx.x == 0) nslot = 0;
    __syncthreads();
    for (int64_t r = threadIdx.x; r < I; r += blockDim.x) {
        if (cnt[r] >= lo) {
            const int slot = atomicAdd(&nslot, 1);
            if (slot < a.nhot) {
                a.hot[a.row_off[k] + r] = slot;
                a.hot_rows[k * kMaxHot + slot] = (int32_t)r;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static int num_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

cudaError_t launch_ingest(const IngestArgs& a, int64_t nnz, cudaStream_t st, int64_t* launches) {
    const int threads = 256;
    int64_t want = (nnz + threads - 1) / threads;
    const int blocks = (int)(want < 1 ? 1 : (want > 8 * num_sms() ? 8 * num_sms() : want));
    switch (a.ndim) {
        case 2: k_ingest<2><<<blocks, threads, 0, st>>>(a); break;
        case 3: k_ingest<3><<<blocks, threads, 0, st>>>(a); break;
        case 4: k_ingest<4><<<blocks, threads, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    if (a.nhot > 0) {
        k_hot_select<<<a.ndim, 1024, 0, st>>>(a);
        if (launches) *launches += 1;
    }
    if (launches) *launches += 1;
    return cudaGetLastError();
}

template <int D, int RP, int CPL, bool WG = true>
static cudaError_t run_sparse(const SparseGradArgs& a, int64_t total, cudaStream_t st) {
    const int threads = 256;
    const int nhot = (a.want & SGCP_WANT_FACTORS) ? a.nhot : 0;
    const size_t smem = (size_t)(D * nhot * RP + RP) * sizeof(float) + 8 * sizeof(double);
    static int occ = 0;
    static size_t occ_smem = 0;
    if (occ == 0 || occ_smem != smem) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_sparse_grad<D, RP, CPL, WG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sparse_grad<D, RP, CPL, WG>, threads, smem);
        if (occ < 1) occ = 1;
        occ_smem = smem;
    }
    const int64_t chunks = (total + 31) / 32;
    int64_t want = (chunks + (threads / 32) - 1) / (threads / 32);
    const int64_t cap = (int64_t)occ * num_sms();
    const int blocks = (int)(want < 1 ? 1 : (want > cap ? cap : want));
    if (a.overlap) return launch_after_prev(k_sparse_grad<D, RP, CPL, WG>, dim3(blocks), dim3(threads), smem, st, a);
    k_sparse_grad<D, RP, CPL, WG><<<blocks, threads, smem, st>>>(a);
    return cudaGetLastError();
}

// Columns per lane: 4 when the kernel scatters factor rows (more lanes issue
// the atomics), 8 for the gather-only temporal / loss launches; a nonzero
// a.cpl (4, 8, 16) overrides the choice.  Defaults measured on GB300 with
// the 10000 x 5000 x 2000, R = 32 workload.
template <int D, int RP>
static cudaError_t run_sparse_cpl(const SparseGradArgs& a, int64_t total, cudaStream_t st) {
    if (a.cpl == 0 && !(a.want & SGCP_WANT_FACTORS))   // gather-only launches at the default width
        return run_sparse<D, RP, (RP >= 16 ? 8 : 4), false>(a, total, st);
    int cpl = a.cpl ? a.cpl : ((a.want & SGCP_WANT_FACTORS) ? 4 : (RP >= 16 ? 8 : 4));
    if (cpl > RP) cpl = RP;
    if (RP / cpl > 32) cpl = RP / 32;
    if (cpl >= 16 && RP >= 16) return run_sparse<D, RP, (RP >= 16 ? 16 : 4)>(a, total, st);
    if (cpl >= 8 && RP >= 8) return run_sparse<D, RP, (RP >= 8 ? 8 : 4)>(a, total, st);
    return run_sparse<D, RP, (RP / 4 <= 32 ? 4 : 8)>(a, total, st);
}

template <int D>
static cudaError_t dispatch_rank(const SparseGradArgs& a, int64_t total, cudaStream_t st) {
    if (a.R <= 4) return run_sparse_cpl<D, 4>(a, total, st);
    if (a.R <= 8) return run_sparse_cpl<D, 8>(a, total, st);
    if (a.R <= 16) return run_sparse_cpl<D, 16>(a, total, st);
    if (a.R <= 32) return run_sparse_cpl<D, 32>(a, total, st);
    if (a.R <= 64) return run_sparse_cpl<D, 64>(a, total, st);
    return run_sparse_cpl<D, 128>(a, total, st);
}

cudaError_t launch_sparse_grad(const SparseGradArgs& a, int64_t total, cudaStream_t st, int64_t* launches) {
    if (launches) *launches += 1;
    switch (a.ndim) {
        case 2: return dispatch_rank<2>(a, total, st);
        case 3: return dispatch_rank<3>(a, total, st);
        case 4: return dispatch_rank<4>(a, total, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sample_coords(const SparseGradArgs& a, int64_t total, cudaStream_t st, int64_t* launches) {
    const int threads = 256;
    int64_t want = (total + threads - 1) / threads;
    const int blocks = (int)(want < 1 ? 1 : (want > 8 * num_sms() ? 8 * num_sms() : want));
    if (launches) *launches += 1;
    switch (a.ndim) {
        case 2: k_sample_coords<2><<<blocks, threads, 0, st>>>(a); break;
        case 3: k_sample_coords<3><<<blocks, threads, 0, st>>>(a); break;
        case 4: k_sample_coords<4><<<blocks, threads, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace sgcp

namespace sgcp {

// Hash-only slice ingest used by the no-allocation gradient entry point:
// checks coordinates and inserts the linear keys into a caller-provided
// table (already cleared to all ones); no row histograms.
template <int D>
__global__ void k_hash_build(SliceDesc sd, int64_t d0, int64_t d1, int64_t d2, int64_t d3,
                             unsigned long long* keys, int hlog2, int* err) {
    const int64_t dims[4] = {d0, d1, d2, d3};
    const unsigned long long mask = (1ull << hlog2) - 1ull;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < sd.nnz; e += (int64_t)gridDim.x * blockDim.x) {
        bool bad = false;
        unsigned long long key = 0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const int c = sd.idx[e * D + k];
            if (c < 0 || (int64_t)c >= dims[k]) bad = true;
            key = key * (unsigned long long)dims[k] + (unsigned long long)(unsigned)c;
        }
        if (bad) {
            set_err(err, ERRB_COORD);
            continue;
        }
        unsigned long long h = hash_home(key, hlog2);
        for (unsigned long long probe = 0;; ++probe) {
            if (probe > mask) {
                set_err(err, ERRB_HASH);
                break;
            }
            const unsigned long long prev = atomicCAS(keys + h, kEmpty, key);
            if (prev == kEmpty) break;
            if (prev == key) {
                set_err(err, ERRB_DUP);
                break;
            }
            h = (h + 1ull) & mask;
        }
    }
}

cudaError_t launch_hash_build(const SliceDesc& sd, int ndim, const int64_t* dims, unsigned long long* keys, int hlog2,
                              int* err, cudaStream_t st) {
    const int threads = 256;
    const int64_t want = (sd.nnz + threads - 1) / threads;
    const int blocks = (int)(want < 1 ? 1 : (want > 8 * num_sms() ? 8 * num_sms() : want));
    const int64_t d3 = ndim > 3 ? dims[3] : 1, d2 = ndim > 2 ? dims[2] : 1;
    switch (ndim) {
        case 2: k_hash_build<2><<<blocks, threads, 0, st>>>(sd, dims[0], dims[1], d2, d3, keys, hlog2, err); break;
        case 3: k_hash_build<3><<<blocks, threads, 0, st>>>(sd, dims[0], dims[1], d2, d3, keys, hlog2, err); break;
        case 4: k_hash_build<4><<<blocks, threads, 0, st>>>(sd, dims[0], dims[1], d2, d3, keys, hlog2, err); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace sgcp
