// Batched streams: many independent OnlineGCP streams (dense 3-way FP32
// slices of uneven shape, rank and loss) advanced by ONE persistent kernel per
// time step.  Every stream runs the whole Alg. 1 body of arXiv 2110.14514:
// Alg. 3 temporal ADAM epochs, Alg. 4 factor ADAM epochs with the history
// penalty of eq. spatial_gcp_grad, Alg. 2 checkpoints and rollbacks, then
// Abar <- A and the reservoir slot update.
//
// Phase program of one stream (identical arithmetic to the single-stream step):
//   p = 0                        PRE     1 unit; tail: S_H, temporal ADAM init (s = 0), solver init
//   p = 1                        LOSS_W  slice-loss units; tail: F_w, begin epoch 0
//   p = 2 + e (tau_w+1) + j      TGRAD   gradient-of-s units; tail: ADAM step on s      (j < tau_w)
//                                LOSS_W  slice-loss units; tail: epoch end, next begin   (j = tau_w)
//   p = PF0                      LOSS_F  slice-loss + Gram-chunk units; tail: F_f, begin epoch 0
//   p = PF0 + 1 + e (2 tau_f+1) + q
//                                FGRAD   factor-gradient + (A'A, D'A) Gram units; tail: B_k, C_k (q = 2j)
//                                UPD     32-row chunks: g = G + lambda A + D B_k + Abar C_k, ADAM (q = 2j+1)
//                                LOSS_F  objective, epoch end, next begin                 (q = 2 tau_f)
//   after the last tail          Abar <- A, history slot <- s_t
// A solver whose loop test fails (F <= tol) jumps to the next solver.
//
// Gradient units are boxes of 64-row x 32-column tiles (dense_tile.cuh).
//
// Scheduling.  A stream's claim word holds (phase << 32 | next unit); a block
// takes a unit with one atomicAdd.  The block that completes the phase's last
// unit runs the tail and publishes the next phase.  So streams advance
// independently, a block never waits for a particular block, and the only
// waits are polls for work, bounded by spin_limit (ERRB_TIMEOUT).  Data that
// another block may have written during the launch is read through L2
// (ld.global.cg), and each block fences its writes before it counts a unit
// done, so the tail and the next phase see them.
#include "dense_tile.cuh"
#include "internal.h"
#include "sgcp.h"

namespace sgcp {

namespace {

enum PhaseKind : int { PH_PRE = 0, PH_LOSS_W = 1, PH_TGRAD = 2, PH_LOSS_F = 3, PH_FGRAD = 4, PH_UPD = 5 };

struct PhaseInfo {
    int kind;
    int e;      // epoch (-1 for the initial objective)
    int it;     // iteration within the epoch
};

__device__ __forceinline__ PhaseInfo phase_of(const BatchStream& S, int p) {
    PhaseInfo ph{PH_PRE, -1, 0};
    if (p == 0) return ph;
    if (p == 1) {
        ph.kind = PH_LOSS_W;
        return ph;
    }
    if (p < S.PF0) {
        const int q = p - 2, per = S.tau_w + 1;
        ph.e = q / per;
        ph.it = q - ph.e * per;
        ph.kind = ph.it < S.tau_w ? PH_TGRAD : PH_LOSS_W;
        return ph;
    }
    if (p == S.PF0) {
        ph.kind = PH_LOSS_F;
        return ph;
    }
    const int q = p - S.PF0 - 1, per = 2 * S.tau_f + 1;
    ph.e = q / per;
    const int r = q - ph.e * per;
    if (r == 2 * S.tau_f) {
        ph.kind = PH_LOSS_F;
        ph.it = S.tau_f;
    } else {
        ph.kind = (r & 1) ? PH_UPD : PH_FGRAD;
        ph.it = r >> 1;
    }
    return ph;
}

__device__ __forceinline__ int units_of(const BatchStream& S, const BatchStepEntry& E, int kind) {
    switch (kind) {
        case PH_PRE: return 1;
        case PH_LOSS_W:
        case PH_TGRAD: return S.n_box;
        case PH_LOSS_F: return S.n_box + S.n_gram;
        case PH_FGRAD: return S.n_box + (E.hist_on ? S.n_gram : 0);
        default: return S.n_upd;
    }
}

// Shared memory of one block (floats): the gradient-unit plan of dense_tile.cuh;
// Gram and update units reuse the front of the same buffer.
constexpr int kSmemFloats = kBoxSmemFloats;
static_assert(2 * kBatchGramRows * kBatchMaxR + kBatchMaxR * kBatchMaxR <= kSmemFloats, "Gram unit staging");
static_assert(2 * kBatchMaxR * kBatchMaxR <= kSmemFloats, "update unit coefficients");

// Gradient unit u of a stream: one box of the slice (dense_tile.cuh) with the
// loss, the gradient of s or the factor gradients selected by the phase.
__device__ void box_unit(const BatchStream& S, const float* __restrict__ X, int kind, SolverState* st_obj, int u,
                         float* sm) {
    const int R = S.R;
    const int B1 = 1 << S.b1log, B2 = 64 >> S.b1log;
    const int nb12 = S.nb1 * S.nb2;
    const int b3 = u / nb12, rem = u - b3 * nb12;
    const int bb1 = rem / S.nb2, bb2 = rem - bb1 * S.nb2;
    BoxGeom g;
    g.R = R;
    g.loss = S.loss;
    g.eps = S.eps;
    g.I1 = S.dims[0];
    g.I2 = S.dims[1];
    g.I3 = S.dims[2];
    g.lb1 = S.b1log;
    g.n1 = S.n1;
    g.n2 = S.n2;
    g.o1 = bb1 * B1 * S.n1;
    g.o2 = bb2 * B2 * S.n2;
    g.o3 = b3 * 32;
    g.A1 = S.A;
    g.A2 = S.A + (int64_t)S.row_off[1] * R;
    g.A3 = S.A + (int64_t)S.row_off[2] * R;
    g.s = S.s;
    g.X = X;
    g.G1 = S.G;
    g.G2 = S.G + (int64_t)S.row_off[1] * R;
    g.G3 = S.G + (int64_t)S.row_off[2] * R;
    g.gs = S.gs;
    g.f = st_obj ? &st_obj->F_new : nullptr;
    g.ysc = 1.0f;
    const int want = kind == PH_FGRAD ? SGCP_WANT_FACTORS : (kind == PH_TGRAD ? SGCP_WANT_TEMPORAL : SGCP_WANT_LOSS);
    dense_box_any(g, want, sm);
}

// Gram pair list of a unit: npairs = 1 -> (A,A); 2 -> (A,A), (D,A);
// 6 -> (A,A), (Abar,Abar), (Abar,A), (D,D), (D,A), (Abar,D).
__device__ __forceinline__ void pair_sel(int npairs, int pr, int& su, int& svv) {
    if (npairs == 2) {
        su = pr == 0 ? SEL_A : SEL_D;
        svv = SEL_A;
        return;
    }
    // 2-bit selectors, pair pr at bits 2pr: U = (A, Abar, Abar, D, D, Abar), V = (A, Abar, A, D, A, D)
    constexpr int kU = SEL_A | SEL_ABAR << 2 | SEL_ABAR << 4 | SEL_D << 6 | SEL_D << 8 | SEL_ABAR << 10;
    constexpr int kV = SEL_A | SEL_ABAR << 2 | SEL_A << 4 | SEL_D << 6 | SEL_A << 8 | SEL_D << 10;
    su = (kU >> (2 * pr)) & 3;
    svv = (kV >> (2 * pr)) & 3;
}

__device__ __forceinline__ float pick(int sel, float a, float ab) {
    return sel == SEL_A ? a : (sel == SEL_ABAR ? ab : a - ab);
}

// Gram-chunk unit g: partial Gram(U, V) over rows [64c, 64c + 64) of one
// mode, for the phase's pairs, written to gpart[g][pair] (summed by the tail).
__device__ void gram_unit(const BatchStream& S, int g, int npairs, float* sm) {
    const int R = S.R, RR = R * R, tid = threadIdx.x;
    int k = 0, c = g;
    while (k < 2 && c >= S.gch[k]) c -= S.gch[k++];
    const int r0 = c * kBatchGramRows;
    const int nr = min(kBatchGramRows, S.dims[k] - r0);
    float* Us = sm;                               // [64][R] rows of A
    float* Vs = sm + kBatchGramRows * kBatchMaxR; // [64][R] rows of Abar
    float* red = Vs + kBatchGramRows * kBatchMaxR;
    const int64_t base = ((int64_t)S.row_off[k] + r0) * R;
    for (int i = tid; i < nr * R; i += kBatchThreads) {
        Us[i] = __ldcg(S.A + base + i);
        Vs[i] = __ldcg(S.Abar + base + i);
    }
    const int tq = R >> 2, tiles = tq * tq;
    const int groups = kBatchThreads / tiles;
    const int grp = tid / tiles, tile = tid - grp * tiles;
    const bool act = grp < groups;
    const int tl = tile / tq, tm = tile - tl * tq;
    for (int pp = 0; pp < npairs; pp += 3) {
        float acc[3][4][4];
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[q][x][y] = 0.f;
        int su[3], svv[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            su[q] = SEL_A;
            svv[q] = SEL_A;
            if (pp + q < npairs) pair_sel(npairs, pp + q, su[q], svv[q]);
        }
        __syncthreads();
        if (act) {
            for (int r = grp; r < nr; r += groups) {
                float al[4], bl[4], am[4], bm[4];
#pragma unroll
                for (int x = 0; x < 4; ++x) {
                    al[x] = Us[r * R + tl * 4 + x];
                    bl[x] = Vs[r * R + tl * 4 + x];
                    am[x] = Us[r * R + tm * 4 + x];
                    bm[x] = Vs[r * R + tm * 4 + x];
                }
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    if (pp + q >= npairs) break;
#pragma unroll
                    for (int x = 0; x < 4; ++x) {
                        const float uu = pick(su[q], al[x], bl[x]);
#pragma unroll
                        for (int y = 0; y < 4; ++y) acc[q][x][y] += uu * pick(svv[q], am[y], bm[y]);
                    }
                }
            }
        }
        for (int q = 0; q < 3 && pp + q < npairs; ++q) {
            __syncthreads();
            if (act)
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) red[grp * RR + (tl * 4 + x) * R + tm * 4 + y] = acc[q][x][y];
            __syncthreads();
            float* out = S.gpart + ((int64_t)g * 6 + pp + q) * RR;
            for (int i = tid; i < RR; i += kBatchThreads) {
                float sum = 0.f;
                for (int gg = 0; gg < groups; ++gg) sum += red[gg * RR + i];
                out[i] = sum;
            }
        }
    }
}

// Factor-update unit: rows [32c, 32c + 32) of one mode.  g = G + lambda a +
// d B_k + abar C_k (the collapsed history gradient), ADAM step with the
// iteration's bias-corrected rate, projection a <- max(a, l), G <- 0.
// Warp per row; lane l holds columns l and l + 32.
__device__ void upd_unit(const BatchStream& S, const BatchStepEntry& E, int u, int it, float* sm) {
    const int R = S.R, RR = R * R, tid = threadIdx.x;
    int k = 0, c = u;
    while (k < 2 && c >= S.uch[k]) c -= S.uch[k++];
    const int r0 = c * kBatchUpdRows;
    const int r1 = min(r0 + kBatchUpdRows, S.dims[k]);
    const bool hist = E.hist_on != 0;
    float* Bs = sm;
    float* Cs = sm + kBatchMaxR * kBatchMaxR;
    if (hist)
        for (int i = tid; i < RR; i += kBatchThreads) {
            Bs[i] = __ldcg(S.Bc + k * RR + i);
            Cs[i] = __ldcg(S.Cc + k * RR + i);
        }
    __syncthreads();
    const float rate = (float)__ldcg(S.rates_f + it);
    const float b1 = (float)S.beta1, b2 = (float)S.beta2, c1 = (float)(1.0 - S.beta1), c2 = (float)(1.0 - S.beta2);
    const float lam = (float)S.lam, eps = (float)S.adam_eps, lower = S.lower;
    const int lane = tid & 31, warp = tid >> 5;
    const int R0 = R < 32 ? R : 32;
    for (int r = r0 + warp; r < r1; r += kBatchThreads / 32) {
        const int64_t rowb = ((int64_t)S.row_off[k] + r) * R;
        float av[2], bv[2], dv[2], g[2], uo[2], vo[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int j = lane + 32 * q;
            const bool on = j < R;
            av[q] = on ? __ldcg(S.A + rowb + j) : 0.f;
            bv[q] = on ? __ldcg(S.Abar + rowb + j) : 0.f;
            g[q] = on ? __ldcg(S.G + rowb + j) : 0.f;
            uo[q] = on ? __ldcg(S.u + rowb + j) : 0.f;
            vo[q] = on ? __ldcg(S.v + rowb + j) : 0.f;
            dv[q] = av[q] - bv[q];
            g[q] += lam * av[q];
        }
        if (hist) {
            float sb[2] = {0.f, 0.f}, sc[2] = {0.f, 0.f};
            for (int l = 0; l < R0; ++l) {
                const float dl = __shfl_sync(SGCP_FULL_MASK, dv[0], l);
                const float bl = __shfl_sync(SGCP_FULL_MASK, bv[0], l);
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int j = lane + 32 * q;
                    if (j < R) {
                        sb[q] += dl * Bs[l * R + j];
                        sc[q] += bl * Cs[l * R + j];
                    }
                }
            }
            for (int l = 32; l < R; ++l) {
                const float dl = __shfl_sync(SGCP_FULL_MASK, dv[1], l - 32);
                const float bl = __shfl_sync(SGCP_FULL_MASK, bv[1], l - 32);
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int j = lane + 32 * q;
                    if (j < R) {
                        sb[q] += dl * Bs[l * R + j];
                        sc[q] += bl * Cs[l * R + j];
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) g[q] += sb[q] + sc[q];
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int j = lane + 32 * q;
            if (j >= R) continue;
            const float uu = b1 * uo[q] + c1 * g[q];
            const float vv = b2 * vo[q] + c2 * g[q] * g[q];
            float an = av[q] - rate * uu / (sqrtf(vv) + eps);
            if (an < lower) an = lower;
            S.u[rowb + j] = uu;
            S.v[rowb + j] = vv;
            S.A[rowb + j] = an;
            S.G[rowb + j] = 0.f;
        }
    }
}

// ---------------------------------------------------------------------------
// Tails (one block, serial per stream).  Each returns the next phase.
// ---------------------------------------------------------------------------
__device__ void tail_obj_w(const BatchStream& S, int set_cur, int* err) {
    if (threadIdx.x == 0) {
        double ss = 0.0;
        for (int j = 0; j < S.R; ++j) {
            const double v = (double)__ldcg(S.s + j);
            ss += v * v;
        }
        const double F = __ldcg(&S.st_w->F_new) + 0.5 * S.mu * ss;
        S.st_w->F_new = F;
        if (!isfinite(F)) set_err(err, ERRB_NUMERIC);
        if (set_cur) S.st_w->F_cur = F;
    }
    __syncthreads();
}

// Alg. 2 Update for a solver over n elements, run by the whole block.
__device__ void tail_epoch_end(SolverState* st, int64_t n, float* a, float* u, float* v, float* a_o, float* u_o,
                               float* v_o, int tau, const BatchStream& S) {
    const bool passed = epoch_passed(st);
    for (int64_t i = threadIdx.x; i < n; i += kBatchThreads) epoch_end_elem(passed, i, a, u, v, a_o, u_o, v_o);
    __syncthreads();
    if (threadIdx.x == 0) epoch_end_state(st, passed, tau, S.decay, S.beta1, S.beta2);
    __syncthreads();
}

// Epoch begin; returns whether the solver's loop test failed (skip the rest).
__device__ bool tail_epoch_begin(SolverState* st, double tol, double* rates, int tau, const BatchStream& S,
                                 int* flag) {
    epoch_begin_block(st, tol, rates, tau, S.beta1, S.beta2);
    __syncthreads();
    if (threadIdx.x == 0) *flag = __ldcg(&st->done);
    __syncthreads();
    return *flag != 0;
}

// grams[pr][k] = sum of the mode's chunk partials (double).
__device__ void tail_gram_reduce(const BatchStream& S, int npairs) {
    const int RR = S.R * S.R;
    for (int idx = threadIdx.x; idx < npairs * 3 * RR; idx += kBatchThreads) {
        const int i = idx % RR, pk = idx / RR, k = pk % 3, pr = pk / 3;
        int g0 = 0;
        for (int q = 0; q < k; ++q) g0 += S.gch[q];
        double sum = 0.0;
        for (int c = 0; c < S.gch[k]; ++c) sum += (double)__ldcg(S.gpart + ((int64_t)(g0 + c) * 6 + pr) * RR + i);
        S.grams[((int64_t)pr * 3 + k) * RR + i] = sum;
    }
    __syncthreads();
}

__device__ void tail_finish(const BatchStream& S, const BatchStepEntry& E) {
    for (int i = threadIdx.x; i < S.N; i += kBatchThreads) S.Abar[i] = __ldcg(S.A + i);
    if (E.slot >= 0) {
        for (int j = threadIdx.x; j < S.R; j += kBatchThreads) S.s_hist[(int64_t)E.slot * S.R + j] = __ldcg(S.s + j);
        if (threadIdx.x == 0) {
            S.h_dev[E.slot] = E.t;
            *S.hist_len = E.len;
        }
    }
    __syncthreads();
}

__device__ int run_tail(const BatchStream& S, const BatchStepEntry& E, int p, const PhaseInfo& ph, int* err,
                        int* flag) {
    const int R = S.R, RR = R * R, tid = threadIdx.x;
    switch (ph.kind) {
        case PH_PRE: {
            const int n = __ldcg(S.hist_len);
            for (int i = tid; i < RR; i += kBatchThreads)
                S.SH[i] = history_SH_elem<float>(R, S.s_hist, S.h_dev, n, E.t, S.w, S.theta, i);
            for (int j = tid; j < R; j += kBatchThreads) {   // Alg. 3 starts from s = 0
                S.s[j] = 0.f;
                S.s_u[j] = 0.f;
                S.s_v[j] = 0.f;
                S.s_uo[j] = 0.f;
                S.s_vo[j] = 0.f;
                S.s_ao[j] = 0.f;
                S.gs[j] = 0.f;
            }
            if (tid == 0) solver_init_state(S.st_w, S.alpha_w, 1);
            __syncthreads();
            return 1;
        }
        case PH_TGRAD: {   // g = Z'y + mu s; ADAM step on s (Alg. 3, Alg. 2 Step)
            const float rate = (float)__ldcg(S.rates_w + ph.it);
            for (int j = tid; j < R; j += kBatchThreads) {
                const float sj = __ldcg(S.s + j);
                const float g = __ldcg(S.gs + j) + (float)S.mu * sj;
                const float u = (float)S.beta1 * __ldcg(S.s_u + j) + (float)(1.0 - S.beta1) * g;
                const float v = (float)S.beta2 * __ldcg(S.s_v + j) + (float)(1.0 - S.beta2) * g * g;
                float sn = sj - rate * u / (sqrtf(v) + (float)S.adam_eps);
                if (sn < S.lower) sn = S.lower;
                S.s_u[j] = u;
                S.s_v[j] = v;
                S.s[j] = sn;
                S.gs[j] = 0.f;
            }
            __syncthreads();
            return p + 1;
        }
        case PH_LOSS_W: {
            const bool init = ph.e < 0;
            tail_obj_w(S, init ? 1 : 0, err);
            int e_next = 0;
            if (!init) {
                tail_epoch_end(S.st_w, R, S.s, S.s_u, S.s_v, S.s_ao, S.s_uo, S.s_vo, S.tau_w, S);
                e_next = ph.e + 1;
            }
            if (e_next < S.kappa_w && !tail_epoch_begin(S.st_w, S.tol_w, S.rates_w, S.tau_w, S, flag)) return p + 1;
            if (tid == 0) solver_init_state(S.st_f, S.alpha_f, 0);   // on to the factor solver (Alg. 4)
            __syncthreads();
            return S.PF0;
        }
        case PH_LOSS_F: {
            const bool init = ph.e < 0;
            tail_gram_reduce(S, E.hist_on ? 6 : 1);
            obj_finish_f_block(S.st_f, 3, R, S.grams, S.SH, E.hist_on != 0, S.lam, init ? 1 : 0, err);
            int e_next = 0;
            if (!init) {
                tail_epoch_end(S.st_f, S.N, S.A, S.u, S.v, S.a_o, S.u_o, S.v_o, S.tau_f, S);
                e_next = ph.e + 1;
            }
            if (e_next < S.kappa_f && !tail_epoch_begin(S.st_f, S.tol_f, S.rates_f, S.tau_f, S, flag)) return p + 1;
            tail_finish(S, E);
            return S.P;
        }
        case PH_FGRAD: {
            if (E.hist_on) {
                tail_gram_reduce(S, 2);
                for (int i = tid; i < RR; i += kBatchThreads)
                    hist_coeff_elem<float>(3, RR, S.grams, S.grams + 3 * RR, S.SH, i, true, S.Bc, S.Cc);
                __syncthreads();
            }
            return p + 1;
        }
        default:
            return p + 1;
    }
}

__device__ void run_unit(const BatchStream& S, const BatchStepEntry& E, const PhaseInfo& ph, int u, float* sm) {
    switch (ph.kind) {
        case PH_PRE: return;
        case PH_LOSS_W: box_unit(S, E.X, ph.kind, S.st_w, u, sm); return;
        case PH_TGRAD: box_unit(S, E.X, ph.kind, nullptr, u, sm); return;
        case PH_LOSS_F:
            if (u < S.n_box) box_unit(S, E.X, ph.kind, S.st_f, u, sm);
            else gram_unit(S, u - S.n_box, E.hist_on ? 6 : 1, sm);
            return;
        case PH_FGRAD:
            if (u < S.n_box) box_unit(S, E.X, ph.kind, nullptr, u, sm);
            else gram_unit(S, u - S.n_box, 2, sm);
            return;
        default: upd_unit(S, E, u, ph.it, sm); return;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// The persistent step kernel.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBatchThreads, 2) k_batch_step(const BatchArgs b) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* sm = reinterpret_cast<float*>(smem_raw);
    __shared__ int c_cmd, c_s, c_p, c_u, c_flag;
    const int tid = threadIdx.x, lane = tid & 31;
    long long idle = 0;
    unsigned ns = 32;
    for (;;) {
        __syncthreads();   // everyone is done with the previous command
        if (tid < 32) {
            // warp 0 scans the streams in priority order; the first with an
            // unclaimed unit of its current phase gets an atomicAdd
            int cmd = 0, ws = 0, wp = 0, wu = 0;
            for (int base = 0; base < b.nS && cmd == 0; base += 32) {
                const int k = base + lane;
                int s = 0;
                bool avail = false;
                if (k < b.nS) {
                    s = b.order[k];
                    const BatchStream& S = b.S[s];
                    const unsigned long long w = __ldcg(&b.ctl[s].claim);
                    const int ph = (int)(w >> 32);
                    if (ph < S.P) avail = (unsigned)w < (unsigned)units_of(S, b.E[s], phase_of(S, ph).kind);
                }
                unsigned m = __ballot_sync(SGCP_FULL_MASK, avail);
                while (m) {
                    const int L = __ffs(m) - 1;
                    int got = 0, gp = 0, gu = 0;
                    if (lane == L) {
                        const BatchStream& S = b.S[s];
                        const unsigned long long old = atomicAdd(&b.ctl[s].claim, 1ull);
                        const int ph = (int)(old >> 32);
                        if (ph < S.P && (unsigned)old < (unsigned)units_of(S, b.E[s], phase_of(S, ph).kind)) {
                            got = 1;
                            gp = ph;
                            gu = (int)(unsigned)old;
                        }
                    }
                    got = __shfl_sync(SGCP_FULL_MASK, got, L);
                    if (got) {
                        ws = __shfl_sync(SGCP_FULL_MASK, s, L);
                        wp = __shfl_sync(SGCP_FULL_MASK, gp, L);
                        wu = __shfl_sync(SGCP_FULL_MASK, gu, L);
                        cmd = 1;
                        break;
                    }
                    m &= m - 1;
                }
            }
            __threadfence();   // acquire: the lane that claimed saw the publishing block's release
            if (lane == 0) {
                if (cmd == 0) {
                    if (__ldcg(b.finished) >= b.nS) {
                        cmd = 2;
                    } else if (++idle > b.spin_limit) {
                        set_err(b.err, ERRB_TIMEOUT);
                        cmd = 2;
                    } else {
                        __nanosleep(ns);
                        if (ns < 1024) ns <<= 1;
                    }
                } else {
                    idle = 0;
                    ns = 32;
                    c_s = ws;
                    c_p = wp;
                    c_u = wu;
                }
                c_cmd = cmd;
            }
        }
        __syncthreads();
        const int cmd = c_cmd;
        if (cmd == 2) break;
        if (cmd == 0) continue;
        const int s = c_s, p = c_p, u = c_u;
        const BatchStream& S = b.S[s];
        const BatchStepEntry& E = b.E[s];
        const PhaseInfo ph = phase_of(S, p);
        run_unit(S, E, ph, u, sm);
        __threadfence();   // this block's results are visible before the unit counts as done
        __syncthreads();
        if (tid == 0) {
            const int prev = atomicAdd(&b.ctl[s].done, 1);
            c_flag = (prev == units_of(S, E, ph.kind) - 1);
            __threadfence();
        }
        __syncthreads();
        if (c_flag) {
            __shared__ int t_flag;
            const int next = run_tail(S, E, p, ph, b.err, &t_flag);
            __threadfence();
            __syncthreads();
            if (tid == 0) {
                b.ctl[s].done = 0;
                __threadfence();
                atomicExch(&b.ctl[s].claim, (unsigned long long)next << 32);
                if (next >= S.P) atomicAdd(b.finished, 1);
            }
        }
    }
}

// Per-step inputs and scheduling words (not part of the captured graph: the
// entries are kernel arguments by value, so no host buffer must outlive the call).
constexpr int kEntriesPerLaunch = 64;
struct EntryChunk {
    BatchStepEntry e[kEntriesPerLaunch];
};

__global__ void k_batch_begin(BatchStepEntry* dE, int off, int n, const EntryChunk chunk, BatchCtl* ctl, int nS,
                              int* finished) {
    const int i = threadIdx.x;
    if (i < n) dE[off + i] = chunk.e[i];
    if (off == 0) {
        for (int s = i; s < nS; s += blockDim.x) {
            ctl[s].claim = 0ull;
            ctl[s].done = 0;
        }
        if (i == 0) *finished = 0;
    }
}

// Timing launch of the autotuner: factor-gradient unit (blockIdx.x mod n_box)
// of one stream description, results added into that description's buffers.
__global__ void __launch_bounds__(kBatchThreads, 2) k_batch_units(const BatchStream* S, const BatchStepEntry* E,
                                                                   int n_box) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    box_unit(*S, E->X, PH_FGRAD, nullptr, (int)(blockIdx.x % (unsigned)n_box), reinterpret_cast<float*>(smem_raw));
}

size_t batch_smem_bytes() { return (size_t)kSmemFloats * sizeof(float); }

int batch_blocks_per_sm() {
    int n = 0;
    const size_t smem = batch_smem_bytes();
    cudaFuncSetAttribute(k_batch_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_step, kBatchThreads, smem);
    return n > 0 ? n : 1;
}

cudaError_t launch_batch_begin(BatchStepEntry* dE, const BatchStepEntry* host_entries, int n, BatchCtl* ctl, int nS,
                               int* finished, cudaStream_t st, int64_t* launches) {
    for (int off = 0; off < n || off == 0; off += kEntriesPerLaunch) {
        EntryChunk ch{};
        const int m = n - off < kEntriesPerLaunch ? n - off : kEntriesPerLaunch;
        for (int i = 0; i < m; ++i) ch.e[i] = host_entries[off + i];
        k_batch_begin<<<1, 128, 0, st>>>(dE, off, m, ch, ctl, nS, finished);
        if (launches) *launches += 1;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (n == 0) break;
    }
    return cudaSuccess;
}

cudaError_t launch_batch_step(const BatchArgs& a, int grid, cudaStream_t st, int64_t* launches) {
    const size_t smem = batch_smem_bytes();
    cudaFuncSetAttribute(k_batch_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_batch_step<<<grid, kBatchThreads, smem, st>>>(a);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_batch_units(const BatchStream* S_dev, const BatchStepEntry* E_dev, int n_box, int blocks,
                               cudaStream_t st) {
    const size_t smem = batch_smem_bytes();
    cudaFuncSetAttribute(k_batch_units, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_batch_units<<<blocks, kBatchThreads, smem, st>>>(S_dev, E_dev, n_box);
    return cudaGetLastError();
}

}  // namespace sgcp
