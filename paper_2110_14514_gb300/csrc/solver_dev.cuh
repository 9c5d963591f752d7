// Device-side solver arithmetic shared by the single-stream kernels
// (k_solver.cu) and the batched persistent kernel (k_batch.cu): Alg. 2
// epoch bookkeeping, the history-penalty coefficients of eq. spatial_gcp_grad
// in collapsed / telescoped form, the telescoped history objective (Alg. 5
// with the model-based penalty of Sec. 4.2) and the history weight matrix S_H.
#pragma once

#include "common.cuh"

namespace sgcp {

// Which factor set a Gram pair uses (A, Abar or D = A - Abar).
enum GramSel : int { SEL_A = 0, SEL_ABAR = 1, SEL_D = 2 };

template <typename T>
__device__ __forceinline__ T gsel(int sel, const T* A, const T* Ab, int64_t i) {
    return sel == SEL_A ? A[i] : (sel == SEL_ABAR ? Ab[i] : A[i] - Ab[i]);
}

// ---------------------------------------------------------------------------
// Alg. 2 bookkeeping on the device-resident SolverState.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void solver_init_state(SolverState* st, double alpha, int reset_counter) {
    st->alpha = alpha;
    st->epoch = 0;
    st->done = 0;
    st->accept = 0u;
    st->ticket = 0u;
    st->F_new = 0.0;
    if (reset_counter) {
        st->i = 0;
        st->b1pow = 1.0;
        st->b2pow = 1.0;
    }
}

// Reads of solver state go through L2 (ld.global.cg): inside one persistent
// kernel the state may have been written by a block on another SM, and L1 is
// not coherent across SMs.

// Epoch start, run by one block: the rates of the epoch's tau iterations, then
// (thread 0) the Alg. 3/4 loop test "while F > tol" and F_old <- F_cur.
__device__ __forceinline__ void epoch_begin_block(SolverState* st, double tol, double* rates, int tau, double beta1,
                                                  double beta2) {
    SolverState s0{};
    s0.alpha = __ldcg(&st->alpha);
    s0.b1pow = __ldcg(&st->b1pow);
    s0.b2pow = __ldcg(&st->b2pow);
    for (int j = threadIdx.x; j < tau; j += blockDim.x) rates[j] = adam_rate(s0, beta1, beta2, j);
    __syncthreads();
    if (threadIdx.x == 0) {
        const double Fc = __ldcg(&st->F_cur);
        if (!__ldcg(&st->done) && !(Fc > tol)) st->done = 1;
        st->F_old = Fc;
        st->F_new = 0.0;
    }
}

// Alg. 2 Update(passed): passed = (F_new <= F_old) and F_new finite.
__device__ __forceinline__ bool epoch_passed(const SolverState* st) {
    const double Fn = __ldcg(&st->F_new), Fo = __ldcg(&st->F_old);
    return !(Fn > Fo) && isfinite(Fn);
}

// Checkpoint (passed) or rollback of element i of (a, u, v).
template <typename T>
__device__ __forceinline__ void epoch_end_elem(bool passed, int64_t i, T* a, T* u, T* v, T* a_o, T* u_o, T* v_o) {
    if (passed) {
        u_o[i] = __ldcg(u + i);
        v_o[i] = __ldcg(v + i);
        a_o[i] = __ldcg(a + i);
    } else {
        u[i] = __ldcg(u_o + i);
        v[i] = __ldcg(v_o + i);
        a[i] = __ldcg(a_o + i);
    }
}

// Scalar part of the epoch end (one thread): an accepted epoch's tau
// iterations count for the bias correction, a rejected one decays alpha.
__device__ __forceinline__ void epoch_end_state(SolverState* st, bool passed, int tau, double decay, double beta1,
                                                double beta2) {
    const int32_t ep = __ldcg(&st->epoch);
    if (passed) {
        st->F_cur = __ldcg(&st->F_new);
        st->accept = __ldcg(&st->accept) | ((ep < 32) ? (1u << ep) : 0u);
        st->i = __ldcg(&st->i) + tau;
        st->b1pow = __ldcg(&st->b1pow) * pow(beta1, (double)tau);
        st->b2pow = __ldcg(&st->b2pow) * pow(beta2, (double)tau);
    } else {
        st->F_cur = __ldcg(&st->F_old);
        st->alpha = __ldcg(&st->alpha) * decay;
    }
    st->epoch = ep + 1;
}

// ---------------------------------------------------------------------------
// History coefficients B_k = Gamma_k * S_H, C_k = (Gamma_k - Gammabar_k) * S_H
// at entry i of the R x R matrices, from P_n = A'A and E_n = D'A.
// Gamma_k - Gammabar_k is telescoped: prod P - prod Q = sum_m (prod_{n<m} Q)
// E_m (prod_{n>m} P), Q = P - E, so nothing cancels when A ~ Abar.
// ---------------------------------------------------------------------------
// B_k and C_k at one entry from that entry's P_n, E_n (n < ndim <= 4) and S_H.
template <typename T>
__device__ __forceinline__ void hist_coeff_k(int ndim, int k, const T (&p)[4], const T (&e)[4], T sh, T& b, T& c) {
    T gam = T(1), dgam = T(0);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        if (m == k || m >= ndim) continue;
        gam *= p[m];
        T term = e[m];
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            if (n == k || n == m || n >= ndim) continue;
            term *= (n < m) ? (p[n] - e[n]) : p[n];
        }
        dgam += term;
    }
    b = gam * sh;
    c = dgam * sh;
}

template <typename T>
__device__ __forceinline__ void hist_coeff_elem(int ndim, int RR, const double* P, const double* E, const double* SH,
                                                int i, bool on, T* B, T* C) {
    T p[4], e[4];
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        p[n] = on && n < ndim ? (T)__ldcg(P + n * RR + i) : T(0);
        e[n] = on && n < ndim ? (T)__ldcg(E + n * RR + i) : T(0);
    }
    const T sh = on ? (T)__ldcg(SH + i) : T(0);
    for (int k = 0; k < ndim; ++k) {
        T b = T(0), c = T(0);
        if (on) hist_coeff_k<T>(ndim, k, p, e, sh, b, c);
        B[k * RR + i] = b;
        C[k * RR + i] = c;
    }
}

// ---------------------------------------------------------------------------
// History objective 1/2 sum_h w_h ||Mbar_h - M_h||^2 in telescoped form:
// M_h - Mbar_h = sum_k [[s_h; Abar^(1..k-1), D^(k), A^(k+1..d)]], so
// ||.||^2 = sum_{k,l} s_h' (*_n Gram(U_kn, U_ln)) s_h with U_kn = Abar (n < k),
// D (n = k), A (n > k); summed over h through S_H.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int which_mat(int k, int n) { return n < k ? SEL_ABAR : (n == k ? SEL_D : SEL_A); }

// grams layout: pair index p in [(A,A), (Abar,Abar), (Abar,A), (D,D), (D,A), (Abar,D)].
__device__ __forceinline__ double gram_entry(const double* grams, int ndim, int R, int n, int u, int v, int l, int m) {
    // Gram(u, v)[l][m] for mode n, through Gram(v, u)[m][l] when only the transpose is stored
    int p = -1;
    bool tr = false;
    if (u == SEL_A && v == SEL_A) p = 0;
    else if (u == SEL_ABAR && v == SEL_ABAR) p = 1;
    else if (u == SEL_ABAR && v == SEL_A) p = 2;
    else if (u == SEL_A && v == SEL_ABAR) { p = 2; tr = true; }
    else if (u == SEL_D && v == SEL_D) p = 3;
    else if (u == SEL_D && v == SEL_A) p = 4;
    else if (u == SEL_A && v == SEL_D) { p = 4; tr = true; }
    else if (u == SEL_ABAR && v == SEL_D) p = 5;
    else { p = 5; tr = true; }   // (D, Abar)
    const double* g = grams + ((int64_t)p * ndim + n) * R * R;
    return tr ? __ldcg(g + m * R + l) : __ldcg(g + l * R + m);
}

// Factor objective finish, run by one block of blockDim.x threads (a multiple
// of 32, at most 1024): F_new += 1/2 <S_H, telescoped history Gram sum> +
// lambda/2 sum_n trace(A_n'A_n).  hist selects the history term.
__device__ __forceinline__ void obj_finish_f_block(SolverState* st, int ndim, int R, const double* grams,
                                                   const double* SH, bool hist, double lam, int set_cur, int* err) {
    __shared__ double red_of[32];
    double acc = 0.0, reg = 0.0;
    for (int i = threadIdx.x; i < R * R; i += blockDim.x) {
        const int l = i / R, m = i % R;
        if (hist) {
            double tot = 0.0;
            for (int k = 0; k < ndim; ++k)
                for (int kk = 0; kk < ndim; ++kk) {
                    double prod = 1.0;
                    for (int n = 0; n < ndim; ++n)
                        prod *= gram_entry(grams, ndim, R, n, which_mat(k, n), which_mat(kk, n), l, m);
                    tot += prod;
                }
            acc += __ldcg(SH + i) * tot;
        }
        if (l == m)
            for (int n = 0; n < ndim; ++n) reg += __ldcg(grams + (int64_t)n * R * R + i);
    }
    double v = 0.5 * acc + 0.5 * lam * reg;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(SGCP_FULL_MASK, v, off);
    if ((threadIdx.x & 31) == 0) red_of[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += red_of[i];
        const double F = __ldcg(&st->F_new) + tot;
        st->F_new = F;
        if (!isfinite(F)) set_err(err, ERRB_NUMERIC);
        if (set_cur) st->F_cur = F;
    }
    __syncthreads();
}

// S_H[l][m] = sum_{h in window} w theta^(t - h) s_h[l] s_h[m] at entry i.
template <typename T>
__device__ __forceinline__ double history_SH_elem(int R, const T* s_hist, const int64_t* h_dev, int n, int64_t t,
                                                  double w, double theta, int i) {
    const int l = i / R, m = i % R;
    double acc = 0.0;
    for (int h = 0; h < n; ++h) {
        const double wh = w * pow(theta, (double)(t - __ldcg(h_dev + h)));
        acc += wh * (double)__ldcg(s_hist + h * R + l) * (double)__ldcg(s_hist + h * R + m);
    }
    return acc;
}

}  // namespace sgcp
