// vbh_sweep.cuh -- the fused CAVI sweep for one data set (FP32 per
// observation, FP64 across chunks, blocks and in the global update).
//
// One launch = one sweep of Section 3.5:
//   (a) per observation, with Sigma0 = E[Lambda]^{-1} = L L^T, kappa, E[rho]:
//       D_i = d_{i,1:M} - d_{i,S},  y_i = r_i - d_{i,S}
//       q_i = D_i^T Sigma0 D_i = |L^T D_i|^2,  t_i = kappa^T D_i,  e_i = y_i - t_i
//   (b) the exact Q(beta_i) of Eq. 20-21 in rank-1 form (Sherman-Morrison on
//       Eq. 20; it is never materialised):
//       c_i = E[rho] / (1 + E[rho] q_i),  w_i = c_i e_i
//       Sigma_i = Sigma0 - c_i u_i u_i^T,  mu_{beta_i} = kappa + w_i u_i,  u_i = Sigma0 D_i
//       braces of Eq. 17:  S_i = e_i^2 / (1 + E[rho] q_i)^2 + q_i / (1 + E[rho] q_i)
//       ln|Sigma_i| = ln|Sigma0| - ln(1 + E[rho] q_i)   (matrix determinant lemma)
//   (c) block-local sums g = sum w_i D_i, G = sum (w_i^2 - c_i) D_i D_i^T,
//       T3 = sum S_i and T4 = sum ln(1 + E[rho] q_i): FP32 over chunks of 64
//       observations per thread, a warp butterfly, FP64 from there on.  T4 is
//       carried as a running product of (1 + E[rho] q_i) whose binary exponent
//       is peeled off every two observations; one log per chunk;
//   (d) the last block to finish adds the per-block FP64 partials in block
//       order (deterministic) and runs the closed-form updates of Eq. 16-18,
//       22-25 and 28-31 in FP64, written in centred form:
//       s = Sigma0 g, delta = (s + q0 (K0 - kappa)) / (q0 + V), kappa' = kappa + delta
//       W'^{-1} = Lambda_0^{-1} + V Sigma0 + Sigma0 G Sigma0 + q0 (K0-kappa)(K0-kappa)^T
//                 - (q0 + V) delta delta^T        (= Eq. 25 exactly)
//   (e) the ELBO of Eq. 11 and the convergence test, and the FP32 globals of
//       the next sweep.
// The inputs (r, d) are read from HBM exactly once per sweep, through 1-D
// bulk copies (cp.async.bulk) into a ring of shared-memory stages.
#pragma once

#include "vbh_internal.cuh"

namespace vbh {

template <int S>
struct SweepCfg {
    static constexpr int M = S - 1;
    static constexpr int MA = M > 0 ? M : 1;                // array extent
    static constexpr int NG = M * (M + 1) / 2;              // packed lower G
    static constexpr int NGA = NG > 0 ? NG : 1;
    static constexpr int I_G = 0, I_g = NG, I_T3 = NG + M, I_T4 = NG + M + 1, I_E4 = NG + M + 2;
    static constexpr int NSTAT = NG + M + 3;                // G, g, T3, T4 (ln of mantissas), E4 (exponents)
    static constexpr int NGRP = (NSTAT + 31) / 32;          // 32-wide butterfly groups
    static constexpr int THREADS = 256;
    static constexpr int MINB = (S <= 8) ? 2 : 1;           // resident blocks per SM the registers are sized for
    static constexpr int OPT = 4;                           // observations per thread per tile
    static constexpr int T = THREADS * OPT;                 // observations per tile
    static constexpr int STAGES = 3;
    static constexpr int FLUSH_TILES = 16;                  // 64 observations per thread per FP32 chunk
    static constexpr uint32_t R_BYTES = T * 4u;
    static constexpr uint32_t D_BYTES = T * S * 4u;
    static constexpr uint32_t STAGE_BYTES = R_BYTES + D_BYTES;
    static constexpr size_t RING_BYTES = size_t(STAGES) * STAGE_BYTES;
    static constexpr size_t SMEM_BYTES = RING_BYTES + 64;   // + mbarriers
};

// Load the S profile entries of row j of a shared-memory tile with the widest
// vector loads S allows (16, 8 or 4 bytes).  For S = 8 two consecutive rows of
// a phase of eight threads share banks (a 2-way conflict); the load/store
// unit has the headroom, and fixing it would cost selects in the FP32 pipe.
template <int S>
__device__ __forceinline__ void load_row(const float *__restrict__ dt, int j, float (&x)[S])
{
    if constexpr (S % 4 == 0) {
        const float4 *p = reinterpret_cast<const float4 *>(dt + size_t(j) * S);
#pragma unroll
        for (int q = 0; q < S / 4; ++q) {
            const float4 v = p[q];
            x[4 * q + 0] = v.x;
            x[4 * q + 1] = v.y;
            x[4 * q + 2] = v.z;
            x[4 * q + 3] = v.w;
        }
    } else if constexpr (S % 2 == 0) {
        const float2 *p = reinterpret_cast<const float2 *>(dt + size_t(j) * S);
#pragma unroll
        for (int q = 0; q < S / 2; ++q) {
            const float2 v = p[q];
            x[2 * q] = v.x;
            x[2 * q + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int q = 0; q < S; ++q) x[q] = dt[size_t(j) * S + q];
    }
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Steps (a)-(b) and the accumulation of (c) for one observation.  prod
// collects the product of (1 + E[rho] q_i).
template <int S>
__device__ __forceinline__ void observe(const float (&x)[S], float rr, const float (&L)[SweepCfg<S>::NGA],
                                        const float (&kap)[SweepCfg<S>::MA], float erho,
                                        float (&acc)[SweepCfg<S>::NSTAT], float &prod)
{
    using C = SweepCfg<S>;
    constexpr int M = C::M;
    const float dS = x[S - 1];
    const float y = rr - dS;
    float D[C::MA];
    float q = 0.0f, t = 0.0f;
#pragma unroll
    for (int j = 0; j < M; ++j) D[j] = x[j] - dS;
#pragma unroll
    for (int j = 0; j < M; ++j) {
        float v = 0.0f;                                    // (L^T D)_j
#pragma unroll
        for (int k = j; k < M; ++k) v = fmaf(L[k * (k + 1) / 2 + j], D[k], v);
        q = fmaf(v, v, q);
        t = fmaf(kap[j], D[j], t);
    }
    const float e = y - t;
    const float den = fmaf(erho, q, 1.0f);
    float inv = rcp_approx(den);
    inv = fmaf(inv, fmaf(-den, inv, 1.0f), inv);           // one Newton step
    const float c = erho * inv;
    const float w = c * e;
    const float gam = fmaf(w, w, -c);
    const float ei = e * inv;
    acc[C::I_T3] += fmaf(ei, ei, q * inv);                 // S_i
    prod *= den;
#pragma unroll
    for (int j = 0; j < M; ++j) {
        acc[C::I_g + j] = fmaf(w, D[j], acc[C::I_g + j]);
        const float gd = gam * D[j];
#pragma unroll
        for (int k = 0; k <= j; ++k) acc[j * (j + 1) / 2 + k] = fmaf(gd, D[k], acc[j * (j + 1) / 2 + k]);
    }
}

// prod = m 2^(E - 127) with m in [1, 2): keep m, add E - 127 to ex.  Valid
// while prod stays finite, i.e. for (1 + E[rho] q_i) < 2^62 per observation.
__device__ __forceinline__ void peel_exponent(float &prod, int &ex)
{
    const uint32_t b = __float_as_uint(prod);
    ex += int(b >> 23) - 127;
    prod = __uint_as_float((b & 0x007fffffu) | 0x3f800000u);
}

// Move the FP32 chunk sums of a warp into FP64: first the product into
// (ln mantissa, exponent), then a butterfly reduce-scatter over each group of
// 32 statistics leaves lane l with the warp total of statistic 32 g + l,
// which it adds to its FP64 accumulator.
template <int S>
__device__ __forceinline__ void flush_warp(float (&acc)[SweepCfg<S>::NSTAT], double (&acc64)[SweepCfg<S>::NGRP],
                                           float &prod, int &ex, int lane)
{
    using C = SweepCfg<S>;
    constexpr int NSTAT = C::NSTAT;
    peel_exponent(prod, ex);
    acc[C::I_T4] += logf(prod);
    acc[C::I_E4] += static_cast<float>(ex);                // exact: |ex| < 2^24
    prod = 1.0f;
    ex = 0;
#pragma unroll
    for (int g = 0; g < C::NGRP; ++g) {
        float v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = (g * 32 + i < NSTAT) ? acc[(g * 32 + i < NSTAT) ? g * 32 + i : 0] : 0.0f;
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            const bool up = (lane & off) != 0;
#pragma unroll
            for (int i = 0; i < off; ++i) {
                const float keep = up ? v[i + off] : v[i];
                const float send = up ? v[i] : v[i + off];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
            }
        }
        acc64[g] += static_cast<double>(v[0]);
    }
#pragma unroll
    for (int i = 0; i < NSTAT; ++i) acc[i] = 0.0f;
}

// ---------------------------------------------------------------------------
// Cholesky factor L (lower, row-major) of a symmetric positive-definite M x M
// matrix A in shared memory, column by column, by one warp.  Returns nonzero
// in every lane when A is not positive definite (a unit pivot is used then).
// ---------------------------------------------------------------------------
__device__ inline int warp_cholesky_rt(int M, const double *A, double *L, int lane)
{
    int fail = 0;
    for (int i = lane; i < M * M; i += 32) L[i] = 0.0;
    __syncwarp();
    for (int j = 0; j < M; ++j) {
        if (lane == 0) {
            double s = A[j * M + j];
            for (int k = 0; k < j; ++k) s -= L[j * M + k] * L[j * M + k];
            if (!(s > 0.0) || !isfinite(s)) {
                fail = 1;
                s = 1.0;
            }
            L[j * M + j] = sqrt(s);
        }
        __syncwarp();
        const double rjj = 1.0 / L[j * M + j];
        for (int i = j + 1 + lane; i < M; i += 32) {
            double s = A[i * M + j];
            for (int k = 0; k < j; ++k) s -= L[i * M + k] * L[j * M + k];
            L[i * M + j] = s * rjj;
        }
        __syncwarp();
    }
    return __shfl_sync(0xffffffffu, fail, 0);
}

template <int M>
__device__ __forceinline__ int warp_cholesky(const double *A, double *L, int lane)
{
    return warp_cholesky_rt(M, A, L, lane);
}

// Sum over the lanes of a warp (fixed order).
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// What the next data pass reads, from W^{-1} and nu (Eq. 28: E[Lambda] = nu W,
// so Sigma0 = W^{-1}/nu): the FP32 Cholesky factor of Sigma0 (plus Sigma0 and
// ln|Sigma0| for information).  Sweep 0 uses (Lambda_0^{-1}, nu = 1).  One
// warp; Lw receives chol(W^{-1}); returns ln|W^{-1}| in every lane.  The
// global update and the set-up kernel both use this function, so a fit
// resumed from saved factors continues bit for bit.
__device__ inline double derive_pass_globals_rt(int M, DevState *st, const double *Wn, double nu, double *Lw,
                                                int lane, int *fail)
{
    *fail = warp_cholesky_rt(M, Wn, Lw, lane);
    const double rs = rsqrt(nu);
    for (int i = lane; i < M; i += 32)
        for (int k = 0; k <= i; ++k) st->sw.L[i * (i + 1) / 2 + k] = static_cast<float>(Lw[i * M + k] * rs);
    for (int i = lane; i < M * M; i += 32) st->Sigma0[i] = Wn[i] / nu;
    const double ld = warp_sum(lane < M ? 2.0 * log(Lw[lane * M + lane]) : 0.0);
    if (lane == 0) st->lndetSigma0 = ld - M * log(nu);
    return ld;
}

template <int M>
__device__ __forceinline__ double derive_pass_globals(DevState *st, const double *Wn, double nu, double *Lw, int lane,
                                                     int *fail)
{
    return derive_pass_globals_rt(M, st, Wn, nu, Lw, lane, fail);
}

// ---------------------------------------------------------------------------
// (d)+(e): FP64 global update, ELBO and control, run by the whole last block.
// ws: shared-memory workspace of at least gu_ws_doubles(M) doubles.  The
// statistics of the partials are laid out as in SweepCfg: packed lower G,
// g, T3, T4 (ln of mantissas), E4 (binary exponents).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int gu_ws_doubles_rt(int M)
{
    return ((M * (M + 1) / 2 + M + 3 + 31) / 32) * 32 + 9 * (M > 0 ? M * M : 1) + 6 * (M > 0 ? M : 1) + 32;
}

template <int M>
constexpr int gu_ws_doubles()
{
    return gu_ws_doubles_rt(M);
}

__device__ inline void global_update_rt(int M, DevState *st, const double *__restrict__ part, int nblk,
                                        const SweepArgs &a, double *ws)
{
    const int NG = M * (M + 1) / 2;
    const int NSTAT = NG + M + 3;
    const int I_g = NG, I_T3 = NG + M, I_T4 = NG + M + 1, I_E4 = NG + M + 2;
    const int MM = M > 0 ? M * M : 1;
    const int MV = M > 0 ? M : 1;
    const int MD = M > 0 ? M : 1;                   // divisor (loops over M*M entries are empty at M = 0)
    constexpr double LN2PI = 1.8378770664093454836;
    constexpr double LN2 = 0.69314718055994530942;
    constexpr double LNPI = 1.1447298858494002;
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
    const int mode = a.mode;

    double *stat = ws;
    double *Sg = stat + ((NSTAT + 31) / 32) * 32;   // Sigma0~ = L~ L~^T of this pass
    double *G = Sg + MM;                            // sum (w^2 - c) D D^T (full)
    double *A = G + MM;                             // Sigma0~ G
    double *B = A + MM;                             // Sigma0~ G Sigma0~
    double *Wn = B + MM;                            // new W^{-1}
    double *Lw = Wn + MM;                           // chol(W^{-1})
    double *Li = Lw + MM;                           // Lw^{-1}
    double *EL = Li + MM;                           // E[Lambda] = nu W
    double *Cm = EL + MM;                           // sum_i E[(beta_i - kappa')(beta_i - kappa')^T]
    double *sv = Cm + MM;                           // Sigma0~ g
    double *dv = sv + MV;                           // kappa' - kappa~
    double *ko = dv + MV;                           // kappa~ (this pass)
    double *kn = ko + MV;                           // kappa'
    double *av = kn + MV;                           // K0 - kappa~
    double *gv = av + MV;                           // g
    double *sc = gv + MV;                           // scalars
    __shared__ int s_fail;

    // 1. partials -> totals (fixed order per statistic); Sigma0~, kappa~.
    //    The data pass used the FP32 factor L~ and kappa~ of st->sw; its
    //    Q(beta_i) is the exact Eq. 20-21 posterior for Sigma0~ = L~ L~^T and
    //    kappa~, so every FP64 quantity below is taken with those values: each
    //    sweep is an exact coordinate step from the rounded globals and the
    //    ELBO sequence is smooth (FP32 rounding enters at second order only).
    for (int j = warp; j < NSTAT; j += nwarp) {
        double s = 0.0;
#pragma unroll 4
        for (int b = lane; b < nblk; b += 32) s += __ldcg(part + size_t(b) * NSTAT + j);
        s = warp_sum(s);
        if (lane == 0) stat[j] = s;
    }
    if (warp == nwarp - 1) {
        const double ld = warp_sum(lane < M ? 2.0 * log(static_cast<double>(st->sw.L[lane * (lane + 1) / 2 + lane]))
                                            : 0.0);
        if (lane == 0) {
            sc[1] = ld;                                  // ln|Sigma0~|
            s_fail = 0;
        }
    }
    for (int i = tid; i < M * M; i += nth) {
        const int r = i / MD, c = i % MD;
        const int kmax = r < c ? r : c;
        double s = 0.0;
        for (int k = 0; k <= kmax; ++k)
            s = fma(static_cast<double>(st->sw.L[r * (r + 1) / 2 + k]), static_cast<double>(st->sw.L[c * (c + 1) / 2 + k]), s);
        Sg[i] = s;
    }
    for (int i = tid; i < M; i += nth) {
        ko[i] = static_cast<double>(st->sw.kappa[i]);
        av[i] = st->K0[i] - ko[i];
    }
    __syncthreads();

    const ElboConst kc = (mode == MODE_ELBO) ? st->kc_given : st->kc_upd;
    // EM (Eq. 42-47): the pass used the point estimates K~ = kappa~, Lambda^{-1}~ =
    // Sigma0~ and rho~ = E[rho] of sw; the statistics of the pass are the same sums
    const bool em = st->em != 0;
    const double V = st->V;
    const double T3 = stat[I_T3];
    const double T4 = stat[I_T4] + LN2 * stat[I_E4];
    const double q0 = st->q0, n0 = st->n0, b0 = st->b0, a0 = st->a0;
    const double lam = kc.lam, nu = kc.nu;

    // 2. G (full), g, s = Sigma0~ g, A = Sigma0~ G
    for (int i = tid; i < M * M; i += nth) {
        const int r = i / MD, c = i % MD;
        G[i] = (r >= c) ? stat[r * (r + 1) / 2 + c] : stat[c * (c + 1) / 2 + r];
    }
    for (int i = tid; i < M; i += nth) gv[i] = stat[I_g + i];
    __syncthreads();
    for (int i = tid; i < M * M; i += nth) {
        const int r = i / MD, c = i % MD;
        double s = 0.0;
        for (int k = 0; k < M; ++k) s = fma(Sg[r * M + k], G[k * M + c], s);
        A[i] = s;
    }
    for (int i = tid; i < M; i += nth) {
        double s = 0.0;
        for (int k = 0; k < M; ++k) s = fma(Sg[i * M + k], gv[k], s);
        sv[i] = s;
    }
    __syncthreads();
    // 3. B = Sigma0~ G Sigma0~, delta, kappa'
    for (int i = tid; i < M * M; i += nth) {
        const int r = i / MD, c = i % MD;
        double s = 0.0;
        for (int k = 0; k < M; ++k) s = fma(A[r * M + k], Sg[k * M + c], s);
        B[i] = s;
    }
    for (int i = tid; i < M; i += nth) {
        if (em) {                                   // Eq. 46: K' = (1/V) sum M_i = K~ + Sigma0~ g / V
            dv[i] = sv[i] / V;
            kn[i] = ko[i] + dv[i];
        } else if (mode == MODE_ELBO) {             // kappa is given; kappa~ is its FP32 rounding
            kn[i] = st->kappa[i];
            dv[i] = kn[i] - ko[i];
        } else {
            dv[i] = (sv[i] + q0 * av[i]) / lam;     // Eq. 24, centred on kappa~
            kn[i] = ko[i] + dv[i];
        }
    }
    __syncthreads();
    // 4. W'^{-1} (Eq. 25, centred) and C
    for (int i = tid; i < M * M; i += nth) {
        const int r = i / MD, c = i % MD;
        const double Bs = 0.5 * (B[r * M + c] + B[c * M + r]);
        if (em) {
            // Eq. 47: (1/V) sum (M_i M_i^T + Sigma_i) - K' K'^T = Sigma0~ + Sigma0~ G Sigma0~ / V - a a^T
            Wn[i] = Sg[i] + Bs / V - dv[r] * dv[c];
        } else if (mode == MODE_ELBO) {
            Wn[i] = st->Winv[i];
        } else {
            Wn[i] = st->L0inv[i] + V * Sg[i] + Bs + q0 * av[r] * av[c] - lam * dv[r] * dv[c];
        }
        // C = V Sigma0~ + Sigma0~ G Sigma0~ - s delta^T - delta s^T + V delta delta^T
        Cm[i] = V * Sg[i] + Bs - sv[r] * dv[c] - dv[r] * sv[c] + V * dv[r] * dv[c];
    }
    __syncthreads();
    // 5. Cholesky of W'^{-1} (warp 0) and, unless only the ELBO is wanted,
    //    the FP32 factor of the next data pass; Lw^{-1}
    if (warp == 0) {
        int fail;
        double lndetWn;
        if (mode == MODE_ELBO && !em) {
            fail = warp_cholesky_rt(M, Wn, Lw, lane);
            lndetWn = warp_sum(lane < M ? 2.0 * log(Lw[lane * M + lane]) : 0.0);
        } else {
            lndetWn = derive_pass_globals_rt(M, st, Wn, em ? 1.0 : nu, Lw, lane, &fail);
        }
        if (lane == 0) {
            if (fail) s_fail = 1;
            sc[2] = lndetWn;
        }
        __syncwarp();
        for (int c = lane; c < M; c += 32) {        // lane c solves Lw x = e_c
            for (int i = 0; i < c; ++i) Li[i * M + c] = 0.0;
            for (int i = c; i < M; ++i) {
                double s = (i == c) ? 1.0 : 0.0;
                for (int k = c; k < i; ++k) s -= Lw[i * M + k] * Li[k * M + c];
                Li[i * M + c] = s / Lw[i * M + i];
            }
        }
    }
    __syncthreads();
    // 6. E[Lambda] = nu Li^T Li (Eq. 28)
    for (int i = tid; i < M * M; i += nth) {
        const int r = i / MD, c = i % MD;
        double s = 0.0;
        for (int k = (r > c ? r : c); k < M; ++k) s = fma(Li[k * M + r], Li[k * M + c], s);
        EL[i] = nu * s;
    }
    __syncthreads();
    // 7. traces (warp 0), then the ELBO (or, for EM, ln p(r | theta)) and control (thread 0)
    if (em && warp == 0) {
        // ln p(r | theta~) = sum_i ln N(y_i; D_i^T K~, 1/rho~ + q_i): with the pass's sums,
        // V/2 (ln rho~ - ln 2 pi) - rho~/2 sum S_i - 1/2 sum ln(1 + rho~ q_i) - 1/2 tr(Sigma0~ G)
        double t1 = 0.0;
        for (int i = lane; i < M * M; i += 32) t1 = fma(Sg[i], G[i], t1);
        const double trSG = warp_sum(t1);
        if (lane == 0) {
            const double rho_t = static_cast<double>(st->sw.erho);
            const double L = 0.5 * V * (log(rho_t) - LN2PI) - 0.5 * rho_t * T3 - 0.5 * T4 - 0.5 * trSG;
            const double rho_n = V / T3;                                             // Eq. 45
            bool finite = isfinite(L) && isfinite(rho_n) && rho_n > 0.0 && !s_fail;
            for (int j = 0; j < M; ++j) finite = finite && isfinite(kn[j]);
            st->elbo = L;
            st->const_dropped = 0;
            st->a_rho = rho_n;                                                       // point estimate as (rho, 1)
            st->b_rho = 1.0;
            st->nu = 1.0;
            st->lam = V;
            st->erho = rho_n;
            if (mode == MODE_INIT) {
                st->iter = 0;
                st->converged = 0;
            } else {
                st->iter += 1;
                st->converged = (fabs(L - st->elbo_prev) < st->tol * fabs(L)) ? 1 : 0;
            }
            if (st->trace && st->iter <= st->max_iter) st->trace[st->iter] = L;
            st->elbo_prev = L;
            if (!finite && st->status == ST_OK) st->status = ST_ENONFINITE;
            sc[0] = rho_n;
        }
    }
    if (!em && warp == 0) {
        double t1 = 0.0, t2 = 0.0, t3 = 0.0;
        for (int i = lane; i < M * M; i += 32) {
            const int r = i / MD, c = i % MD;
            t1 = fma(EL[i], Cm[i], t1);                                   // tr(E[Lambda] C), both symmetric
            t2 = fma(st->L0inv[i], EL[i], t2);                            // tr(Lambda_0^{-1} E[Lambda])
            t3 = fma((kn[r] - st->K0[r]) * EL[i], kn[c] - st->K0[c], t3);  // (kappa'-K0)^T E[Lambda] (kappa'-K0)
        }
        const double trELC = warp_sum(t1), trL0EL = warp_sum(t2), quadK = warp_sum(t3);
        if (lane == 0) {
            const double lndetS0 = sc[1];
            const double lndetW = -sc[2];
            const double a_rho = kc.a_rho;                                           // Eq. 16
            const double b_rho = (mode == MODE_ELBO) ? st->b_rho : b0 + 0.5 * T3;    // Eq. 17
            const double Er = a_rho / b_rho;                                         // Eq. 29
            const double logb = log(b_rho);
            const double Elr = kc.psi_a - logb;
            const double ElL = kc.sum_psi_nu + M * LN2 + lndetW;
            const double lnBq = -0.5 * nu * lndetW - 0.5 * nu * M * LN2 - 0.25 * M * (M - 1) * LNPI - kc.sum_lgamma_nu;
            double L = st->prior_const;
            L += 0.5 * V * (Elr - LN2PI) - 0.5 * Er * T3;                            // E ln p(r | beta, rho)
            L += 0.5 * V * (ElL - M * LN2PI) - 0.5 * trELC - 0.5 * V * M / lam;     // E ln p(beta | K, Lambda)
            L += 0.5 * ElL - 0.5 * q0 * (quadK + M / lam);                           // E ln p(K | Lambda)
            L += 0.5 * (n0 - M - 1.0) * ElL - 0.5 * trL0EL;                          // E ln p(Lambda)
            L += (a0 - 1.0) * Elr - b0 * Er;                                         // E ln p(rho)
            L += 0.5 * (V * lndetS0 - T4) + 0.5 * V * M * (1.0 + LN2PI);             // H[Q(beta)]
            L += -0.5 * ElL - 0.5 * M * (kc.log_lam - LN2PI) + 0.5 * M;              // H[Q(K | Lambda)]
            if (M > 0) L += -lnBq - 0.5 * (nu - M - 1.0) * ElL + 0.5 * nu * M;      // H[Q(Lambda)]
            L += a_rho - logb + kc.lgamma_a + (1.0 - a_rho) * kc.psi_a;              // H[Q(rho)]

            bool finite = isfinite(L) && isfinite(b_rho) && b_rho > 0.0 && !s_fail;
            for (int j = 0; j < M; ++j) finite = finite && isfinite(kn[j]);
            st->elbo = L;
            st->const_dropped = st->prior_dropped;
            if (mode != MODE_ELBO) {
                st->a_rho = a_rho;
                st->b_rho = b_rho;
                st->nu = nu;
                st->lam = lam;
                st->erho = Er;
                if (mode == MODE_INIT) {
                    st->iter = 0;
                    st->converged = 0;
                } else {
                    st->iter += 1;
                    st->converged = (fabs(L - st->elbo_prev) < st->tol * fabs(L)) ? 1 : 0;
                }
                if (st->trace && st->iter <= st->max_iter) st->trace[st->iter] = L;
                st->elbo_prev = L;
            } else {
                // sweep 0 of a fit started from given factors: L_0 of that state
                st->elbo_prev = L;
                if (st->trace) st->trace[0] = L;
            }
            if (!finite && st->status == ST_OK) st->status = ST_ENONFINITE;
            sc[0] = Er;
        }
    }
    __syncthreads();
    // 8. write the new globals and the FP32 inputs of the next sweep
    if (mode != MODE_ELBO || em) {
        for (int i = tid; i < M * M; i += nth) st->Winv[i] = Wn[i];
        for (int i = tid; i < M; i += nth) {
            st->kappa[i] = kn[i];
            st->sw.kappa[i] = static_cast<float>(kn[i]);
        }
        if (tid == 0) st->sw.erho = static_cast<float>(sc[0]);
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const int keep = (mode == MODE_ITER || mode == MODE_INIT) && st->status == ST_OK && !st->converged &&
                         st->iter < st->target && st->iter < st->max_iter;
        if (a.use_cond) cudaGraphSetConditional(a.cond, keep ? 1u : 0u);
    }
}

template <int M>
__device__ __forceinline__ void global_update(DevState *st, const double *__restrict__ part, int nblk,
                                              const SweepArgs &a, double *ws)
{
    global_update_rt(M, st, part, nblk, a, ws);
}

// ---------------------------------------------------------------------------
// The fused sweep kernel.
// ---------------------------------------------------------------------------
template <int S>
__global__ void __launch_bounds__(SweepCfg<S>::THREADS, SweepCfg<S>::MINB) sweep_kernel(SweepArgs a)
{
    using C = SweepCfg<S>;
    constexpr int M = C::M, NG = C::NG, NSTAT = C::NSTAT, NGRP = C::NGRP;
    constexpr int THREADS = C::THREADS, T = C::T, STAGES = C::STAGES;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + C::RING_BYTES);
    __shared__ int s_bad, s_last;

    DevState *st = a.st;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_bad = 0;

    // Every block takes the same decision: the control fields are only written
    // by the last block of a launch, after all other blocks have finished.
    const bool run = (a.mode != MODE_ITER) ||
                     (st->status == ST_OK && !st->converged && st->iter < st->target && st->iter < st->max_iter);

    float acc[NSTAT];
    double acc64[NGRP];
    float prod = 1.0f;
    int ex = 0;
#pragma unroll
    for (int i = 0; i < NSTAT; ++i) acc[i] = 0.0f;
#pragma unroll
    for (int g = 0; g < NGRP; ++g) acc64[g] = 0.0;

    if (run) {
        float L[C::NGA], kap[C::MA];
        const float erho = st->sw.erho;          // 0 in sweep 0 of a CAVI fit from the paper's start: c_i = 0
#pragma unroll
        for (int i = 0; i < NG; ++i) L[i] = st->sw.L[i];
#pragma unroll
        for (int i = 0; i < M; ++i) kap[i] = st->sw.kappa[i];
        if constexpr (NG == 0) L[0] = 0.0f;
        if constexpr (M == 0) kap[0] = 0.0f;

        const long long V = a.V;
        const long long ntf = V / T;                         // full tiles
        const long long bid = blockIdx.x, nb = gridDim.x;
        const long long nk = (ntf > bid) ? (ntf - bid + nb - 1) / nb : 0;   // my full tiles

        if (tid == 0) {
            for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
            fence_mbar_init();
        }
        __syncthreads();
        if (tid == 0) {
            for (long long k = 0; k < nk && k < STAGES; ++k) {
                const long long tile = bid + k * nb;
                unsigned char *stage = smem + size_t(k) * C::STAGE_BYTES;
                mbar_arrive_expect_tx(&full[k], C::STAGE_BYTES);
                bulk_load(stage, a.r + tile * T, C::R_BYTES, &full[k]);
                bulk_load(stage + C::R_BYTES, a.d + tile * T * S, C::D_BYTES, &full[k]);
            }
        }
        long long k = 0;
        int ftile = 0;
        for (; k < nk; ++k) {
            const int s = int(k % STAGES);
            const uint32_t parity = uint32_t((k / STAGES) & 1);
            const bool ok = mbar_wait_bounded(&full[s], parity, 2000000000ull);
            if (ok) {
                const float *rt = reinterpret_cast<const float *>(smem + size_t(s) * C::STAGE_BYTES);
                const float *dt = rt + T;
#pragma unroll
                for (int u = 0; u < C::OPT; ++u) {
                    const int j = tid + u * THREADS;
                    float x[S];
                    load_row<S>(dt, j, x);
                    observe<S>(x, rt[j], L, kap, erho, acc, prod);
                    if (u & 1) peel_exponent(prod, ex);
                }
            }
            if (__syncthreads_or(!ok)) {
                if (tid == 0) s_bad = 1;
                break;
            }
            if (tid == 0 && k + STAGES < nk) {
                const long long tile = bid + (k + STAGES) * nb;
                unsigned char *stage = smem + size_t(s) * C::STAGE_BYTES;
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&full[s], C::STAGE_BYTES);
                bulk_load(stage, a.r + tile * T, C::R_BYTES, &full[s]);
                bulk_load(stage + C::R_BYTES, a.d + tile * T * S, C::D_BYTES, &full[s]);
            }
            if (++ftile == C::FLUSH_TILES) {
                flush_warp<S>(acc, acc64, prod, ex, lane);
                ftile = 0;
            }
        }
        __syncthreads();
        if (s_bad) {
            // a wait ran out: record it, then let the copies this block issued
            // and did not consume land before the block exits (bounded)
            if (tid == 0) {
                atomicCAS(&st->status, ST_OK, ST_ETIMEOUT);
                for (long long kk = k; kk < nk && kk < k + STAGES; ++kk)
                    (void)mbar_wait_bounded(&full[kk % STAGES], uint32_t((kk / STAGES) & 1), 200000000ull);
            }
        } else {
            // ragged tail: the observations after the last full tile, plain loads
            const long long tail0 = ntf * T;
            if (tail0 < V && bid == (ntf % nb)) {
                for (long long i = tail0 + tid; i < V; i += THREADS) {
                    float x[S];
#pragma unroll
                    for (int q = 0; q < S; ++q) x[q] = __ldg(a.d + i * S + q);
                    observe<S>(x, __ldg(a.r + i), L, kap, erho, acc, prod);
                    peel_exponent(prod, ex);
                }
            }
        }
    }
    flush_warp<S>(acc, acc64, prod, ex, lane);
    __syncthreads();   // the ring is idle from here on: reuse it for the block reduction

    // block reduction in FP64, fixed order, then this block's partials
    double *s_red = reinterpret_cast<double *>(smem);      // [THREADS / 32][NGRP * 32]
#pragma unroll
    for (int g = 0; g < NGRP; ++g) s_red[warp * (NGRP * 32) + g * 32 + lane] = acc64[g];
    __syncthreads();
    for (int j = tid; j < NSTAT; j += THREADS) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < THREADS / 32; ++w) s += s_red[w * (NGRP * 32) + j];
        a.partials[size_t(blockIdx.x) * NSTAT + j] = s;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(&st->ticket, 1u) == gridDim.x - 1) ? 1 : 0;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (run && !s_bad) {
        // every copy of this block has landed, so the ring's shared memory
        // serves as the workspace of the global update
        global_update<M>(st, a.partials, gridDim.x, a, reinterpret_cast<double *>(smem));
    } else if (tid == 0 && a.use_cond) {
        cudaGraphSetConditional(a.cond, 0u);
    }
    if (tid == 0) st->ticket = 0u;
}

// ---------------------------------------------------------------------------
// Set-up before the first data pass of a fit (one warp):
//   init != 0: sweep 0 reads Sigma0 = Lambda_0^{-1}, kappa = K0, E[rho] = 0;
//   init == 0: it reads Sigma0 = W^{-1}/nu, kappa, E[rho] = a_rho / b_rho of
//              the given global factors.
// Also the per-fit constants of the ELBO: ln|Lambda_0^{-1}|, the prior-only
// terms, and the special functions of (a_rho, nu, lambda) for the updates of
// this data set (Eq. 16, 22, 23) and for the given factors.
// ---------------------------------------------------------------------------
__device__ inline void elbo_const(ElboConst *k, int M, double a_rho, double nu, double lam, int lane)
{
    double sp = 0.0, sl = 0.0;
    for (int j = lane; j < M; j += 32) {
        const double x = 0.5 * (nu - j);                 // (nu + 1 - (j + 1)) / 2
        sp += digamma_d(x);
        sl += lgamma(x);
    }
    sp = warp_sum(sp);
    sl = warp_sum(sl);
    if (lane == 0) {
        k->a_rho = a_rho;
        k->nu = nu;
        k->lam = lam;
        k->lgamma_a = lgamma(a_rho);
        k->psi_a = digamma_d(a_rho);
        k->sum_psi_nu = sp;
        k->sum_lgamma_nu = sl;
        k->log_lam = log(lam);
    }
}

// The set-up body for one state, run by one warp (lane = 0..31); A and Lc
// are shared-memory scratch of M*M doubles each.
__device__ inline void setup_state_rt(int M, DevState *st, int init, int lane, double *A, double *Lc)
{
    constexpr double LN2PI = 1.8378770664093454836;
    constexpr double LN2 = 0.69314718055994530942;
    constexpr double LNPI = 1.1447298858494002;
    for (int i = lane; i < M * M; i += 32) A[i] = st->L0inv[i];
    __syncwarp();
    int fail = warp_cholesky_rt(M, A, Lc, lane);
    const double l0 = warp_sum(lane < M ? 2.0 * log(Lc[lane * M + lane]) : 0.0);
    // prior-only terms: M/2 (ln q0 - ln 2 pi) + a0 ln b0 - lnGamma(a0) + ln B(Lambda_0, n0)
    const double n0 = st->n0;
    const bool proper = (M == 0) || (n0 > M - 1.0);
    const double lg0 = warp_sum((lane < M && proper) ? lgamma(0.5 * (n0 - lane)) : 0.0);
    if (lane == 0) {
        st->lndetL0inv = l0;
        double pc = 0.5 * M * (log(st->q0) - LN2PI) + st->a0 * log(st->b0) - lgamma(st->a0);
        if (M > 0 && proper)                            // ln B(W0, n0), ln|W0| = -ln|Lambda_0^{-1}|
            pc += 0.5 * n0 * l0 - 0.5 * n0 * M * LN2 - 0.25 * M * (M - 1) * LNPI - lg0;
        st->prior_const = pc;
        st->prior_dropped = (M > 0 && !proper) ? 1 : 0;
    }
    const double V = st->V;
    elbo_const(&st->kc_upd, M, st->a0 + 0.5 * V, n0 + V, st->q0 + V, lane);
    if (!init) elbo_const(&st->kc_given, M, st->a_rho, st->nu, st->lam, lane);
    __syncwarp();
    if (!init)
        for (int i = lane; i < M * M; i += 32) A[i] = st->Winv[i];
    __syncwarp();
    int fail2 = 0;
    (void)derive_pass_globals_rt(M, st, A, init ? 1.0 : st->nu, Lc, lane, &fail2);
    fail |= fail2;
    for (int i = lane; i < M; i += 32) {
        const double kv = init ? st->K0[i] : st->kappa[i];
        st->sw.kappa[i] = static_cast<float>(kv);
        if (init) st->kappa[i] = kv;
    }
    if (lane == 0) {
        st->erho = init ? 0.0 : st->a_rho / st->b_rho;
        st->sw.erho = static_cast<float>(st->erho);
        st->ticket = 0u;
        if (fail) st->status = ST_ENONFINITE;
    }
}

template <int M>
__device__ __forceinline__ void setup_state(DevState *st, int init, int lane, double *A, double *Lc)
{
    setup_state_rt(M, st, init, lane, A, Lc);
}

template <int M>
__global__ void setup_kernel(DevState *st, int init)
{
    constexpr int MM = M > 0 ? M * M : 1;
    __shared__ double A[MM], Lc[MM];
    if (threadIdx.x >= 32) return;
    setup_state<M>(st, init, threadIdx.x, A, Lc);
}

} // namespace vbh
