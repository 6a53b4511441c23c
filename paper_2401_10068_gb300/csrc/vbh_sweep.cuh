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
//   (d) the block that finishes the launch (a ticket; above 128 blocks the
//       last block of each group of 32 first sums its group) adds the FP64
//       partials in a fixed order (deterministic) and runs the closed-form
//       updates of Eq. 16-18, 22-25 and 28-31 in FP64, written in centred form:
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
    // compensated statistics: one more column, U = sum c_i e_i^2
    static constexpr int I_U = NSTAT, NSTATC = NSTAT + 1, NGRPC = (NSTATC + 31) / 32;
    static constexpr int THREADS = 256;
    static constexpr int MINB = (S <= 8) ? 2 : 1;           // resident blocks per SM the registers are sized for
    static constexpr int MINB_C = (S <= 8) ? 2 : 1;         // the same for the compensated form
    static constexpr int MINB_BC = (S <= 9) ? 2 : 1;        // and for its batched pass
    static constexpr int OPT = 4;                           // observations per thread per tile
    static constexpr int T = THREADS * OPT;                 // observations per tile
    static constexpr int STAGES = 3;
    static constexpr int FLUSH_TILES = 16;                  // 64 observations per thread per FP32 chunk
    static constexpr uint32_t R_BYTES = T * 4u;
    static constexpr uint32_t D_BYTES = T * S * 4u;
    static constexpr uint32_t STAGE_BYTES = R_BYTES + D_BYTES;
    static constexpr size_t RING_BYTES = size_t(STAGES) * STAGE_BYTES;
    static constexpr size_t SMEM_BYTES = RING_BYTES + 64;   // + mbarriers
    // compensated form: a ring of STAGES_C stages (two at S = 8, so that two blocks
    // and their tables fit in an SM's shared memory), the table of profile terms
    // (2^S entries of 32 bytes) and the split pass globals
    static constexpr int STAGES_C = (S == 8) ? 2 : 3;
    static constexpr size_t RING_BYTES_C = size_t(STAGES_C) * STAGE_BYTES;
    static constexpr size_t TAB_BYTES = size_t(32) << S;
    static constexpr int SPLIT_FLOATS = 2 * NG + 2 * M;
    static constexpr size_t SPLIT_BYTES = ((size_t(SPLIT_FLOATS) * 4 + 63) / 64) * 64 + 64;
    static constexpr size_t OFF_TAB = RING_BYTES_C, OFF_SPLIT = OFF_TAB + TAB_BYTES;
    static constexpr size_t SMEM_BYTES_C = OFF_SPLIT + SPLIT_BYTES + 64;   // + mbarriers
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

// ---------------------------------------------------------------------------
// Compensated statistics for the stopping test.  With binary profiles every
// observation of a profile repeats the FP32 rounding of the terms that depend
// on the profile alone (q_i, 1 + E[rho] q_i, c_i, t_i), and FP32 chunk sums
// round at the size of the running total; both leave a rounding noise of
// about 1e-8 |L| in the ELBO that changes from sweep to sweep, which a
// relative stopping tolerance of 1e-8 cannot tell from convergence.  The
// ELBO depends on the statistics at first order only through
//     E[rho] T3 + tr(Sigma0~ G) + T4,
// and E[rho] S_i + (w_i^2 - c_i) q_i = c_i e_i^2 exactly (with
// h_i = 1/(1 + E[rho] q_i): E[rho] e^2 h^2 + E[rho] q h + E[rho]^2 h^2 e^2 q
// - E[rho] h q = E[rho] e^2 h).  So the compensated pass carries, next to the
// FP32 statistics of the update, U = sum c_i e_i^2 and T4 = sum ln(1 +
// E[rho] q_i) as two-part FP32 numbers (hi + lo) evaluated to ~2^-40:
//   q_i and t_i from the split Sigma0~ = Sh + Sl and kappa~ = kh + kl of the
//   pass globals (the Sh and kh sums are exact for entries in {0, 1}),
//   e_i = y_i - t_i, 1 + E[rho] q_i, 1/(1 + E[rho] q_i) and c_i by
//   error-free transformations (two-sum, FMA products) and one Newton
//   correction, U by a two-part running sum, T4 as a two-part running
//   product of (1 + E[rho] q_i) with one logarithm per warp and chunk.
// The global update then replaces the first-order part of the FP32
// statistics in the ELBO by these.  y_i and D_i are formed in FP32 once per
// observation, independent of the globals, so their rounding is part of the
// data and cancels in the ELBO differences.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// The profile-only terms of the compensated pass for one D (y enters only
// through e = y - t): t = th + tl, 1 + E[rho] q = dh + dl, h = 1/(1 + E[rho] q)
// (FP32), c = E[rho] h = ch + cl, and q h (FP32).  split: Sh[NG], Sl[NG],
// kh[M], kl[M] (the split pass globals, in shared memory).
struct ProfileTerms {
    float th, tl, dh, dl, h, ch, cl, qh;
};

template <int S>
__device__ __forceinline__ ProfileTerms profile_terms(const float (&D)[SweepCfg<S>::MA], const float *__restrict__ split,
                                                      float erho)
{
    using C = SweepCfg<S>;
    constexpr int M = C::M, NG = C::NG;
    const float *Sh = split, *Sl = split + NG, *kh = split + 2 * NG, *kl = split + 2 * NG + M;
    float qh = 0.0f, ql = 0.0f, th = 0.0f, tl = 0.0f;
#pragma unroll
    for (int j = 0; j < M; ++j) {
#pragma unroll
        for (int k = 0; k <= j; ++k) {
            const int e = j * (j + 1) / 2 + k;
            const float P = D[j] * D[k];
            qh = fmaf(Sh[e], P, qh);
            ql = fmaf(Sl[e], P, ql);
        }
        th = fmaf(kh[j], D[j], th);
        tl = fmaf(kl[j], D[j], tl);
    }
    ProfileTerms pt;
    pt.th = th;
    pt.tl = tl;
    const float p = erho * qh;                             // 1 + E[rho] q = dh + dl
    const float pe = fmaf(erho, qh, -p);
    const float big = fmaxf(1.0f, p), sml = fminf(1.0f, p);
    pt.dh = big + sml;
    pt.dl = fmaf(erho, ql, (sml - (pt.dh - big)) + pe);
    float h = rcp_approx(pt.dh);                           // 1/(1 + E[rho] q) = h + hl
    h = fmaf(h, fmaf(-pt.dh, h, 1.0f), h);
    const float res = fmaf(-pt.dl, h, fmaf(-pt.dh, h, 1.0f));
    const float hl = h * res;
    pt.h = h;
    pt.ch = erho * h;                                      // c = ch + cl
    pt.cl = fmaf(erho, hl, fmaf(erho, h, -pt.ch));
    pt.qh = (qh + ql) * h;
    return pt;
}

// The table of profile terms for 0/1 profiles: entry `code` (bit j = d_j,
// j < S) holds the ProfileTerms of D_j = d_j - d_S as two float4.  Built by
// threads t0, t0 + nt, ... of the block.
template <int S>
__device__ __forceinline__ void build_profile_table(float4 *__restrict__ tab, const float *__restrict__ split,
                                                    float erho, int t0, int nt)
{
    using C = SweepCfg<S>;
    for (int code = t0; code < (1 << S); code += nt) {
        const float dS = float((code >> (S - 1)) & 1);
        float D[C::MA];
#pragma unroll
        for (int j = 0; j < C::MA; ++j) D[j] = (j < C::M) ? float((code >> j) & 1) - dS : 0.0f;
        const ProfileTerms pt = profile_terms<S>(D, split, erho);
        tab[2 * code] = make_float4(pt.th, pt.tl, pt.dh, pt.dl);
        tab[2 * code + 1] = make_float4(pt.h, pt.ch, pt.cl, pt.qh);
    }
}

// Steps (a)-(c) of the compensated pass for one observation: the profile
// terms from the table when every d_ij is 0 or 1, else computed; then the
// FP32 statistics of the update, U += c e^2 and the two-part running product.
template <int S>
__device__ __forceinline__ void observe_comp(const float (&x)[S], float rr, const float4 *__restrict__ tab,
                                             const float *__restrict__ split, float erho,
                                             float (&acc)[SweepCfg<S>::NSTAT], float &ph, float &pl, float &uh,
                                             float &ul)
{
    using C = SweepCfg<S>;
    constexpr int M = C::M;
    const float dS = x[S - 1];
    const float y = rr - dS;
    float D[C::MA];
#pragma unroll
    for (int j = 0; j < M; ++j) D[j] = x[j] - dS;
    // code = sum d_j 2^j (exact for 0/1 entries); bad = sum |d_j - d_j^2| is 0 exactly when every d_j is 0 or 1
    float code = 0.0f, bad = 0.0f;
#pragma unroll
    for (int j = 0; j < S; ++j) {
        code = fmaf(x[j], float(1 << j), code);
        bad += fabsf(fmaf(-x[j], x[j], x[j]));
    }
    ProfileTerms pt;
    if (bad == 0.0f) {
        const int c = __float2int_rz(code);
        const float4 t0 = tab[2 * c], t1 = tab[2 * c + 1];
        pt = ProfileTerms{t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
    } else {
        pt = profile_terms<S>(D, split, erho);
    }
    float eh, el;                                          // e = y - t
    two_sum(y, -pt.th, eh, el);
    el -= pt.tl;
    // the FP32 statistics of the update
    const float w = pt.ch * eh;
    const float gam = fmaf(w, w, -pt.ch);
    const float ei = eh * pt.h;
    acc[C::I_T3] += fmaf(ei, ei, pt.qh);
#pragma unroll
    for (int j = 0; j < M; ++j) {
        acc[C::I_g + j] = fmaf(w, D[j], acc[C::I_g + j]);
        const float gd = gam * D[j];
#pragma unroll
        for (int k = 0; k <= j; ++k) acc[j * (j + 1) / 2 + k] = fmaf(gd, D[k], acc[j * (j + 1) / 2 + k]);
    }
    // U += c e^2
    const float e2h = eh * eh;
    const float e2l = fmaf(eh + eh, el, fmaf(eh, eh, -e2h));
    const float u = pt.ch * e2h;
    const float ue = fmaf(pt.cl, e2h, fmaf(pt.ch, e2l, fmaf(pt.ch, e2h, -u)));
    float su, sue;
    two_sum(uh, u, su, sue);
    uh = su;
    ul += sue + ue;
    // running product of (1 + E[rho] q)
    const float m = ph * pt.dh;
    const float me = fmaf(pl, pt.dh, fmaf(ph, pt.dl, fmaf(ph, pt.dh, -m)));
    ph = m + me;
    pl = me - (ph - m);
}

// (ph + pl) = m 2^E with m in [1, 2): keep m, scale pl alike, add E to ex.
// Valid while the product stays finite (each factor below 2^62).
__device__ __forceinline__ void peel_exponent2(float &ph, float &pl, int &ex)
{
    const uint32_t b = __float_as_uint(ph);
    const int E = int(b >> 23) - 127;
    ex += E;
    ph = __uint_as_float((b & 0x007fffffu) | 0x3f800000u);
    pl *= __uint_as_float(uint32_t(127 - E) << 23);
}

// prod = m 2^(E - 127) with m in [1, 2): keep m, add E - 127 to ex.  Valid
// while prod stays finite, i.e. for (1 + E[rho] q_i) < 2^62 per observation.
__device__ __forceinline__ void peel_exponent(float &prod, int &ex)
{
    const uint32_t b = __float_as_uint(prod);
    ex += int(b >> 23) - 127;
    prod = __uint_as_float((b & 0x007fffffu) | 0x3f800000u);
}

// Warp totals of NSTAT <= 16 FP32 statistics with fewer shuffles than the
// 32-slot reduce-scatter below: the values, padded to NV = 2^k >= NSTAT, are
// halved per level while more than one remains (lane bit `off` keeps the upper
// half), the remaining levels add; lane 4 s (for NV = 8) then holds the total
// of statistic s, and one more shuffle gives lane j the total of statistic j.
// A fixed order of additions, the same in every warp.
template <int NSTAT>
__device__ __forceinline__ float warp_totals_narrow(const float (&acc)[NSTAT], int lane)
{
    constexpr int NV = NSTAT <= 1 ? 1 : NSTAT <= 2 ? 2 : NSTAT <= 4 ? 4 : NSTAT <= 8 ? 8 : 16;
    float v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = (i < NSTAT) ? acc[i < NSTAT ? i : 0] : 0.0f;
    int n = NV;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        if (n > 1) {
            const bool up = (lane & off) != 0;
            const int h = n / 2;
#pragma unroll
            for (int i = 0; i < NV / 2; ++i) {
                if (i < h) {
                    const float keep = up ? v[i + h] : v[i];
                    const float send = up ? v[i] : v[i + h];
                    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
                }
            }
            n = h;
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], off);
        }
    }
    // statistic s sits in the lanes whose top log2(NV) bits spell s
    return __shfl_sync(0xffffffffu, v[0], (lane % NV) * (32 / NV));
}

// Move the FP32 chunk sums of a warp into FP64: first the product into
// (ln mantissa, exponent), then a butterfly reduce-scatter over each group of
// 32 statistics leaves lane l with the warp total of statistic 32 g + l,
// which it adds to its FP64 accumulator.
template <int S, bool ADD = true, bool NARROW = false>
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
    if constexpr (NARROW && NSTAT <= 16) {
        const float t = warp_totals_narrow<NSTAT>(acc, lane);
        const double x = (lane < NSTAT) ? static_cast<double>(t) : 0.0;
        acc64[0] = ADD ? acc64[0] + x : x;
#pragma unroll
        for (int i = 0; i < NSTAT; ++i) acc[i] = 0.0f;
        return;
    }
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
        if (ADD)
            acc64[g] += static_cast<double>(v[0]);
        else
            acc64[g] = static_cast<double>(v[0]);              // the first flush: no FP64 addition
    }
#pragma unroll
    for (int i = 0; i < NSTAT; ++i) acc[i] = 0.0f;
}

// Flush of the compensated pass: the running products of the warp's lanes
// are multiplied (two-part) and lane 0 takes one logarithm, ln(ph + pl) =
// ln ph + pl/ph (ph in [1, 2)); U is summed over the lanes in two parts and
// added in FP64 by the lane that holds column I_U; the FP32 statistics go
// through the butterfly of flush_warp.
template <int S, bool ADD = true, bool NARROW = false>
__device__ __forceinline__ void flush_warp_comp(float (&acc)[SweepCfg<S>::NSTAT],
                                                double (&acc64)[SweepCfg<S>::NGRPC], float &ph, float &pl, int &ex,
                                                float &uh, float &ul, int lane)
{
    using C = SweepCfg<S>;
    constexpr int NSTAT = C::NSTAT;
    peel_exponent2(ph, pl, ex);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, ph, off);
        const float ol = __shfl_xor_sync(0xffffffffu, pl, off);
        const int oe = __shfl_xor_sync(0xffffffffu, ex, off);
        const float m = ph * oh;
        const float me = fmaf(pl, oh, fmaf(ph, ol, fmaf(ph, oh, -m)));
        ph = m + me;
        pl = me - (ph - m);
        ex += oe;
        peel_exponent2(ph, pl, ex);
        const float vh = __shfl_xor_sync(0xffffffffu, uh, off);
        const float vl = __shfl_xor_sync(0xffffffffu, ul, off);
        float s, e;
        two_sum(uh, vh, s, e);
        uh = s;
        ul = (ul + vl) + e;
    }
    acc[C::I_T4] = (lane == 0) ? logf(ph) + pl / ph : 0.0f;
    acc[C::I_E4] = (lane == 0) ? static_cast<float>(ex) : 0.0f;     // exact: |ex| < 2^24
    ph = 1.0f;
    pl = 0.0f;
    ex = 0;
    if constexpr (NARROW && NSTAT <= 16) {
        const float t = warp_totals_narrow<NSTAT>(acc, lane);
        double x = (lane < NSTAT) ? static_cast<double>(t) : 0.0;
        if (lane == C::I_U) x = static_cast<double>(uh) + static_cast<double>(ul);   // I_U = NSTAT < 32
        acc64[0] = ADD ? acc64[0] + x : x;
        uh = 0.0f;
        ul = 0.0f;
#pragma unroll
        for (int i = 0; i < NSTAT; ++i) acc[i] = 0.0f;
        return;
    }
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
        if (ADD)
            acc64[g] += static_cast<double>(v[0]);
        else
            acc64[g] = static_cast<double>(v[0]);
    }
    if (lane == C::I_U % 32) {
        const double u = static_cast<double>(uh) + static_cast<double>(ul);
        acc64[C::I_U / 32] = ADD ? acc64[C::I_U / 32] + u : u;   // column I_U of the butterfly is zero
    }
    uh = 0.0f;
    ul = 0.0f;
#pragma unroll
    for (int i = 0; i < NSTAT; ++i) acc[i] = 0.0f;
}

// ---------------------------------------------------------------------------
// Named barriers of the global update (ids the sweep kernels leave unused).
// The main warps (all but the last) synchronise on BAR_MAIN; the last warp,
// the scalar warp, evaluates the logarithms and divisions of the update off
// the matrix chain and waits on BAR_T3 for the reduced statistics and on
// BAR_PIV for the Cholesky pivots.  FP64 divisions and logarithms are slow
// next to FP64 multiply-adds, so keeping them off the chain is what sets the
// latency of the update.
// ---------------------------------------------------------------------------
constexpr int BAR_MAIN = 1, BAR_T3 = 2, BAR_PIV = 3;

// Both are aligned barriers (every thread of the calling warp reaches them
// together), so the warp reconverges first.
__device__ __forceinline__ void named_sync(int id, int count)
{
    __syncwarp();
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

__device__ __forceinline__ void named_arrive(int id, int count)
{
    __syncwarp();
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Sum over the lanes of a warp (fixed order).
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// 1/sqrt(nu) as the pass factors use it (exactly 1 for nu = 1).
__device__ __forceinline__ double rs_of(double nu) { return nu == 1.0 ? 1.0 : rsqrt(nu); }

// ---------------------------------------------------------------------------
// Cholesky factor L (lower, row-major, zero above the diagonal) of a symmetric
// positive-definite M x M matrix A (M <= 32) in shared memory, by one warp,
// right-looking: for column j every lane forms the pivot's reciprocal square
// root r_j, lanes i > j scale the column below the pivot, and the trailing
// entries (i, k), j < k <= i, are updated in parallel, each lane owning the
// entries e = lane, lane + 32, ... of the packed lower triangle (row by row).
// One FP64 multiply-add per lane and column for M <= 7, so the chain per
// column is the pivot's rsqrt, one multiply and one multiply-add.  rd[j] =
// 1/L_jj and piv[j] = L_jj^2 (the pivots, whose logarithms add up to ln|A|).
// Returns nonzero in every lane when A is not positive definite (a unit
// pivot is used then).
// ---------------------------------------------------------------------------
__device__ inline int warp_cholesky_rt(int M, const double *__restrict__ A, double *__restrict__ L,
                                       double *__restrict__ rd, double *__restrict__ piv, double *__restrict__ col,
                                       int lane)
{
    if (M <= 3) {
        // the same operations in the same order by lane 0 alone, in registers:
        // for three columns or fewer the warp's shared-memory steps and
        // synchronisations cost more than they save
        int fail = 0;
        if (lane == 0) {
            double a[3][3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int k = 0; k < 3; ++k) a[i][k] = (i < M && k <= i) ? A[i * M + k] : 0.0;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                if (j >= M) break;
                double p = a[j][j];
                const long long pb = __double_as_longlong(p);
                const bool bad = pb <= 0 || ((pb >> 52) & 0x7ff) == 0x7ff;
                if (bad) p = 1.0;
                fail |= bad ? 1 : 0;
                const double r = rsqrt_fast(p);
                a[j][j] = p * r;
                rd[j] = r;
                piv[j] = p;
#pragma unroll
                for (int i = j + 1; i < 3; ++i)
                    if (i < M) a[i][j] *= r;
#pragma unroll
                for (int i = j + 1; i < 3; ++i)
#pragma unroll
                    for (int k = j + 1; k <= i; ++k)
                        if (i < M) a[i][k] = fma(-a[i][j], a[k][j], a[i][k]);
            }
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    if (i < M && k < M) L[i * M + k] = (k <= i) ? a[i][k] : 0.0;
        }
        fail = __shfl_sync(0xffffffffu, fail, 0);
        __syncwarp();
        return fail;
    }
    const int MD = M > 0 ? M : 1;
    for (int e = lane; e < M * M; e += 32) {
        const int r = e / MD, c = e - (e / MD) * MD;
        L[e] = (c <= r) ? A[e] : 0.0;
    }
    __syncwarp();
    int fail = 0;
    const int NG = M * (M + 1) / 2;
    for (int j = 0; j < M; ++j) {
        double p = L[j * M + j];
        const long long pb = __double_as_longlong(p);
        const bool bad = pb <= 0 || ((pb >> 52) & 0x7ff) == 0x7ff;   // not positive, or not finite (integer tests)
        if (bad) p = 1.0;
        fail |= bad ? 1 : 0;
        const double r = rsqrt_fast(p);
        __syncwarp();                               // the pivot is read before lane j overwrites it
        if (lane > j && lane < M) {
            const double lij = L[lane * M + j] * r;
            L[lane * M + j] = lij;
            col[lane] = lij;                        // column j below the pivot
        } else if (lane == j) {
            L[j * M + j] = p * r;
            rd[j] = r;
            piv[j] = p;
        }
        __syncwarp();
        // trailing update: entries (i, k) with k > j of the packed lower triangle
        int i = 0, k = lane;                        // packed entry e = lane -> (i, k)
        while (k > i) {
            k -= i + 1;
            ++i;
        }
        for (int e = lane; e < NG; e += 32) {
            if (k > j) L[i * M + k] = fma(-col[i], col[k], L[i * M + k]);
            k += 32;                                // next entry of this lane
            while (k > i) {
                k -= i + 1;
                ++i;
            }
        }
        __syncwarp();
    }
    return fail;
}

// Li = L^{-1} (lower) of a Cholesky factor L with reciprocal diagonal rd, by
// one warp: lane c forms column c by forward substitution, subtracting each
// finished row from the rows below it (lanes never wait on one another).
__device__ inline void warp_tri_inverse_rt(int M, const double *__restrict__ L, const double *__restrict__ rd,
                                           double *__restrict__ Li, int lane)
{
    const int c = lane;
    if (c < M) {
        for (int i = 0; i < M; ++i) Li[i * M + c] = (i == c) ? 1.0 : 0.0;
        for (int i = 0; i < M; ++i) {
            if (c <= i) {
                const double x = Li[i * M + c] * rd[i];
                Li[i * M + c] = x;
                for (int l = i + 1; l < M; ++l) Li[l * M + c] = fma(-L[l * M + i], x, Li[l * M + c]);
            }
        }
    }
    __syncwarp();
}

// ln|A| from the pivots of its Cholesky factorisation (one warp, every lane).
__device__ __forceinline__ double warp_logdet_rt(int M, const double *piv, int lane)
{
    return warp_sum(lane < M ? log(piv[lane]) : 0.0);
}

// What the next data pass reads, from W^{-1}, its Cholesky factor Lw and nu
// (Eq. 28: E[Lambda] = nu W, so Sigma0 = W^{-1}/nu): the FP32 Cholesky
// factor of Sigma0, and Sigma0 itself for information.  Threads t0, t0 + nt,
// ... of the block.  The global update and the set-up kernel both use this
// function and warp_cholesky_rt, so a fit resumed from saved factors
// continues bit for bit.
__device__ inline void write_pass_globals_rt(int M, DevState *st, const double *Wn, const double *Lw, double nu,
                                             double rs, int t0, int nt)
{
    const int MD = M > 0 ? M : 1;
    for (int e = t0; e < M * M; e += nt) {
        const int r = e / MD, c = e - (e / MD) * MD;
        st->Sigma0[e] = Wn[e] / nu;
        if (c <= r) st->sw.L[r * (r + 1) / 2 + c] = static_cast<float>(Lw[e] * rs);
    }
}

// The split pass globals of the compensated statistics, by one warp (lane =
// 0..31), from the FP32 factor L~ and kappa~ already in sw (M <= 10).
// Entry e of the packed lower triangle, (r, c), holds s = Sigma0~_rc (times 2
// off the diagonal): the products L~_ri L~_ci are exact as two-part FP32
// numbers and are summed in two parts.  With E the largest binary exponent
// over the entries, Sh = s rounded to a multiple of 2^(E - 17) and Sl = the
// rest: at most 55 grid parts of magnitude < 2^(E + 1) with signs from
// D_j D_k in {-1, 0, 1} sum exactly in FP32 (every partial sum is a multiple
// of 2^(E - 17) below 2^(E + 7)).  kappa~ likewise on the grid 2^(E' - 19)
// (at most 10 parts).  Sl and kl are 2^-18 of the largest entry or less, so
// their FP32 sums add about 2^-42 relative.
__device__ inline void write_pass_splits_sigma_rt(int M, SweepGlobalsF32 *sw, int lane)
{
    const int NG = M * (M + 1) / 2;
    float hi[2], lo[2];
    int emax = -1000;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int e = lane + 32 * u;
        hi[u] = 0.0f;
        lo[u] = 0.0f;
        if (e < NG) {
            int r = 0;
            while ((r + 1) * (r + 2) / 2 <= e) ++r;
            const int c = e - r * (r + 1) / 2;
            float sh = 0.0f, sl = 0.0f;
            for (int i = 0; i <= c; ++i) {
                const float a = sw->L[r * (r + 1) / 2 + i], b = sw->L[c * (c + 1) / 2 + i];
                const float pp = a * b;
                float t, te;
                two_sum(sh, pp, t, te);
                sh = t;
                sl += te + fmaf(a, b, -pp);
            }
            const float t = sh + sl;                        // renormalise: |sl| <= ulp(sh) / 2
            sl = sl - (t - sh);
            sh = t;
            if (r != c) {
                sh *= 2.0f;
                sl *= 2.0f;
            }
            hi[u] = sh;
            lo[u] = sl;
            if (sh != 0.0f) emax = max(emax, ilogbf(sh));
        }
    }
    emax = __reduce_max_sync(0xffffffffu, emax);
    const int eq = emax - 17;
    const float qinv = (eq > -127 && eq < 127) ? __uint_as_float(uint32_t(127 - eq) << 23) : 1.0f;
    const float qs = (eq > -127 && eq < 127) ? __uint_as_float(uint32_t(127 + eq) << 23) : 1.0f;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int e = lane + 32 * u;
        if (e < NG) {
            const float h = rintf(hi[u] * qinv) * qs;      // scalings by powers of two: exact
            sw->Sh[e] = h;
            sw->Sl[e] = (hi[u] - h) + lo[u];               // hi - h is exact
        }
    }
}

__device__ inline void write_pass_splits_kappa_rt(int M, SweepGlobalsF32 *sw, int lane)
{
    const float kv = (lane < M) ? sw->kappa[lane] : 0.0f;
    int ek = (kv != 0.0f) ? ilogbf(kv) : -1000;
    ek = __reduce_max_sync(0xffffffffu, ek);
    const int eqk = ek - 19;
    const float kqinv = (eqk > -127 && eqk < 127) ? __uint_as_float(uint32_t(127 - eqk) << 23) : 1.0f;
    const float kqs = (eqk > -127 && eqk < 127) ? __uint_as_float(uint32_t(127 + eqk) << 23) : 1.0f;
    if (lane < M) {
        const float h = rintf(kv * kqinv) * kqs;
        sw->kh[lane] = h;
        sw->kl[lane] = kv - h;                              // exact
    }
}

__device__ inline void write_pass_splits_rt(int M, SweepGlobalsF32 *sw, int lane)
{
    write_pass_splits_sigma_rt(M, sw, lane);
    write_pass_splits_kappa_rt(M, sw, lane);
}

// ---------------------------------------------------------------------------
// Column sums of rows [0, nrows) of a row-major [nrows][ns] FP64 array in
// global memory, in a fixed order: thread t (t < R ns, of the first nt
// threads) takes column t % ns and the t / ns-th of R chunks of consecutive
// rows (four interleaved accumulators) and writes the chunk sum to red[t].
// R = nt / ns clamped to [1, 8]; returns R.  FP64 additions are costly on
// this hardware (one warp instruction every few dozen cycles), so the rows
// are spread over as many threads as there are.
// ---------------------------------------------------------------------------
__device__ inline int chunk_sums(const double *__restrict__ part, int nrows, int ns, double *__restrict__ red,
                                 int tid, int nt)
{
    int R = nt / ns;
    R = R < 1 ? 1 : (R > 8 ? 8 : R);
    const int len = (nrows + R - 1) / R;
    for (int t = tid; t < R * ns; t += nt) {
        const int c = t / ns, j = t - c * ns;
        const int b0 = c * len, b1 = (b0 + len < nrows) ? b0 + len : nrows;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int b = b0;
        for (; b + 3 < b1; b += 4) {
            s0 += __ldcg(part + size_t(b) * ns + j);
            s1 += __ldcg(part + size_t(b + 1) * ns + j);
            s2 += __ldcg(part + size_t(b + 2) * ns + j);
            s3 += __ldcg(part + size_t(b + 3) * ns + j);
        }
        for (; b < b1; ++b) s0 += __ldcg(part + size_t(b) * ns + j);
        red[t] = (s0 + s1) + (s2 + s3);
    }
    return R;
}

// Total of column j from the R chunk sums of chunk_sums (chunk order).
__device__ __forceinline__ double chunk_total(const double *red, int R, int ns, int j)
{
    double s0 = 0.0, s1 = 0.0;
    int c = 0;
    for (; c + 1 < R; c += 2) {
        s0 += red[c * ns + j];
        s1 += red[(c + 1) * ns + j];
    }
    if (c < R) s0 += red[c * ns + j];
    return s0 + s1;
}

// ---------------------------------------------------------------------------
// Completion of a sweep launch, called by every thread of every block after
// the block wrote its row of `part` ([nblk][ns] FP64, then one row per
// group).  Thread 0 publishes the block's writes (a CTA barrier, then an
// acquire-release fetch-and-add on the counter) and takes a ticket.  Up to
// TICKET_SINGLE_MAX blocks the last block to arrive finishes the launch and
// reads every row.  Above, the last block of each group of TICKET_GROUP
// blocks sums the group's rows (fixed order, scratch: >= 512 doubles of
// shared memory) into the group's row and takes a second ticket; the last
// group's reducer finishes the launch and reads the group rows.  Returns true
// in the finishing block only, with the rows it reads in [*row0, *row0 +
// *nrows).  Counters are reset by the block that read them.
// ---------------------------------------------------------------------------
// Device-scope acquire-release fetch-and-add: publishes the block's writes
// (ordered before it by a CTA barrier) and acquires the other blocks'.
__device__ __forceinline__ unsigned atomic_add_acq_rel(unsigned *p, unsigned v)
{
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ inline bool finish_ticket(DevState *st, double *part, int nblk, int ns, volatile int *s_flag, int *row0,
                                     int *nrows, double *scratch)
{
    const int tid = threadIdx.x, nth = blockDim.x;
    __syncthreads();
    if (nblk == 1) {                                // the only block: its own writes are visible after the barrier
        *row0 = 0;
        *nrows = 1;
        return true;
    }
    if (nblk <= TICKET_SINGLE_MAX) {
        if (tid == 0) {
            const int last = (atomic_add_acq_rel(&st->ticket, 1u) == unsigned(nblk - 1)) ? 1 : 0;
            if (last) st->ticket = 0u;
            *s_flag = last;
        }
        __syncthreads();
        if (!*s_flag) return false;
        *row0 = 0;
        *nrows = nblk;
        return true;
    }
    const int g = blockIdx.x / TICKET_GROUP, ng = (nblk + TICKET_GROUP - 1) / TICKET_GROUP;
    const int b0 = g * TICKET_GROUP;
    const int gsz = (nblk - b0 < TICKET_GROUP) ? nblk - b0 : TICKET_GROUP;
    if (tid == 0) {
        const int last = (atomic_add_acq_rel(&st->gticket[g], 1u) == unsigned(gsz - 1)) ? 1 : 0;
        if (last) st->gticket[g] = 0u;
        *s_flag = last;
    }
    __syncthreads();
    if (!*s_flag) return false;
    const int R = chunk_sums(part + size_t(b0) * ns, gsz, ns, scratch, tid, nth);
    __syncthreads();
    double *out = part + size_t(nblk + g) * ns;
    for (int j = tid; j < ns; j += nth) out[j] = chunk_total(scratch, R, ns, j);
    __syncthreads();
    if (tid == 0) {
        const int last = (atomic_add_acq_rel(&st->ticket, 1u) == unsigned(ng - 1)) ? 1 : 0;
        if (last) st->ticket = 0u;
        *s_flag = last;
    }
    __syncthreads();
    if (!*s_flag) return false;
    *row0 = nblk;
    *nrows = ng;
    return true;
}

// ---------------------------------------------------------------------------
// (d)+(e): FP64 global update, ELBO and control, run by the whole block that
// finishes the launch (blockDim.x a multiple of 32, at least 96 threads).
// part: nrows rows of per-block (or per-group) statistics, laid out as in
// SweepCfg: packed lower G, g, T3, T4 (ln of mantissas), E4 (binary
// exponents), and with st->comp the compensated U.  ws: shared-memory
// workspace of at least gu_ws_doubles(M) doubles.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int gu_ws_doubles_rt(int M)
{
    // statistics (rounded up to 32), 10 M x M matrices, 10 M-vectors, 32 scalars, 512 of reduction scratch
    return ((M * (M + 1) / 2 + M + 4 + 31) / 32) * 32 + 10 * (M > 0 ? M * M : 1) + 10 * (M > 0 ? M : 1) + 32 + 512;
}

template <int M>
constexpr int gu_ws_doubles()
{
    return gu_ws_doubles_rt(M);
}

__device__ __forceinline__ void global_update_rt(int M, DevState *st, const double *__restrict__ part, int nrows,
                                                 const SweepArgs &a, double *ws)
{
    const int NG = M * (M + 1) / 2;
    const bool comp = st->comp != 0;
    const int NSTAT = NG + M + 3 + (comp ? 1 : 0);
    const int I_T3 = NG + M, I_T4 = NG + M + 1, I_E4 = NG + M + 2, I_U = NG + M + 3;
    const int MM = M > 0 ? M * M : 1;
    const int MV = M > 0 ? M : 1;
    const int MD = M > 0 ? M : 1;                   // divisor (loops over M*M entries are empty at M = 0)
    constexpr double LN2PI = 1.8378770664093454836;
    constexpr double LN2 = 0.69314718055994530942;
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
    const int nthm = nth - 32;                      // threads of the main warps
    const int mode = a.mode;
    const bool em = st->em != 0;
    const bool elbo_only = (mode == MODE_ELBO) && !em;   // the ELBO of given factors: nothing is updated
    const ElboConst *kc = (mode == MODE_ELBO) ? &st->kc_given : &st->kc_upd;

    double *stat = ws;
    double *Sg = stat + ((NSTAT + 31) / 32) * 32;   // Sigma0~ = L~ L~^T of this pass
    double *G = Sg + MM;                            // sum (w^2 - c) D D^T (full)
    double *A = G + MM;                             // Sigma0~ G
    double *B = A + MM;                             // Sigma0~ G Sigma0~
    double *Wn = B + MM;                            // new W^{-1}
    double *Lw = Wn + MM;                           // chol(W^{-1})
    double *Li = Lw + MM;                           // Lw^{-1}
    double *X = Li + MM;                            // C + Lambda_0^{-1} + q0 (kappa'-K0)(kappa'-K0)^T
    double *Lf = X + MM;                            // L~ (packed) in FP64
    double *L0s = Lf + MM;                          // Lambda_0^{-1}
    double *sv = L0s + MM;                          // Sigma0~ g
    double *dv = sv + MV;                           // kappa' - kappa~
    double *ko = dv + MV;                           // kappa~ (this pass)
    double *kn = ko + MV;                           // kappa'
    double *av = kn + MV;                           // K0 - kappa~
    double *gv = av + MV;                           // g
    double *rd = gv + MV;                           // 1 / diag(Lw)
    double *piv = rd + MV;                          // Cholesky pivots of W'^{-1}
    double *K0s = piv + MV;                         // K0
    double *sc = K0s + 2 * MV;                      // scalars (after K0 and the Cholesky column scratch)
    double *red = sc + 32;                          // reduction scratch [R][NSTAT]
    __shared__ int s_fail;

    if (warp < nwarp - 1) {
        const double V = st->V, q0 = st->q0;
        const double inv_V = kc->inv_V, inv_lam = kc->inv_lam, lam = kc->lam, nu = kc->nu, rs_nu = kc->rs_nu;
        // 1. rows -> chunk sums; FP64 copies of the pass factors and of the
        //    prior.  The data pass used the FP32 factor L~ and kappa~ of st->sw;
        //    its Q(beta_i) is the exact Eq. 20-21 posterior for Sigma0~ = L~ L~^T
        //    and kappa~, so every FP64 quantity below is taken with those
        //    values: each sweep is an exact coordinate step from the rounded
        //    globals and the ELBO sequence is smooth (FP32 rounding enters at
        //    second order only).
        const int R = chunk_sums(part, nrows, NSTAT, red, tid, nthm);
        for (int e = tid; e < NG; e += nthm) Lf[e] = static_cast<double>(st->sw.L[e]);
        for (int e = tid; e < M * M; e += nthm) {
            L0s[e] = st->L0inv[e];
            if (elbo_only) Wn[e] = st->Winv[e];
        }
        for (int i = tid; i < M; i += nthm) {
            ko[i] = static_cast<double>(st->sw.kappa[i]);
            K0s[i] = st->K0[i];
            av[i] = K0s[i] - ko[i];
            if (mode == MODE_ELBO && !em) kn[i] = st->kappa[i];
        }
        if (tid == 0) s_fail = 0;
        named_sync(BAR_MAIN, nthm);
        //    chunk sums -> totals, scattered into G (full) and g; Sigma0~
        for (int j = tid; j < NSTAT; j += nthm) {
            const double s = chunk_total(red, R, NSTAT, j);
            stat[j] = s;
            if (j < NG) {
                int r = static_cast<int>((sqrtf(8.0f * j + 1.0f) - 1.0f) * 0.5f);
                while (r * (r + 1) / 2 > j) --r;
                while ((r + 1) * (r + 2) / 2 <= j) ++r;
                const int cc = j - r * (r + 1) / 2;
                G[r * M + cc] = s;
                G[cc * M + r] = s;
            } else if (j < NG + M) {
                gv[j - NG] = s;
            }
        }
        named_arrive(BAR_T3, nth);                  // the statistics are in place for the scalar warp
        for (int e = tid; e < M * M; e += nthm) {
            const int r = e / MD, c = e - r * MD;
            const int kmax = r < c ? r : c;
            double s = 0.0;
            for (int k = 0; k <= kmax; ++k) s = fma(Lf[r * (r + 1) / 2 + k], Lf[c * (c + 1) / 2 + k], s);
            Sg[e] = s;
        }
        named_sync(BAR_MAIN, nthm);

        // 2. A = Sigma0~ G, s = Sigma0~ g
        for (int e = tid; e < M * M; e += nthm) {
            const int r = e / MD, c = e - r * MD;
            double s0 = 0.0, s1 = 0.0;
            int k = 0;
            for (; k + 1 < M; k += 2) {
                s0 = fma(Sg[r * M + k], G[k * M + c], s0);
                s1 = fma(Sg[r * M + k + 1], G[(k + 1) * M + c], s1);
            }
            if (k < M) s0 = fma(Sg[r * M + k], G[k * M + c], s0);
            A[e] = s0 + s1;
        }
        for (int i = tid; i < M; i += nthm) {
            double s0 = 0.0, s1 = 0.0;
            int k = 0;
            for (; k + 1 < M; k += 2) {
                s0 = fma(Sg[i * M + k], gv[k], s0);
                s1 = fma(Sg[i * M + k + 1], gv[k + 1], s1);
            }
            if (k < M) s0 = fma(Sg[i * M + k], gv[k], s0);
            sv[i] = s0 + s1;
        }
        named_sync(BAR_MAIN, nthm);
        // 3. B = Sigma0~ G Sigma0~, delta, kappa'
        for (int e = tid; e < M * M; e += nthm) {
            const int r = e / MD, c = e - r * MD;
            double s0 = 0.0, s1 = 0.0;
            int k = 0;
            for (; k + 1 < M; k += 2) {
                s0 = fma(A[r * M + k], Sg[k * M + c], s0);
                s1 = fma(A[r * M + k + 1], Sg[(k + 1) * M + c], s1);
            }
            if (k < M) s0 = fma(A[r * M + k], Sg[k * M + c], s0);
            B[e] = s0 + s1;
        }
        for (int i = tid; i < M; i += nthm) {
            if (em) {                               // Eq. 46: K' = (1/V) sum M_i = K~ + Sigma0~ g / V
                dv[i] = sv[i] * inv_V;
                kn[i] = ko[i] + dv[i];
            } else if (mode == MODE_ELBO) {         // kappa is given; kappa~ is its FP32 rounding
                dv[i] = kn[i] - ko[i];
            } else {
                dv[i] = fma(q0, av[i], sv[i]) * inv_lam;   // Eq. 24, centred on kappa~
                kn[i] = ko[i] + dv[i];
            }
        }
        named_sync(BAR_MAIN, nthm);
        // 4. W'^{-1} (Eq. 25, centred) and X
        for (int e = tid; e < M * M; e += nthm) {
            const int r = e / MD, c = e - r * MD;
            const double Bs = 0.5 * (B[r * M + c] + B[c * M + r]);
            if (em) {
                // Eq. 47: (1/V) sum (M_i M_i^T + Sigma_i) - K' K'^T = Sigma0~ + Sigma0~ G Sigma0~ / V - a a^T
                Wn[e] = fma(Bs, inv_V, Sg[e]) - dv[r] * dv[c];
            } else if (!elbo_only) {
                Wn[e] = L0s[e] + V * Sg[e] + Bs + q0 * av[r] * av[c] - lam * dv[r] * dv[c];
            } else {
                // C = V Sigma0~ + Sigma0~ G Sigma0~ - s delta^T - delta s^T + V delta delta^T
                const double Cm = V * Sg[e] + Bs - sv[r] * dv[c] - dv[r] * sv[c] + V * dv[r] * dv[c];
                X[e] = Cm + L0s[e] + q0 * (kn[r] - K0s[r]) * (kn[c] - K0s[c]);
            }
        }
        named_sync(BAR_MAIN, nthm);
        // 5. Cholesky of W'^{-1} (warp 0); its pivots go to the scalar warp
        if (warp == 0) {
            const int fail = warp_cholesky_rt(M, Wn, Lw, rd, piv, K0s + MV, lane);
            if (lane == 0 && fail) s_fail = 1;
            named_arrive(BAR_PIV, 64);
        }
        named_sync(BAR_MAIN, nthm);
        // 6. warp 0: tr(E[Lambda] X) with E[Lambda] = nu Li^T Li (Eq. 28);
        //    warp 1 (EM or the compensated form): tr(Sigma0~ G); the other main
        //    warps: the new globals.
        //    After the CAVI update of Q(K, Lambda) X equals the new W'^{-1}: with
        //    a = K0 - kappa~, X - W'^{-1} = -(s + q0 a) delta^T - delta (s + q0 a)^T
        //    + 2 lam delta delta^T = 0 since lam delta = s + q0 a (Eq. 24-25), so
        //    tr(E[Lambda] X) = nu M and only the ELBO of given factors forms it.
        if (warp == 0) {
            if (elbo_only) {
                warp_tri_inverse_rt(M, Lw, rd, Li, lane);
                double t0 = 0.0;
                for (int e = lane; e < M * M; e += 32) {
                    const int r = e / MD, c = e - r * MD;
                    double e0 = 0.0, e1 = 0.0;
                    int k = r > c ? r : c;
                    for (; k + 1 < M; k += 2) {
                        e0 = fma(Li[k * M + r], Li[k * M + c], e0);
                        e1 = fma(Li[(k + 1) * M + r], Li[(k + 1) * M + c], e1);
                    }
                    if (k < M) e0 = fma(Li[k * M + r], Li[k * M + c], e0);
                    t0 = fma(X[e], e0 + e1, t0);
                }
                const double t = warp_sum(t0);
                if (lane == 0) sc[6] = nu * t;
            } else if (lane == 0) {
                sc[6] = nu * M;
            }
        } else {
            if ((em || comp) && warp == 1) {
                double t1 = 0.0;
                for (int e = lane; e < M * M; e += 32) t1 = fma(Sg[e], G[e], t1);
                const double t = warp_sum(t1);
                if (lane == 0) sc[7] = t;
            }
            if (!elbo_only) {
                write_pass_globals_rt(M, st, Wn, Lw, em ? 1.0 : nu, em ? 1.0 : rs_nu, tid - 32, nthm - 32);
                for (int e = tid - 32; e < M * M; e += nthm - 32) st->Winv[e] = Wn[e];
                for (int i = tid - 32; i < M; i += nthm - 32) {
                    st->kappa[i] = kn[i];
                    st->sw.kappa[i] = static_cast<float>(kn[i]);
                }
            }
        }
        __syncwarp();
        __syncthreads();
        // the split globals of the next compensated pass (from the FP32 L~
        // and kappa~ just written by the other main warps)
        if (comp && !elbo_only && warp == 0) write_pass_splits_rt(M, &st->sw, lane);
        return;
    }

    // the scalar warp: what the final step reads, loaded while the main warps
    // reduce; ln|Sigma0~| of this pass (and, for EM, ln rho~); then E[rho]
    // and ln b_rho (Eq. 16-17, 29) or rho' = V / T3 (Eq. 45); then ln|W'^{-1}|;
    // then (lane 0) the ELBO, control and the scalar globals
    const double V = st->V, b0 = st->b0, tol = st->tol, elbo_prev = st->elbo_prev, given_brho = st->b_rho;
    const double a_rho = kc->a_rho, e0 = kc->e0, e_logb = kc->e_logb, e_ldw = kc->e_ldw, log_nu = kc->log_nu;
    const double nu = kc->nu, lam = kc->lam;
    const int iter = st->iter, target = st->target, max_iter = st->max_iter, status = st->status;
    const int prior_dropped = st->prior_dropped;
    double *trace = st->trace;
    const float erho_f = st->sw.erho;
    double x = 1.0;
    if (lane < M) x = static_cast<double>(st->sw.L[lane * (lane + 1) / 2 + lane]);
    else if (lane == 31 && em) x = static_cast<double>(erho_f);
    const double lx = log(x);
    const double lnS0 = warp_sum(lane < M ? 2.0 * lx : 0.0);
    const double lr = __shfl_sync(0xffffffffu, lx, 31);
    named_sync(BAR_T3, nth);
    const double T3 = stat[I_T3];
    const double T4 = fma(LN2, stat[I_E4], stat[I_T4]);
    const double U = comp ? stat[I_U] : 0.0;
    double q, lb = 0.0, brho = 0.0;
    if (em) {
        q = V / T3;                                 // rho' (Eq. 45)
    } else {
        brho = elbo_only ? given_brho : fma(0.5, T3, b0);
        q = a_rho / brho;                           // E[rho]
        lb = log(brho);
    }
    named_sync(BAR_PIV, 64);
    const double ldW = warp_logdet_rt(M, piv, lane);
    __syncthreads();
    if (lane != 0) return;

    double L;
    bool finite;
    if (em) {
        // ln p(r | theta~) = sum_i ln N(y_i; D_i^T K~, 1/rho~ + q_i): with the pass's sums,
        // V/2 (ln rho~ - ln 2 pi) - rho~/2 sum S_i - 1/2 sum ln(1 + rho~ q_i) - 1/2 tr(Sigma0~ G);
        // rho~ T3 + tr(Sigma0~ G) = U exactly, which the compensated form carries
        L = comp ? 0.5 * V * (lr - LN2PI) - 0.5 * (U + T4)
                 : 0.5 * V * (lr - LN2PI) - 0.5 * (fma(static_cast<double>(erho_f), T3, T4) + sc[7]);
        finite = isfinite(L) && isfinite(q) && q > 0.0 && !s_fail;
        st->a_rho = q;                              // point estimate as (rho, 1)
        st->b_rho = 1.0;
        st->nu = 1.0;
        st->lam = V;
        st->const_dropped = 0;
    } else {
        const double erb = elbo_only ? q * fma(0.5, T3, b0) : a_rho;   // E[rho] (b0 + T3/2)
        L = (fma(e_logb, lb, e0) - fma(e_ldw, ldW, 0.5 * sc[6])) + (fma(0.5 * V, lnS0, -0.5 * T4) - erb);
        if (comp) {
            // The ELBO depends on T3 and G at first order through
            // -1/2 (E[rho]' T3 + tr(E[Lambda]' Sigma0~ G Sigma0~)), which is
            // -1/2 (E[rho]~ T3 + tr(Sigma0~ G)) = -1/2 U at the fixed point of
            // the sweep (and exactly so for the ELBO of given factors): swap the
            // FP32 sums' part of it for the compensated U.
            L += 0.5 * (fma(static_cast<double>(erho_f), T3, sc[7]) - U);
        }
        finite = isfinite(L) && isfinite(brho) && brho > 0.0 && !s_fail;
        st->const_dropped = prior_dropped;
        if (!elbo_only) {
            st->a_rho = a_rho;
            st->b_rho = brho;
            st->nu = nu;
            st->lam = lam;
        }
    }
    for (int j = 0; j < M; ++j) finite = finite && isfinite(kn[j]);
    st->elbo = L;
    int it = iter, conv = 0;
    if (!elbo_only) {
        st->erho = q;
        st->sw.erho = static_cast<float>(q);
        st->lndetSigma0 = em ? ldW : fma(-double(M), log_nu, ldW);
        if (M <= S_FP32_MAX - 1) {
            st->carry_ldw = ldW;
            for (int j = 0; j < M; ++j) st->carry_piv[j] = piv[j];
            st->carry_ok = 1;
        }
        if (mode != MODE_INIT) {
            it = iter + 1;
            conv = (fabs(L - elbo_prev) < tol * fabs(L)) ? 1 : 0;
        } else {
            it = 0;
        }
        st->iter = it;
        st->converged = conv;
        if (trace && it <= max_iter) trace[it] = L;
    } else if (trace) {
        trace[0] = L;                               // sweep 0 of a fit started from given factors: L_0 of that state
    }
    st->elbo_prev = L;
    int stat_now = status;
    if (!finite && status == ST_OK) {
        st->status = ST_ENONFINITE;
        stat_now = ST_ENONFINITE;
    }
    if (a.use_cond) {
        const int keep = (mode == MODE_ITER || mode == MODE_INIT) && stat_now == ST_OK && !conv && it < target &&
                         it < max_iter;
        cudaGraphSetConditional(a.cond, keep ? 1u : 0u);
    }
}

template <int M>
__device__ __forceinline__ void global_update(DevState *st, const double *__restrict__ part, int nrows,
                                              const SweepArgs &a, double *ws)
{
    global_update_rt(M, st, part, nrows, a, ws);
}

// ---------------------------------------------------------------------------
// The fused sweep kernel.  COMP: the compensated form (U and the two-part T4
// for the stopping test, one more column of partials).
// ---------------------------------------------------------------------------
template <int S, bool COMP>
__global__ void __launch_bounds__(SweepCfg<S>::THREADS, COMP ? SweepCfg<S>::MINB_C : SweepCfg<S>::MINB)
    sweep_kernel(SweepArgs a)
{
    using C = SweepCfg<S>;
    constexpr int M = C::M, NG = C::NG, NSTAT = C::NSTAT;
    constexpr int NS = COMP ? C::NSTATC : C::NSTAT;        // columns of a partial row
    constexpr int NGR = COMP ? C::NGRPC : C::NGRP;
    constexpr int THREADS = C::THREADS, T = C::T;
    constexpr int STAGES = COMP ? C::STAGES_C : C::STAGES;
    constexpr size_t BAR_OFF = COMP ? C::SMEM_BYTES_C - 64 : C::RING_BYTES;
    static_assert(!COMP || S <= S_FP32_MAX, "compensated form: S <= 11");
    static_assert(size_t(gu_ws_doubles_rt(M)) * 8 <= size_t(STAGES) * C::STAGE_BYTES, "workspace exceeds the ring");
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + BAR_OFF);
    float4 *tab = reinterpret_cast<float4 *>(smem + C::OFF_TAB);     // compensated form only
    float *split = reinterpret_cast<float *>(smem + C::OFF_SPLIT);
    __shared__ int s_bad, s_last;

    DevState *st = a.st;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_bad = 0;

    // Every block takes the same decision: the control fields are only written
    // by the last block of a launch, after all other blocks have finished.
    const bool run = (a.mode != MODE_ITER) ||
                     (st->status == ST_OK && !st->converged && st->iter < st->target && st->iter < st->max_iter);

    float acc[NSTAT];
    double acc64[NGR];
    float prod = 1.0f, pl = 0.0f, uh = 0.0f, ul = 0.0f;
    int ex = 0;
#pragma unroll
    for (int i = 0; i < NSTAT; ++i) acc[i] = 0.0f;
#pragma unroll
    for (int g = 0; g < NGR; ++g) acc64[g] = 0.0;

    if (run) {
        // plain form: L~ and kappa~ in registers; compensated form: the split
        // globals in shared memory, and the table of profile terms built from them
        float A[COMP ? 1 : C::NGA], B[COMP ? 1 : C::MA];
        const float erho = st->sw.erho;          // 0 in sweep 0 of a CAVI fit from the paper's start: c_i = 0
        if constexpr (COMP) {
            for (int i = tid; i < C::SPLIT_FLOATS; i += THREADS) {
                float v;
                if (i < NG) v = st->sw.Sh[i];
                else if (i < 2 * NG) v = st->sw.Sl[i - NG];
                else if (i < 2 * NG + M) v = st->sw.kh[i - 2 * NG];
                else v = st->sw.kl[i - 2 * NG - M];
                split[i] = v;
            }
            A[0] = 0.0f;
            B[0] = 0.0f;
        } else {
#pragma unroll
            for (int i = 0; i < NG; ++i) A[i] = st->sw.L[i];
#pragma unroll
            for (int i = 0; i < M; ++i) B[i] = st->sw.kappa[i];
            if constexpr (NG == 0) A[0] = 0.0f;
            if constexpr (M == 0) B[0] = 0.0f;
        }

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
        if constexpr (COMP) {
            build_profile_table<S>(tab, split, erho, tid, THREADS);      // overlaps the first copies
            __syncthreads();
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
                    if constexpr (COMP) {
                        observe_comp<S>(x, rt[j], tab, split, erho, acc, prod, pl, uh, ul);
                        if (u & 1) peel_exponent2(prod, pl, ex);
                    } else {
                        observe<S>(x, rt[j], A, B, erho, acc, prod);
                        if (u & 1) peel_exponent(prod, ex);
                    }
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
                if constexpr (COMP)
                    flush_warp_comp<S>(acc, acc64, prod, pl, ex, uh, ul, lane);
                else
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
                    if constexpr (COMP) {
                        observe_comp<S>(x, __ldg(a.r + i), tab, split, erho, acc, prod, pl, uh, ul);
                        peel_exponent2(prod, pl, ex);
                    } else {
                        observe<S>(x, __ldg(a.r + i), A, B, erho, acc, prod);
                        peel_exponent(prod, ex);
                    }
                }
            }
        }
    }
    if constexpr (COMP)
        flush_warp_comp<S>(acc, acc64, prod, pl, ex, uh, ul, lane);
    else
        flush_warp<S>(acc, acc64, prod, ex, lane);
    __syncthreads();   // the ring is idle from here on: reuse it for the block reduction

    // block reduction in FP64, fixed order, then this block's partials
    double *s_red = reinterpret_cast<double *>(smem);      // [THREADS / 32][NGR * 32]
#pragma unroll
    for (int g = 0; g < NGR; ++g) s_red[warp * (NGR * 32) + g * 32 + lane] = acc64[g];
    __syncthreads();
    for (int j = tid; j < NS; j += THREADS) {
        double sm = 0.0;
#pragma unroll
        for (int w = 0; w < THREADS / 32; ++w) sm += s_red[w * (NGR * 32) + j];
        a.partials[size_t(blockIdx.x) * NS + j] = sm;
    }
    int row0, nrows;
    if (!finish_ticket(st, a.partials, gridDim.x, NS, &s_last, &row0, &nrows, reinterpret_cast<double *>(smem)))
        return;
    if (run && !s_bad) {
        // every copy of this block has landed, so the ring's shared memory
        // serves as the workspace of the global update
        global_update<M>(st, a.partials + size_t(row0) * NS, nrows, a, reinterpret_cast<double *>(smem));
    } else if (tid == 0 && a.use_cond) {
        cudaGraphSetConditional(a.cond, 0u);
    }
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
__device__ inline void elbo_const(ElboConst *k, int M, double a_rho, double nu, double lam, double V, double pc,
                                  const DevState *st, int lane)
{
    constexpr double LN2PI = 1.8378770664093454836;
    constexpr double LN2 = 0.69314718055994530942;
    constexpr double LNPI = 1.1447298858494002;
    double sp = 0.0, sl = 0.0;
    for (int j = lane; j < M; j += 32) {
        const double x = 0.5 * (nu - j);                 // (nu + 1 - (j + 1)) / 2
        sp += digamma_d(x);
        sl += lgamma(x);
    }
    sp = warp_sum(sp);
    sl = warp_sum(sl);
    if (lane == 0) {
        const double q0 = st->q0, n0 = st->n0, a0 = st->a0;
        const double lgamma_a = lgamma(a_rho), psi_a = digamma_d(a_rho), log_lam = log(lam);
        k->a_rho = a_rho;
        k->nu = nu;
        k->lam = lam;
        k->lgamma_a = lgamma_a;
        k->psi_a = psi_a;
        k->sum_psi_nu = sp;
        k->sum_lgamma_nu = sl;
        k->log_lam = log_lam;
        k->log_nu = log(nu);
        k->rs_nu = rs_of(nu);
        k->inv_lam = 1.0 / lam;
        k->inv_V = V > 0.0 ? 1.0 / V : 0.0;
        // Eq. 11 term by term, with E[ln rho] = psi(a_rho) - ln b_rho and
        // E[ln|Lambda|] = sum psi + M ln 2 - ln|W^{-1}|; what a sweep leaves
        // unchanged is collected in e0:
        //   E ln p(r | beta, rho)  V/2 (E ln rho - ln 2pi) - E[rho] T3/2
        //   E ln p(beta | K, L)    V/2 (E ln|L| - M ln 2pi) - tr(E[L] C)/2 - V M/(2 lam)
        //   E ln p(K | L)          E ln|L|/2 - q0 ((kappa-K0)^T E[L] (kappa-K0) + M/lam)/2
        //   E ln p(L)              (n0-M-1)/2 E ln|L| - tr(Lambda_0^{-1} E[L])/2
        //   E ln p(rho)            (a0-1) E ln rho - b0 E[rho]
        //   H[Q(beta)]             (V ln|Sigma0~| - T4)/2 + V M (1 + ln 2pi)/2
        //   H[Q(K | L)]            -E ln|L|/2 - M (ln lam - ln 2pi)/2 + M/2
        //   H[Q(L)] (M > 0)        -ln B(W, nu) - (nu-M-1)/2 E ln|L| + nu M/2
        //   H[Q(rho)]              a_rho - ln b_rho + lnGamma(a_rho) + (1 - a_rho) psi(a_rho)
        // plus the prior-only constant pc.
        const double cr = 0.5 * V + (a0 - 1.0);                                          // of E ln rho
        const double cl = 0.5 * V + 0.5 * (n0 - M - 1.0) - (M > 0 ? 0.5 * (nu - M - 1.0) : 0.0);   // of E ln|L|
        double e0 = pc + cr * psi_a + cl * (sp + M * LN2);
        e0 += -0.5 * V * LN2PI - 0.5 * V * M * LN2PI - 0.5 * (V + q0) * M / lam + 0.5 * V * M * (1.0 + LN2PI);
        e0 += -0.5 * M * (log_lam - LN2PI) + 0.5 * M;
        if (M > 0) e0 += 0.5 * nu * M * LN2 + 0.25 * M * (M - 1) * LNPI + sl + 0.5 * nu * M;
        e0 += a_rho + lgamma_a + (1.0 - a_rho) * psi_a;
        k->e0 = e0;
        k->e_logb = -(cr + 1.0);
        k->e_ldw = cl + (M > 0 ? 0.5 * nu : 0.0);
    }
}

// The set-up body for one state, run by one warp (lane = 0..31); A and Lc
// are shared-memory scratch of M*M doubles each.
__device__ inline void setup_state_rt(int M, DevState *st, int init, int lane, double *A, double *Lc)
{
    constexpr double LN2PI = 1.8378770664093454836;
    constexpr double LN2 = 0.69314718055994530942;
    constexpr double LNPI = 1.1447298858494002;
    __shared__ double s_rd[MMAX], s_piv[MMAX], s_col[MMAX];
    for (int i = lane; i < M * M; i += 32) A[i] = st->L0inv[i];
    __syncwarp();
    int fail = warp_cholesky_rt(M, A, Lc, s_rd, s_piv, s_col, lane);
    __syncwarp();
    const double l0 = warp_logdet_rt(M, s_piv, lane);
    // prior-only terms: M/2 (ln q0 - ln 2 pi) + a0 ln b0 - lnGamma(a0) + ln B(Lambda_0, n0)
    const double n0 = st->n0;
    const bool proper = (M == 0) || (n0 > M - 1.0);
    const double lg0 = warp_sum((lane < M && proper) ? lgamma(0.5 * (n0 - lane)) : 0.0);
    double pc = 0.0;
    if (lane == 0) {
        st->lndetL0inv = l0;
        pc = 0.5 * M * (log(st->q0) - LN2PI) + st->a0 * log(st->b0) - lgamma(st->a0);
        if (M > 0 && proper)                            // ln B(W0, n0), ln|W0| = -ln|Lambda_0^{-1}|
            pc += 0.5 * n0 * l0 - 0.5 * n0 * M * LN2 - 0.25 * M * (M - 1) * LNPI - lg0;
        st->prior_const = pc;
        st->prior_dropped = (M > 0 && !proper) ? 1 : 0;
    }
    pc = __shfl_sync(0xffffffffu, pc, 0);
    const double V = st->V;
    elbo_const(&st->kc_upd, M, st->a0 + 0.5 * V, n0 + V, st->q0 + V, V, pc, st, lane);
    if (!init) elbo_const(&st->kc_given, M, st->a_rho, st->nu, st->lam, V, pc, st, lane);
    __syncwarp();
    if (!init)
        for (int i = lane; i < M * M; i += 32) A[i] = st->Winv[i];
    __syncwarp();
    // the pass factors of sweep 0: from (Lambda_0^{-1}, nu = 1) or (W^{-1}, nu)
    const double nu = init ? 1.0 : st->nu;
    fail |= warp_cholesky_rt(M, A, Lc, s_rd, s_piv, s_col, lane);
    __syncwarp();
    write_pass_globals_rt(M, st, A, Lc, nu, rs_of(nu), lane, 32);
    const double ld = warp_logdet_rt(M, s_piv, lane);
    for (int i = lane; i < M; i += 32) {
        const double kv = init ? st->K0[i] : st->kappa[i];
        st->sw.kappa[i] = static_cast<float>(kv);
        if (init) st->kappa[i] = kv;
    }
    for (int g = lane; g < TICKET_GROUPS_MAX; g += 32) st->gticket[g] = 0u;
    __syncwarp();                                    // sw.L and sw.kappa are in place
    if (st->comp && M < S_FP32_MAX) write_pass_splits_rt(M, &st->sw, lane);
    if (lane == 0) {
        st->lndetSigma0 = ld - M * log(nu);
        st->erho = init ? 0.0 : st->a_rho / st->b_rho;
        st->sw.erho = static_cast<float>(st->erho);
        st->ticket = 0u;
        st->carry_ok = 0;
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
