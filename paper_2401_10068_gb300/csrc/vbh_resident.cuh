// vbh_resident.cuh -- the sweep loop of a data set that fits in the shared
// memory of the GPU: one cooperative launch runs every sweep of a
// vbh_fit_step call.
//
// Each block copies its contiguous slice of (r, d) into shared memory once
// and keeps it there.  Its warps have two roles:
//   * the PASS warps (all but the last) run steps (a)-(c) of the fused sweep
//     over the slice (the same per-observation arithmetic, plain or
//     compensated, and the same FP32 -> FP64 flushes), publish the block's
//     FP64 partial row, collect every block's row and run the matrix part of
//     step (d): Q(K, Lambda) (Eq. 22-25, centred) and the Cholesky factor of
//     the new W^{-1} that gives the FP32 pass factors of the next sweep;
//   * the ELBO warp (the last) forms E[rho] (Eq. 16-17, 29) for the next pass
//     during that chain, and then -- while the pass warps already stream the
//     NEXT sweep -- the ELBO of Eq. 11, the stopping test and the write-back
//     of the fit's state.
// Every block collects the same rows and sums them in the same order, so
// every block computes the same FP64 globals and takes the same stop
// decision; block 0 updates the fit's own state (and its ELBO trace), the
// other blocks private copies of it.  The expressions that produce kappa,
// W^{-1} and the pass factors are those of the streaming sweep's update, so a
// fit resumed from its saved factors continues bit for bit.
//
// Why this shape: on this GPU a dependent FP64 add or multiply-add costs 64
// cycles and an FP64 logarithm about 2,000, so the FP64 update, not the data,
// sets the time of a sweep over a small data set.  The ELBO's logarithms and
// the state write-back are therefore taken off the path between two passes,
// the next pass starting speculatively: when the ELBO warp finds that sweep t
// met the stopping rule (or became non-finite), the pass of sweep t + 1 is
// dropped before any of its results are applied, so the state is exactly the
// state after sweep t.  The logarithms of the ELBO use a table-driven method
// (log_tang) of about a quarter of the library's latency.
//
// Exchange of the partial rows: a block writes its row of sweep k into the
// half k mod 2 of the partials buffer as tagged values -- the two lowest bits
// of each FP64 value replaced by (k + 1) mod 4 -- and a reader polls every
// value until it carries that tag.  An aligned 8-byte access is single-copy
// atomic, so each value is its own flag: no fence and no second read.  The
// reader clears the tag bits before it sums, so the partial sums lose their
// last two bits (a relative change below 2^-51) in the same way in every
// block and whatever the sweep's number within the launch.  A block can only write its row of sweep
// k + 2 after it has seen every row of sweep k + 1, each of which was written
// after its writer had read all rows of sweep k: the two halves suffice, and
// a value of sweep k - 2 (tag k - 1) is never taken for one of sweep k.  The
// buffer is zeroed before each launch (tag 0, which sweeps 0 and 1 do not use).
// Every wait is bounded (2 s of wall time); a wait that runs out records
// VBH_ETIMEOUT in the fit's status and ends the launch in that block.
// Co-residency of the blocks is what the cooperative launch guarantees.
#pragma once

#include "vbh_sweep.cuh"

namespace vbh {

constexpr uint64_t RESIDENT_WAIT_NS = 2000000000ull;   // limit of every wait on another block (2 s)
constexpr int BAR_PASS = 4;                            // named barrier of the pass warps

// What the ELBO of sweep k needs from its update, kept until the ELBO warp
// has used it (two records: sweeps k and k + 1 overlap).
struct ElboIn {
    double T3, T4, U, trSG, brho, q, lnS0, lr;
    double piv[S_FP32_MAX - 1];
    float erho_f;           // E[rho] of the pass
    int fail;               // the Cholesky factorisation of W'^{-1} failed
};

template <int S, bool COMP>
struct ResidentCfg {
    using C = SweepCfg<S>;
    static constexpr int M = C::M;
    static constexpr int MM = M > 0 ? M * M : 1, MV = M > 0 ? M : 1;
    static constexpr int THREADS = 256;
    static constexpr int PT = THREADS - 32;                  // pass threads (warps 0 .. 6)
    static constexpr int PW = PT / 32;
    static constexpr int FLUSH = 64;                         // observations per thread per FP32 chunk
    static constexpr int NS = COMP ? C::NSTATC : C::NSTAT;   // columns of a partial row
    static constexpr int NGR = COMP ? C::NGRPC : C::NGRP;
    static constexpr int NSTAT_R = ((NS + 31) / 32) * 32;
    // FP64 workspace (doubles): statistics, 7 matrices, 10 vectors, Cholesky column,
    // reduction scratch, block-reduction scratch, logarithm table
    static constexpr int D_STAT = 0;
    static constexpr int D_SG = D_STAT + NSTAT_R;
    static constexpr int D_G = D_SG + MM, D_A = D_G + MM, D_B = D_A + MM, D_WN = D_B + MM, D_LW = D_WN + MM;
    static constexpr int D_L0S = D_LW + MM;
    static constexpr int D_SV = D_L0S + MM, D_DV = D_SV + MV, D_KO = D_DV + MV, D_KN = D_KO + MV, D_AV = D_KN + MV;
    static constexpr int D_GV = D_AV + MV, D_RD = D_GV + MV, D_PIV = D_RD + MV, D_K0S = D_PIV + MV;
    static constexpr int D_COL = D_K0S + MV, D_RED = D_COL + 32;
    // every block's partial row of the current sweep (at most 48 KB): at most RB_ROWS blocks
    static constexpr int RB_ROWS = (6144 / NS < 152) ? 6144 / NS : 152;
    static constexpr int D_SRED = D_RED + ((RB_ROWS + 3) / 4) * NS;   // red: the first level of the row tree
    static constexpr int D_LOG = D_SRED + PW * NGR * 32;
    static constexpr int D_RB = D_LOG + 256;
    // M <= 3: coefficients of the W'^{-1} step, from the pass factors (resident_pre_coef)
    static constexpr bool COEF = M <= 3;
    // (packed lower-triangle entries pe = r (r + 1) / 2 + c, c <= r)
    static constexpr int D_CW = D_RB + RB_ROWS * NS;           // [NG]      W'^{-1} terms without the sums
    static constexpr int D_QC = D_CW + C::NGA;                 // [NG][NG]  weights of the packed G entries
    static constexpr int D_SL = D_QC + C::NGA * C::NGA;        // [M][M]    weights of g in delta
    static constexpr int D_CD = D_SL + MM;                     // [M]       delta without the sums
    static constexpr int D_TW = D_CD + MV;                     // [NG]      W'^{-1} before the delta term
    static constexpr int D_LF = D_TW + C::NGA;                 // [NG]      L~ in FP64
    static constexpr int D_END = COEF ? D_LF + C::NGA : D_CW;
    static constexpr int IPT = (((RB_ROWS + 3) / 4) * NS + PT - 1) / PT;   // 4-row items a pass thread collects
    static_assert(IPT * 4 <= 32, "one pending bit per collected value");
    static constexpr size_t OFF_WS = 0;
    static constexpr size_t OFF_EI = ((size_t(D_END) * 8 + 127) / 128) * 128;
    static constexpr size_t OFF_SG = OFF_EI + ((2 * sizeof(ElboIn) + 127) / 128) * 128;
    static constexpr size_t OFF_TAB = OFF_SG + ((sizeof(SweepGlobalsF32) + 127) / 128) * 128;
    static constexpr size_t OFF_SPLIT = OFF_TAB + (COMP ? C::TAB_BYTES : 0);
    static constexpr size_t OFF_SLICE = OFF_SPLIT + (COMP ? C::SPLIT_BYTES : 0);
    static constexpr size_t OBS_BYTES = size_t(S + 1) * 4;  // r and the S profile entries
    static_assert(M <= S_FP32_MAX - 1, "resident loop: S <= 11");
};

// Barriers of the resident kernel.  Both are aligned barriers: every thread of
// a warp must reach them together, so a warp that may have diverged (a lane-0
// branch, a partial loop) reconverges first.
__device__ __forceinline__ void cta_sync()
{
    __syncwarp();
    __syncthreads();
}

__device__ __forceinline__ void pass_sync(int pt)
{
    __syncwarp();
    named_sync(BAR_PASS, pt);
}

// Relaxed 64-bit load / store at GPU scope (single-copy atomic): the partial
// rows are exchanged as tagged values (see resident_kernel).
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// What the ELBO warp reads of the fit, loaded once per launch (the state in
// global memory is only written during the loop).
struct FitConst {
    double V, b0, a_rho, nu, lam, e0, e_logb, e_ldw, log_nu, tol, inv_nus;
    double *trace;
    int max_iter, prior_dropped;
    bool em, comp;
};

__device__ __forceinline__ FitConst fit_const(const DevState *st)
{
    FitConst c;
    const ElboConst *kc = &st->kc_upd;
    c.V = st->V;
    c.b0 = st->b0;
    c.a_rho = kc->a_rho;
    c.nu = kc->nu;
    c.lam = kc->lam;
    c.e0 = kc->e0;
    c.e_logb = kc->e_logb;
    c.e_ldw = kc->e_ldw;
    c.log_nu = kc->log_nu;
    c.tol = st->tol;
    c.em = st->em != 0;
    c.comp = st->comp != 0;
    c.inv_nus = c.em ? 1.0 : 1.0 / kc->nu;
    c.trace = st->trace;
    c.max_iter = st->max_iter;
    c.prior_dropped = st->prior_dropped;
    return c;
}

// ---------------------------------------------------------------------------
// The ELBO warp's part of step (d) (lane 0): E[rho] for the next pass from T3
// (Eq. 16-17, 29; EM: rho' = V / T3, Eq. 45), and the scalars the ELBO of
// this sweep takes.
// ---------------------------------------------------------------------------
template <int M>
__device__ __forceinline__ void resident_rho(const FitConst &fc, const double *stat, int i_u, SweepGlobalsF32 *sg,
                                             ElboIn *ei)
{
    constexpr double LN2 = 0.69314718055994530942;
    constexpr int NG = M * (M + 1) / 2;
    constexpr int I_T3 = NG + M, I_T4 = NG + M + 1, I_E4 = NG + M + 2;
    const double T3 = stat[I_T3];
    const double T4 = fma(LN2, stat[I_E4], stat[I_T4]);
    const double U = fc.comp ? stat[i_u] : 0.0;
    double q, brho = 0.0;
    if (fc.em) {
        q = fc.V / T3;
    } else {
        brho = fma(0.5, T3, fc.b0);
        q = fc.a_rho / brho;
    }
    ei->T3 = T3;
    ei->T4 = T4;
    ei->U = U;
    ei->brho = brho;
    ei->q = q;
    sg->erho = static_cast<float>(q);
}

// Finite (not inf or nan), by the exponent field alone.
__device__ __forceinline__ bool finite_bits(double x) { return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff; }

// Sum of v over lanes 0 .. n - 1 (n <= 32 at compile time; the other lanes
// pass 0): a butterfly over as many levels as n needs; every lane gets the
// total of its group, lane 0 that of lanes 0 .. n - 1 (a fixed order).
template <int N>
__device__ __forceinline__ double lane_sum(double v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
        if (off < N) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// What the ELBO warp's decision on a sweep leaves for its write-back (lane 0).
struct ElboOut {
    double L, ldW;
    int conv, finite;
};

// ---------------------------------------------------------------------------
// The ELBO warp's work on sweep `it`, in two parts.  resident_elbo_decide (on
// the path to the next barrier): the ELBO of Eq. 11 (EM: ln p(r | theta~),
// Eq. 42-47) with the expressions of the streaming sweep's update (the
// logarithms by log_tang, one per lane: the pivots of W'^{-1} in lanes < M,
// b_rho in lane 31) and the stopping test; returns, in every lane, whether
// the fit stops after this sweep (converged, non-finite, or a status set).
// resident_elbo_store (after the barrier, while the rows are exchanged): the
// write-back of the state; its running scalars (the previous ELBO, the
// status, ln|W'^{-1}| for the next sweep's ln|Sigma0~|) live in lane 0's
// registers.
// ---------------------------------------------------------------------------
template <int M>
__device__ bool resident_elbo_decide(const FitConst &fc, const ElboIn &ei, const double *ws_kn, const double *ltab,
                                     double elbo_prev, int status, ElboOut &o, int lane)
{
    constexpr double LN2PI = 1.8378770664093454836;
    double arg = 1.0;
    if (lane < M) arg = ei.piv[lane];
    else if (lane == 31 && !fc.em) arg = ei.brho;
    const double lx = log_tang(arg, ltab);
    const double ldW = lane_sum<M>(lane < M ? lx : 0.0);
    const double l31 = __shfl_sync(0xffffffffu, lx, 31);
    int stop = 0;
    if (lane == 0) {
        double L;
        bool finite;
        const double T3 = ei.T3, T4 = ei.T4, U = ei.U;
        if (fc.em) {
            L = fc.comp ? 0.5 * fc.V * (ei.lr - LN2PI) - 0.5 * (U + T4)
                        : 0.5 * fc.V * (ei.lr - LN2PI) -
                              0.5 * (fma(static_cast<double>(ei.erho_f), T3, T4) + ei.trSG);
            finite = finite_bits(L) && finite_bits(ei.q) && __double_as_longlong(ei.q) > 0 && !ei.fail;
        } else {
            const double sc6 = fc.nu * M;
            L = (fma(fc.e_logb, l31, fc.e0) - fma(fc.e_ldw, ldW, 0.5 * sc6)) +
                (fma(0.5 * fc.V, ei.lnS0, -0.5 * T4) - fc.a_rho);
            if (fc.comp) L += 0.5 * (fma(static_cast<double>(ei.erho_f), T3, ei.trSG) - U);
            finite = finite_bits(L) && finite_bits(ei.brho) && __double_as_longlong(ei.brho) > 0 && !ei.fail;
        }
#pragma unroll
        for (int j = 0; j < M; ++j) finite = finite && finite_bits(ws_kn[j]);
        const int conv = (fabs(L - elbo_prev) < fc.tol * fabs(L)) ? 1 : 0;
        o.L = L;
        o.ldW = ldW;
        o.conv = conv;
        o.finite = finite ? 1 : 0;
        stop = (conv || !finite || status != ST_OK) ? 1 : 0;
    }
    return __shfl_sync(0xffffffffu, stop, 0) != 0;
}

template <int M>
__device__ __forceinline__ void resident_elbo_store(DevState *st, const FitConst &fc, const ElboIn &ei,
                                                    const double *ws_wn, const double *ws_kn,
                                                    const SweepGlobalsF32 *sg, int it, const ElboOut &o,
                                                    double &elbo_prev, int &status, double &ldw, int lane)
{
    constexpr int NG = M * (M + 1) / 2;
    // W^{-1}, Sigma0 = W^{-1}/nu, kappa and the pass factors (every lane a share)
    for (int e = lane; e < M * M; e += 32) {
        st->Winv[e] = ws_wn[e];
        st->Sigma0[e] = ws_wn[e] * fc.inv_nus;
    }
    for (int i = lane; i < NG; i += 32) {
        st->sw.L[i] = sg->L[i];
        if (fc.comp) {
            st->sw.Sh[i] = sg->Sh[i];
            st->sw.Sl[i] = sg->Sl[i];
        }
    }
    for (int i = lane; i < M; i += 32) {
        st->kappa[i] = ws_kn[i];
        st->carry_piv[i] = ei.piv[i];
        st->sw.kappa[i] = sg->kappa[i];
        if (fc.comp) {
            st->sw.kh[i] = sg->kh[i];
            st->sw.kl[i] = sg->kl[i];
        }
    }
    if (lane == 0) {
        if (fc.em) {
            st->a_rho = ei.q;
            st->b_rho = 1.0;
            st->nu = 1.0;
            st->lam = fc.V;
            st->const_dropped = 0;
        } else {
            st->const_dropped = fc.prior_dropped;
            st->a_rho = fc.a_rho;
            st->b_rho = ei.brho;
            st->nu = fc.nu;
            st->lam = fc.lam;
        }
        st->elbo = o.L;
        st->erho = ei.q;
        st->sw.erho = sg->erho;
        st->lndetSigma0 = fc.em ? o.ldW : fma(-double(M), fc.log_nu, o.ldW);
        st->iter = it;
        st->converged = o.conv;
        if (fc.trace && it <= fc.max_iter) fc.trace[it] = o.L;
        st->elbo_prev = o.L;
        elbo_prev = o.L;
        if (!o.finite && status == ST_OK) {
            st->status = ST_ENONFINITE;
            status = ST_ENONFINITE;
        }
        st->carry_ldw = o.ldW;
        st->carry_ok = 1;
        ldw = o.ldW;
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Before the matrix chain of a sweep, from the pass factors that sweep reads:
// Sigma0~ = L~ L~^T and kappa~ in FP64 and K0 - kappa~ (threads t0, t0 + nt,
// ...), the expressions of the streaming update.
// ---------------------------------------------------------------------------
template <int M>
__device__ __forceinline__ void resident_pre_mat(const SweepGlobalsF32 *sg, double *Sg, double *ko, double *av,
                                                const double *K0s, int t0, int nt)
{
    constexpr int MD = M > 0 ? M : 1;
    for (int e = t0; e < M * M; e += nt) {
        const int r = e / MD, c = e - r * MD;
        const int kmax = r < c ? r : c;
        double s = 0.0;
        for (int k = 0; k <= kmax; ++k)
            s = fma(static_cast<double>(sg->L[r * (r + 1) / 2 + k]), static_cast<double>(sg->L[c * (c + 1) / 2 + k]),
                    s);
        Sg[e] = s;
    }
    for (int i = t0; i < M; i += nt) {
        ko[i] = static_cast<double>(sg->kappa[i]);
        av[i] = K0s[i] - ko[i];
    }
}

// ---------------------------------------------------------------------------
// M <= 3: Eq. 25 (EM: Eq. 47) with the pass factors' part taken out of the
// chain.  With Sigma0~ symmetric and G symmetric, Sigma0~ G Sigma0~ is
// symmetric and its entry (r, c) is linear in the packed entries G_kl (k >= l):
//   B_rc = sum_k Sg_rk Sg_kc G_kk + sum_{k > l} (Sg_rk Sg_lc + Sg_rl Sg_kc) G_kl,
// and delta_r = (q0 (K0 - kappa~)_r + (Sigma0~ g)_r) / lambda (EM: (Sigma0~ g)_r / V).
// So, before the sums of the sweep arrive,
//   Cw_rc = Lambda_0^{-1}_rc + V Sg_rc + q0 a_r a_c   (EM: Sg_rc),
//   Qc_rc,kl = the weights above (EM: times 1/V),  Sl_rk = Sg_rk / lambda (EM: / V),
//   cd_r = q0 a_r / lambda (EM: 0),
// and after them W'^{-1}_rc = Cw_rc + sum Qc G - lambda delta_r delta_c (EM: - delta_r delta_c),
// a few FP64 instructions per lane.
// ---------------------------------------------------------------------------
// The three stages, each a few FP64 instructions per item with the items
// dealt round robin (threads t0, t0 + nt, ...; the caller synchronises
// between stages): (1) L~ and kappa~ in FP64 and K0 - kappa~; (2) Sigma0~ =
// L~ L~^T (lower triangle, mirrored; the expressions of resident_pre_mat);
// (3) the coefficients, lower triangle only (W'^{-1} is formed symmetric).
__device__ __forceinline__ void packed_rc(int pe, int &r, int &c)
{
    r = 0;
    while ((r + 1) * (r + 2) / 2 <= pe) ++r;
    c = pe - r * (r + 1) / 2;
}

template <int M>
__device__ __forceinline__ void resident_pre_small_1(const SweepGlobalsF32 *sg, double *Lf, double *ko, double *av,
                                                    const double *K0s, int t0, int nt)
{
    constexpr int NG = M * (M + 1) / 2;
    for (int i = t0; i < NG + M; i += nt) {
        if (i < NG) {
            Lf[i] = static_cast<double>(sg->L[i]);
        } else {
            const int j = i - NG;
            ko[j] = static_cast<double>(sg->kappa[j]);
            av[j] = K0s[j] - ko[j];
        }
    }
}

template <int M>
__device__ __forceinline__ void resident_pre_small_2(const double *Lf, double *Sg, int t0, int nt)
{
    constexpr int NG = M * (M + 1) / 2;
    for (int pe = t0; pe < NG; pe += nt) {
        int r, c;
        packed_rc(pe, r, c);
        double s = 0.0;
        for (int k = 0; k <= c; ++k) s = fma(Lf[r * (r + 1) / 2 + k], Lf[c * (c + 1) / 2 + k], s);
        Sg[r * M + c] = s;
        Sg[c * M + r] = s;
    }
}

template <int M>
__device__ __forceinline__ void resident_pre_small_3(const double *Sg, const double *av, const double *L0s, double *Cw,
                                                    double *Qc, double *Sl, double *cd, bool em, double V, double q0,
                                                    double inv_lam, double inv_V, int t0, int nt)
{
    constexpr int NG = M * (M + 1) / 2, NGA = NG > 0 ? NG : 1;
    const double f2 = em ? inv_V : inv_lam;
    for (int t = t0; t < NG * NG + NG + M; t += nt) {
        if (t < NG * NG) {
            const int pe = t / NGA, pk = t - pe * NGA;
            int r, c, k, l;
            packed_rc(pe, r, c);
            packed_rc(pk, k, l);
            const double w = (k == l) ? Sg[r * M + k] * Sg[k * M + c]
                                      : fma(Sg[r * M + k], Sg[l * M + c], Sg[r * M + l] * Sg[k * M + c]);
            Qc[pe * NGA + pk] = em ? w * inv_V : w;
        } else if (t < NG * NG + NG) {
            const int pe = t - NG * NG;
            int r, c;
            packed_rc(pe, r, c);
            Cw[pe] = em ? Sg[r * M + c] : fma(q0 * av[r], av[c], fma(V, Sg[r * M + c], L0s[r * M + c]));
            const double sl = Sg[r * M + c] * f2;
            Sl[r * M + c] = sl;
            Sl[c * M + r] = sl;
        } else {
            const int i = t - NG * NG - NG;
            cd[i] = em ? 0.0 : q0 * av[i] * inv_lam;
        }
    }
}

// Stages 1 and 2 by the pass warps (one kind of item per warp, on different SM
// sub-partitions), between the block's row and the first barrier; stage 3 is
// the ELBO warp's, while the rows are exchanged.
template <int M>
__device__ __forceinline__ void resident_pre_small_12(const SweepGlobalsF32 *sg, double *Lf, double *Sg, double *ko,
                                                     double *av, const double *K0s, int warp, int lane, int pt)
{
    constexpr int NG = M * (M + 1) / 2;
    if (warp == 0 && lane < NG) Lf[lane] = static_cast<double>(sg->L[lane]);
    if (warp == 1 && lane < M) {
        ko[lane] = static_cast<double>(sg->kappa[lane]);
        av[lane] = K0s[lane] - ko[lane];
    }
    pass_sync(pt);
    if (warp == 0) resident_pre_small_2<M>(Lf, Sg, lane, 32);
}

// ---------------------------------------------------------------------------
// The ELBO's logarithms of the pass factors a sweep reads (ELBO warp):
// ln|Sigma0~| = sum_j ln L~_jj^2 and, for EM, ln E[rho]~ (by log_tang).  When
// the update that produced these factors left ln|W'^{-1}| and the pivots of
// W'^{-1} (prev_piv and ldw_prev, lane 0) the first comes from them: L~_jj =
// fl32(Lw_jj rs) with Lw_jj^2 ~ piv_j and rs^2 = 1/nu (EM: 1), so
//   ln L~_jj^2 = ln piv_j + ln rs^2 + ln(1 + D_j),  D_j = L~_jj^2 / (piv_j rs^2) - 1,
// |D_j| < 2^-22 and ln(1 + D) = D - D^2/2 to 2^-66.  Otherwise (factors from
// a set-up) the logarithms are taken directly.
// ---------------------------------------------------------------------------
template <int M>
__device__ __forceinline__ void resident_pre_logs(const FitConst &fc, const SweepGlobalsF32 *sg, const double *ltab,
                                                 const double *prev_piv, double ldw_prev, ElboIn *ei, int lane)
{
    const double ln_rs2 = fc.em ? 0.0 : -fc.log_nu;          // ln(1/nu)
    double lnS0, lr = 0.0;
    if (prev_piv) {
        double d = 0.0;
        if (lane < M) {
            const double l = static_cast<double>(sg->L[lane * (lane + 1) / 2 + lane]);
            const double ref = prev_piv[lane] * fc.inv_nus;                        // piv_j rs^2
            const double D = fma(l, l, -ref) * static_cast<double>(1.0f / static_cast<float>(ref));
            d = fma(-0.5 * D, D, D);
        }
        lnS0 = fma(double(M), ln_rs2, ldw_prev) + lane_sum<M>(d);
        if (fc.em) {
            const double lx = log_tang(lane == 31 ? static_cast<double>(sg->erho) : 1.0, ltab);
            lr = __shfl_sync(0xffffffffu, lx, 31);
        }
    } else {
        double x = 1.0;
        if (lane < M) x = static_cast<double>(sg->L[lane * (lane + 1) / 2 + lane]);
        else if (lane == 31 && fc.em) x = static_cast<double>(sg->erho);
        const double lx = log_tang(x, ltab);
        lnS0 = lane_sum<M>(lane < M ? 2.0 * lx : 0.0);
        lr = __shfl_sync(0xffffffffu, lx, 31);
    }
    if (lane == 0) {
        ei->lnS0 = lnS0;
        ei->lr = lr;
        ei->erho_f = sg->erho;
    }
}

template <int S, bool COMP>
__global__ void __launch_bounds__(ResidentCfg<S, COMP>::THREADS, 1) resident_kernel(ResidentArgs a)
{
    using C = SweepCfg<S>;
    using R = ResidentCfg<S, COMP>;
    constexpr int M = C::M, NG = C::NG, NSTAT = C::NSTAT;
    constexpr int NS = R::NS, NGR = R::NGR, THREADS = R::THREADS, PT = R::PT, PW = R::PW;
    constexpr int MD = M > 0 ? M : 1;
    static_assert(!COMP || S <= S_FP32_MAX, "compensated form: S <= 11");
    static_assert(sizeof(DevState) % 8 == 0, "state copies move 8-byte words");
    extern __shared__ __align__(128) unsigned char smem[];
    double *ws = reinterpret_cast<double *>(smem + R::OFF_WS);
    double *stat = ws + R::D_STAT, *Sg = ws + R::D_SG, *G = ws + R::D_G, *A = ws + R::D_A, *B = ws + R::D_B;
    double *Wn = ws + R::D_WN, *Lw = ws + R::D_LW, *L0s = ws + R::D_L0S;
    double *sv = ws + R::D_SV, *dv = ws + R::D_DV, *ko = ws + R::D_KO, *kn = ws + R::D_KN, *av = ws + R::D_AV;
    double *gv = ws + R::D_GV, *rd = ws + R::D_RD, *piv = ws + R::D_PIV, *K0s = ws + R::D_K0S;
    double *col = ws + R::D_COL, *red = ws + R::D_RED, *s_red = ws + R::D_SRED, *ltab = ws + R::D_LOG;
    double *rb = ws + R::D_RB;
    double *Cw = ws + R::D_CW, *Qc = ws + R::D_QC, *Sl = ws + R::D_SL, *cd = ws + R::D_CD, *Tw = ws + R::D_TW;
    double *Lf = ws + R::D_LF;
    ElboIn *EI = reinterpret_cast<ElboIn *>(smem + R::OFF_EI);
    SweepGlobalsF32 *sg = reinterpret_cast<SweepGlobalsF32 *>(smem + R::OFF_SG);
    float4 *tab = reinterpret_cast<float4 *>(smem + R::OFF_TAB);
    float *split = reinterpret_cast<float *>(smem + R::OFF_SPLIT);
    float *rs = reinterpret_cast<float *>(smem + R::OFF_SLICE);
    __shared__ int s_n, s_stop, s_timeout;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool elbo_warp = warp == PW;
    const int nblk = gridDim.x;
    const long long v0 = (long long)blockIdx.x * a.per_block;
    const long long rem = a.V - v0;
    const int n = int(rem < a.per_block ? (rem > 0 ? rem : 0) : a.per_block);
    float *ds = rs + ((n + 3) & ~3);

    // ---- prologue: private state copy (blocks 1 ..), slice, tables, pass factors of the first sweep
    DevState *st = a.st;
    if (blockIdx.x != 0) {
        st = a.priv + (blockIdx.x - 1);
        const unsigned long long *src = reinterpret_cast<const unsigned long long *>(a.st);
        unsigned long long *dst = reinterpret_cast<unsigned long long *>(st);
        for (int i = tid; i < int(sizeof(DevState) / 8); i += THREADS) dst[i] = src[i];
    }
    for (int i = tid; i < n; i += THREADS) rs[i] = __ldg(a.r + v0 + i);
    for (long long i = tid; i < (long long)n * S; i += THREADS) ds[i] = __ldg(a.d + v0 * S + i);
    log_tang_table(ltab, tid, THREADS);
    cta_sync();
    if (elbo_warp) {
        if (blockIdx.x != 0 && lane == 0) st->trace = nullptr;   // block 0 alone writes the trace
        __syncwarp();
        {
            const float *src = reinterpret_cast<const float *>(&st->sw);
            float *dst = reinterpret_cast<float *>(sg);
            for (int i = lane; i < int(sizeof(SweepGlobalsF32) / 4); i += 32) dst[i] = src[i];
        }
        for (int e = lane; e < M * M; e += 32) L0s[e] = st->L0inv[e];
        for (int i = lane; i < M; i += 32) K0s[i] = st->K0[i];
        if (lane == 0) {
            const bool go = st->status == ST_OK && !st->converged;
            const int lim = st->target < st->max_iter ? st->target : st->max_iter;
            s_n = (go && lim > st->iter) ? lim - st->iter : 0;
            s_stop = 0;
            s_timeout = 0;
        }
        __syncwarp();
    }
    cta_sync();
    const int nsw = s_n, it0 = st->iter;
    const FitConst fc = fit_const(st);
    double ldw = st->carry_ldw;                  // ELBO warp, lane 0
    ElboOut eo{0.0, 0.0, 0, 1};
    const bool em = fc.em;
    const double V = fc.V, q0 = st->q0;
    const double inv_V = st->kc_upd.inv_V, inv_lam = st->kc_upd.inv_lam, lam = fc.lam;
    const double rs_nu = st->kc_upd.rs_nu;
    if (elbo_warp) {
        if constexpr (R::COEF) {
            resident_pre_small_1<M>(sg, Lf, ko, av, K0s, lane, 32);
            __syncwarp();
            resident_pre_small_2<M>(Lf, Sg, lane, 32);
            __syncwarp();
            resident_pre_small_3<M>(Sg, av, L0s, Cw, Qc, Sl, cd, em, V, q0, inv_lam, inv_V, lane, 32);
        } else {
            resident_pre_mat<M>(sg, Sg, ko, av, K0s, lane, 32);
        }
        resident_pre_logs<M>(fc, sg, ltab, st->carry_ok ? st->carry_piv : nullptr, ldw, &EI[0], lane);
    }
    double elbo_prev = st->elbo_prev;            // ELBO warp, lane 0
    int status = st->status;
    cta_sync();                                  // every read of the state above precedes the first write

    int k = 0;
    for (; k < nsw; ++k) {
        unsigned long long *part = reinterpret_cast<unsigned long long *>(a.partials) + size_t(k & 1) * size_t(nblk) * NS;
        const unsigned long long tag = (unsigned long long)((k + 1) & 3);
        if (!elbo_warp) {
            // ---- steps (a)-(c) of sweep k over the slice
            float A_[COMP ? 1 : C::NGA], B_[COMP ? 1 : C::MA];
            const float erho = sg->erho;
            if constexpr (COMP) {
                for (int i = tid; i < C::SPLIT_FLOATS; i += PT) {
                    float v;
                    if (i < NG) v = sg->Sh[i];
                    else if (i < 2 * NG) v = sg->Sl[i - NG];
                    else if (i < 2 * NG + M) v = sg->kh[i - 2 * NG];
                    else v = sg->kl[i - 2 * NG - M];
                    split[i] = v;
                }
                A_[0] = 0.0f;
                B_[0] = 0.0f;
                pass_sync(PT);
                build_profile_table<S>(tab, split, erho, tid, PT);
                pass_sync(PT);
            } else {
#pragma unroll
                for (int i = 0; i < NG; ++i) A_[i] = sg->L[i];
#pragma unroll
                for (int i = 0; i < M; ++i) B_[i] = sg->kappa[i];
                if constexpr (NG == 0) A_[0] = 0.0f;
                if constexpr (M == 0) B_[0] = 0.0f;
            }
            float acc[NSTAT];
            double acc64[NGR];
            float prod = 1.0f, pl = 0.0f, uh = 0.0f, ul = 0.0f;
            int ex = 0;
#pragma unroll
            for (int i = 0; i < NSTAT; ++i) acc[i] = 0.0f;
#pragma unroll
            for (int g = 0; g < NGR; ++g) acc64[g] = 0.0;
            // rounds of PT observations; the round count is the same for every
            // pass thread, so the warp-wide flushes are reached by whole warps
            int cnt = 0;
            bool flushed = false;                         // acc64 still zero: the first flush assigns
            for (int j0 = 0; j0 < n; j0 += PT) {
                const int j = j0 + tid;
                if (j < n) {
                    float x[S];
                    load_row<S>(ds, j, x);
                    if constexpr (COMP) {
                        observe_comp<S>(x, rs[j], tab, split, erho, acc, prod, pl, uh, ul);
                        peel_exponent2(prod, pl, ex);
                    } else {
                        observe<S>(x, rs[j], A_, B_, erho, acc, prod);
                        peel_exponent(prod, ex);
                    }
                }
                if (++cnt == R::FLUSH) {
                    if constexpr (COMP)
                        flush_warp_comp<S, true, true>(acc, acc64, prod, pl, ex, uh, ul, lane);
                    else
                        flush_warp<S, true, true>(acc, acc64, prod, ex, lane);
                    cnt = 0;
                    flushed = true;
                }
            }
            if (flushed) {
                if constexpr (COMP)
                    flush_warp_comp<S, true, true>(acc, acc64, prod, pl, ex, uh, ul, lane);
                else
                    flush_warp<S, true, true>(acc, acc64, prod, ex, lane);
            } else {
                if constexpr (COMP)
                    flush_warp_comp<S, false, true>(acc, acc64, prod, pl, ex, uh, ul, lane);
                else
                    flush_warp<S, false, true>(acc, acc64, prod, ex, lane);
            }
            // block reduction in FP64 (fixed order: a tree over the pass warps), this
            // block's row of tagged values
#pragma unroll
            for (int g = 0; g < NGR; ++g) s_red[warp * (NGR * 32) + g * 32 + lane] = acc64[g];
            pass_sync(PT);
            if (warp == 0) {
                for (int j = lane; j < NS; j += 32) {
                    double w[PW];
#pragma unroll
                    for (int i = 0; i < PW; ++i) w[i] = s_red[i * (NGR * 32) + j];
#pragma unroll
                    for (int h = 1; h < PW; h *= 2)
#pragma unroll
                        for (int i = 0; i + h < PW; i += 2 * h) w[i] += w[i + h];
                    const unsigned long long bits =
                        (static_cast<unsigned long long>(__double_as_longlong(w[0])) & ~3ull) | tag;
                    st_relaxed_u64(part + size_t(blockIdx.x) * NS + j, bits);
                }
            }
            // the FP64 forms of this sweep's pass factors for its matrix chain (the
            // previous chain is done; sweep 0 took them in the prologue)
            // (items dealt round robin over the pass warps, which sit on different SM
            // sub-partitions: each FP64 instruction holds one for ~64 cycles)
            if (k > 0) {
                const int tw = warp + PW * lane;
                if constexpr (R::COEF) {
                    // (between the block's row and the wait for the other rows: off the path
                    // that sets the sweep, which runs through the last row to arrive)
                    resident_pre_small_12<M>(sg, Lf, Sg, ko, av, K0s, warp, lane, PT);
                } else {
                    resident_pre_mat<M>(sg, Sg, ko, av, K0s, tw, PT);
                }
            }
        } else if (k > 0) {
            // ---- ELBO warp: the ELBO and stopping test of sweep k - 1
            const bool stop = resident_elbo_decide<M>(fc, EI[(k - 1) & 1], kn, ltab, elbo_prev, status, eo, lane);
            if (lane == 0) s_stop = stop ? 1 : 0;
        }
        cta_sync();
        if (elbo_warp && k > 0) {
            // ---- ELBO warp, while the rows are exchanged: the state after sweep k - 1, then
            //      the logarithms of the pass factors sweep k read
            resident_elbo_store<M>(st, fc, EI[(k - 1) & 1], Wn, kn, sg, it0 + k, eo, elbo_prev, status, ldw, lane);
            if (!s_stop) {
                resident_pre_logs<M>(fc, sg, ltab, EI[(k - 1) & 1].piv, ldw, &EI[k & 1], lane);
                if constexpr (R::COEF)
                    resident_pre_small_3<M>(Sg, av, L0s, Cw, Qc, Sl, cd, em, V, q0, inv_lam, inv_V, lane, 32);
            }
        }
        if (s_stop) break;                  // sweep k - 1 ended the fit: sweep k's pass is dropped

        // ---- every block's row of sweep k (pass warps): value (row, column) is ready
        //      when its two low bits carry the tag of sweep k.  Item (g, j) is column j
        //      of rows 4g .. 4g + 3; its owner polls them and, once all are in, takes
        //      their sum (the first level of a 4-ary tree over the rows)
        if (!elbo_warp) {
            const int ngrp = (nblk + 3) / 4, nitem = NS * ngrp;
            uint32_t pending = 0;                        // bit 4i + u: row 4g + u of item i outstanding
#pragma unroll
            for (int i = 0; i < R::IPT; ++i) {
                const int q = tid + i * PT;
                if (q < nitem) {
                    const int g = q / NS, cnt = (nblk - 4 * g < 4) ? nblk - 4 * g : 4;
                    pending |= ((1u << cnt) - 1u) << (4 * i);
                }
            }
            const uint64_t t0 = global_ns();
            for (uint32_t round = 0; pending; ++round) {
#pragma unroll
                for (int i0 = 0; i0 < R::IPT; i0 += 2) {
                    unsigned long long gv4[2][4];
#pragma unroll
                    for (int i = i0; i < i0 + 2 && i < R::IPT; ++i) {
                        const int q = tid + i * PT, g = q / NS, jj = q - g * NS;
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if ((pending >> (4 * i + u)) & 1u) gv4[i - i0][u] = ld_relaxed_u64(part + (4 * g + u) * NS + jj);
                    }
#pragma unroll
                    for (int i = i0; i < i0 + 2 && i < R::IPT; ++i) {
                        if (!((pending >> (4 * i)) & 15u)) continue;
                        const int q = tid + i * PT, g = q / NS, jj = q - g * NS;
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (((pending >> (4 * i + u)) & 1u) && (gv4[i - i0][u] & 3ull) == tag) {
                                rb[(4 * g + u) * NS + jj] =
                                    __longlong_as_double(static_cast<long long>(gv4[i - i0][u] & ~3ull));
                                pending &= ~(1u << (4 * i + u));
                            }
                        if (!((pending >> (4 * i)) & 15u)) {
                            const int cnt = (nblk - 4 * g < 4) ? nblk - 4 * g : 4;
                            const double *x = rb + 4 * g * NS + jj;
                            // missing rows of the last group as zeros (x + 0 = x)
                            const double x0 = x[0], x1 = cnt > 1 ? x[NS] : 0.0, x2 = cnt > 2 ? x[2 * NS] : 0.0,
                                         x3 = cnt > 3 ? x[3 * NS] : 0.0;
                            red[g * NS + jj] = (x0 + x1) + (x2 + x3);
                        }
                    }
                }
                if (pending && (round & 15u) == 15u && global_ns() - t0 > RESIDENT_WAIT_NS) {
                    s_timeout = 1;
                    break;
                }
            }
            pass_sync(PT);
            if (!s_timeout) {
                // the rest of the tree, level by level (rows 4g .. 4g + 3 -> row g, as
                // (a + b) + (c + d)), between red and rb: on this GPU each FP64 warp
                // instruction holds its SM sub-partition for ~64 cycles, so the levels
                // pack one addition per lane over few warps
                const double *src = red;
                double *dst = rb;
                int n = ngrp;
                while (n > 1) {
                    const int n4 = (n + 3) / 4;
                    for (int q = tid; q < NS * n4; q += PT) {
                        const int g = q / NS, jj = q - g * NS;
                        const int b = 4 * g, cnt = (n - b < 4) ? n - b : 4;
                        const double *x = src + b * NS + jj;
                        const double x0 = x[0], x1 = cnt > 1 ? x[NS] : 0.0, x2 = cnt > 2 ? x[2 * NS] : 0.0,
                                     x3 = cnt > 3 ? x[3 * NS] : 0.0;
                        dst[g * NS + jj] = (x0 + x1) + (x2 + x3);
                    }
                    pass_sync(PT);
                    const double *t = src;
                    src = dst;
                    dst = const_cast<double *>(t);
                    n = n4;
                }
                for (int j = tid; j < NS; j += PT) {
                    const double v = src[j];
                    stat[j] = v;
                    if (j < NG) {
                        int r = static_cast<int>((sqrtf(8.0f * j + 1.0f) - 1.0f) * 0.5f);
                        while (r * (r + 1) / 2 > j) --r;
                        while ((r + 1) * (r + 2) / 2 <= j) ++r;
                        const int cc = j - r * (r + 1) / 2;
                        G[r * M + cc] = v;
                        G[cc * M + r] = v;
                    } else if (j < NG + M) {
                        gv[j - NG] = v;
                    }
                }
            }
        }
        cta_sync();
        if (s_timeout) {
            if (tid == 0) atomicCAS(&a.st->status, ST_OK, ST_ETIMEOUT);
            break;
        }

        // ---- step (d) of sweep k: the matrix chain (pass warps) and E[rho] (ELBO warp)
        if (elbo_warp) {
            if (lane == 0) resident_rho<M>(fc, stat, C::I_U, sg, &EI[k & 1]);
            if ((em || fc.comp) && M > 0) {
                double t1 = 0.0;
                for (int e = lane; e < M * M; e += 32) t1 = fma(Sg[e], G[e], t1);
                const double t = lane_sum<(M * M < 32) ? M * M : 32>(t1);
                if (lane == 0) EI[k & 1].trSG = t;
            } else if (lane == 0) {
                EI[k & 1].trSG = 0.0;
            }
        } else {
            if constexpr (R::COEF) {
                // delta and kappa' (warp 0), W'^{-1} before its delta term (warp 1:
                // another SM sub-partition), then the delta term (warp 0)
                const double *Gp = stat, *gs = stat + NG;        // packed G, g
                if (warp == 0 && lane < M) {
                    double d = cd[lane];
#pragma unroll
                    for (int kk = 0; kk < M; ++kk) d = fma(Sl[lane * M + kk], gs[kk], d);
                    dv[lane] = d;
                    kn[lane] = ko[lane] + d;
                } else if (warp == 1 && lane < NG) {
                    double t = Cw[lane];
#pragma unroll
                    for (int pk = 0; pk < NG; ++pk) t = fma(Qc[lane * C::NGA + pk], Gp[pk], t);
                    Tw[lane] = t;
                }
                pass_sync(PT);
                if (warp == 0 && lane < NG) {
                    int r, c;
                    packed_rc(lane, r, c);
                    const double w = fma(-(em ? dv[r] : lam * dv[r]), dv[c], Tw[lane]);
                    Wn[r * M + c] = w;
                    Wn[c * M + r] = w;
                }
                pass_sync(PT);
            } else {
                // A = Sigma0~ G, s = Sigma0~ g
                for (int e = tid; e < M * M; e += PT) {
                    const int r = e / MD, c = e - r * MD;
                    double s0 = 0.0, s1 = 0.0;
                    int kk = 0;
                    for (; kk + 1 < M; kk += 2) {
                        s0 = fma(Sg[r * M + kk], G[kk * M + c], s0);
                        s1 = fma(Sg[r * M + kk + 1], G[(kk + 1) * M + c], s1);
                    }
                    if (kk < M) s0 = fma(Sg[r * M + kk], G[kk * M + c], s0);
                    A[e] = s0 + s1;
                }
                for (int i = tid; i < M; i += PT) {
                    double s0 = 0.0, s1 = 0.0;
                    int kk = 0;
                    for (; kk + 1 < M; kk += 2) {
                        s0 = fma(Sg[i * M + kk], gv[kk], s0);
                        s1 = fma(Sg[i * M + kk + 1], gv[kk + 1], s1);
                    }
                    if (kk < M) s0 = fma(Sg[i * M + kk], gv[kk], s0);
                    sv[i] = s0 + s1;
                }
                pass_sync(PT);
                // B = Sigma0~ G Sigma0~, delta, kappa'
                for (int e = tid; e < M * M; e += PT) {
                    const int r = e / MD, c = e - r * MD;
                    double s0 = 0.0, s1 = 0.0;
                    int kk = 0;
                    for (; kk + 1 < M; kk += 2) {
                        s0 = fma(A[r * M + kk], Sg[kk * M + c], s0);
                        s1 = fma(A[r * M + kk + 1], Sg[(kk + 1) * M + c], s1);
                    }
                    if (kk < M) s0 = fma(A[r * M + kk], Sg[kk * M + c], s0);
                    B[e] = s0 + s1;
                }
                for (int i = tid; i < M; i += PT) {
                    if (em)
                        dv[i] = sv[i] * inv_V;                       // Eq. 46
                    else
                        dv[i] = fma(q0, av[i], sv[i]) * inv_lam;     // Eq. 24, centred on kappa~
                    kn[i] = ko[i] + dv[i];
                }
                pass_sync(PT);
                // W'^{-1} (Eq. 25, centred; EM: Eq. 47)
                for (int e = tid; e < M * M; e += PT) {
                    const int r = e / MD, c = e - r * MD;
                    const double Bs = 0.5 * (B[r * M + c] + B[c * M + r]);
                    if (em)
                        Wn[e] = fma(Bs, inv_V, Sg[e]) - dv[r] * dv[c];
                    else
                        Wn[e] = L0s[e] + V * Sg[e] + Bs + q0 * av[r] * av[c] - lam * dv[r] * dv[c];
                }
                pass_sync(PT);
            }
            // its Cholesky factor (warp 0) -> the FP32 pass factors of sweep k + 1
            if (warp == 0) {
                const int fail = warp_cholesky_rt(M, Wn, Lw, rd, piv, col, lane);
                const double rs = em ? 1.0 : rs_nu;
                for (int e = lane; e < M * M; e += 32) {
                    const int r = e / MD, c = e - r * MD;
                    if (c <= r) sg->L[r * (r + 1) / 2 + c] = static_cast<float>(Lw[e] * rs);
                }
                for (int i = lane; i < M; i += 32) EI[k & 1].piv[i] = piv[i];
                if (lane == 0) EI[k & 1].fail = fail;
                __syncwarp();
                if (COMP) write_pass_splits_sigma_rt(M, sg, lane);
            } else if (warp == 1) {
                // kappa~ and its split, beside the factorisation
                for (int i = lane; i < M; i += 32) sg->kappa[i] = static_cast<float>(kn[i]);
                __syncwarp();
                if (COMP) write_pass_splits_kappa_rt(M, sg, lane);
            }
        }
        cta_sync();
    }
    // the ELBO, stopping test and state of the last sweep whose update ran
    if (elbo_warp && k == nsw && nsw > 0) {
        (void)resident_elbo_decide<M>(fc, EI[(nsw - 1) & 1], kn, ltab, elbo_prev, status, eo, lane);
        resident_elbo_store<M>(st, fc, EI[(nsw - 1) & 1], Wn, kn, sg, it0 + nsw, eo, elbo_prev, status, ldw, lane);
    }
}

} // namespace vbh
