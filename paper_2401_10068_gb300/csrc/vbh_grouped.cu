// vbh_grouped.cu -- the exact profile-grouped form of the sweep for binary
// profiles (d_ij in {0, 1}).
//
// Within a group of observations that share a profile, D_i, q_i, t_i, c_i and
// ln(1 + E[rho] q_i) are the same, and every sum the sweep needs is a
// polynomial of degree <= 2 in e_i = y_i - t: with n, sum y and sum y^2 of the
// group,  sum e = sum y - n t,  sum e^2 = sum y^2 - 2 t sum y + n t^2,
//   sum w D = c (sum e) D,  sum (w^2 - c) D D^T = (c^2 sum e^2 - n c) D D^T,
//   sum S_i = inv^2 sum e^2 + n q inv,  sum ln(1 + E[rho] q) = n ln(1 + E[rho] q),
// with c = E[rho] inv and inv = 1 / (1 + E[rho] q) (Eq. 19-21 in the rank-1
// form of the per-observation sweep).  One histogram pass over the data gives
// (n, sum y, sum y^2) per profile code; after it each sweep costs
// O(2^S M^2), independent of V.  The sweep uses the FP32 globals of the pass
// (as the per-observation sweep does) with FP64 arithmetic, writes the same
// per-block partials and ends in the same global update.
#include <cuda_runtime.h>

#include "vbh.h"
#include "vbh_error.h"
#include "vbh_grouped_host.h"
#include "vbh_sweep.cuh"

namespace vbh {

namespace {
constexpr int GW = GROUPED_THREADS / 32;                        // warps per block
constexpr int GMAX = GROUPED_SMAX - 1;                          // largest M
constexpr int GNSTAT = GMAX * (GMAX + 1) / 2 + GMAX + 3;
} // namespace

__global__ void grouped_hist_kernel(const float *__restrict__ r, const float *__restrict__ d, long long V, int S,
                                    double *__restrict__ stats, unsigned long long *nonbinary)
{
    extern __shared__ double sh[];
    const int P = 1 << S;
    const bool local = P <= 2048;                               // 48 KiB of block histogram
    if (local) {
        for (int i = threadIdx.x; i < 3 * P; i += blockDim.x) sh[i] = 0.0;
        __syncthreads();
    }
    unsigned long long bad = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += stride) {
        const float *di = d + i * S;
        int code = 0;
        for (int j = 0; j < S; ++j) {
            const float x = di[j];
            if (x == 1.0f) code |= 1 << j;
            else if (x != 0.0f) ++bad;
        }
        const double y = static_cast<double>(r[i]) - static_cast<double>(di[S - 1]);
        double *dst = local ? sh + 3 * code : stats + 3 * code;
        atomicAdd(dst, 1.0);
        atomicAdd(dst + 1, y);
        atomicAdd(dst + 2, y * y);
    }
    if (local) {
        __syncthreads();
        for (int i = threadIdx.x; i < 3 * P; i += blockDim.x)
            if (sh[i] != 0.0) atomicAdd(stats + i, sh[i]);
    }
    if (bad) atomicAdd(nonbinary, bad);
}

// The per-code work of the sweep below for M <= GM (loops of GM terms): warp
// w of the grid takes codes w, w + W, ...; lane j < M keeps row j of the
// packed G (columns k <= j) and g_j; D_k = d_k - d_S in {-1, 0, 1} by
// selection (no conversions).
template <int GM>
__device__ __forceinline__ void grouped_codes(const GroupArgs &ga, const DevState *st, int lane, int warp,
                                              double (&gacc)[GMAX], double &gv, double &t3, double &t4)
{
    const int M = st->S - 1;
    // column `lane` of L~ and kappa~ of the pass (FP32 globals, as the per-observation sweep)
    double lcol[GM > 0 ? GM : 1];
#pragma unroll
    for (int k = 0; k < GM; ++k)
        lcol[k] = (lane < M && k < M && k >= lane) ? static_cast<double>(st->sw.L[k * (k + 1) / 2 + lane]) : 0.0;
    const double kap = lane < M ? static_cast<double>(st->sw.kappa[lane]) : 0.0;
    const double erho = static_cast<double>(st->sw.erho);
    const int nwarps = gridDim.x * GW;
    for (int p = blockIdx.x * GW + warp; p < ga.P; p += nwarps) {
        const double n = ga.stats[3 * p];
        if (n == 0.0) continue;                                 // warp-uniform
        const double sy = ga.stats[3 * p + 1], syy = ga.stats[3 * p + 2];
        const int bS = (p >> M) & 1;
        auto Dk = [&](int k) -> double {
            const int b = (p >> k) & 1;
            return b == bS ? 0.0 : (b ? 1.0 : -1.0);
        };
        double v = 0.0;
#pragma unroll
        for (int k = 0; k < GM; ++k) v = fma(lcol[k], (k < M) ? Dk(k) : 0.0, v);   // (L~^T D)_lane
        const double Dj = lane < M ? Dk(lane) : 0.0;
        const double q = warp_sum(v * v);
        const double t = warp_sum(kap * Dj);
        const double den = fma(erho, q, 1.0);
        const double inv = 1.0 / den;
        const double c = erho * inv;
        const double se = sy - n * t;
        const double see = syy - 2.0 * t * sy + n * t * t;
        const double sw = c * se;
        const double sgam = c * c * see - n * c;
        if (lane < M) {
            const double sd = sgam * Dj;
#pragma unroll
            for (int k = 0; k < GM; ++k)
                if (k <= lane) gacc[k] = fma(sd, Dk(k), gacc[k]);
            gv = fma(sw, Dj, gv);
        }
        if (lane == 0) {
            t3 += inv * inv * see + n * q * inv;
            t4 += n * log(den);
        }
    }
}

// One sweep over the profile groups: warp w of the grid takes codes w, w + W, ...;
// lane j < M keeps row j of the packed G (columns k <= j) and g_j in registers.
__global__ void __launch_bounds__(GROUPED_THREADS) grouped_sweep_kernel(GroupArgs ga)
{
    extern __shared__ double gsm[];
    __shared__ int s_last;
    const SweepArgs &a = ga.sa;
    DevState *st = a.st;
    const int S = st->S, M = S - 1;
    const int NG = M * (M + 1) / 2, NSTAT = NG + M + 3;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool run = (a.mode != MODE_ITER) ||
                     (st->status == ST_OK && !st->converged && st->iter < st->target && st->iter < st->max_iter);

    double gacc[GMAX], gv = 0.0, t3 = 0.0, t4 = 0.0;
#pragma unroll
    for (int k = 0; k < GMAX; ++k) gacc[k] = 0.0;
    if (run) {
        switch (M) {                                            // loops of exactly M terms
        case 0: grouped_codes<0>(ga, st, lane, warp, gacc, gv, t3, t4); break;
        case 1: grouped_codes<1>(ga, st, lane, warp, gacc, gv, t3, t4); break;
        case 2: grouped_codes<2>(ga, st, lane, warp, gacc, gv, t3, t4); break;
        case 3: grouped_codes<3>(ga, st, lane, warp, gacc, gv, t3, t4); break;
        case 4: grouped_codes<4>(ga, st, lane, warp, gacc, gv, t3, t4); break;
        case 5: grouped_codes<5>(ga, st, lane, warp, gacc, gv, t3, t4); break;
        case 6: grouped_codes<6>(ga, st, lane, warp, gacc, gv, t3, t4); break;
        case 7: grouped_codes<7>(ga, st, lane, warp, gacc, gv, t3, t4); break;
        case 8: grouped_codes<8>(ga, st, lane, warp, gacc, gv, t3, t4); break;
        case 9: grouped_codes<9>(ga, st, lane, warp, gacc, gv, t3, t4); break;
        case 10: grouped_codes<10>(ga, st, lane, warp, gacc, gv, t3, t4); break;
        default: grouped_codes<GMAX>(ga, st, lane, warp, gacc, gv, t3, t4); break;
        }
    }
    // per-warp partials -> shared memory [warp][NSTAT] -> this block's partials (fixed order)
    double *red = gsm;
    if (lane < M) {
#pragma unroll
        for (int k = 0; k < GMAX; ++k)
            if (k <= lane) red[warp * GNSTAT + lane * (lane + 1) / 2 + k] = gacc[k];
        red[warp * GNSTAT + NG + lane] = gv;
    }
    if (lane == 0) {
        red[warp * GNSTAT + NG + M] = t3;
        red[warp * GNSTAT + NG + M + 1] = t4;
        red[warp * GNSTAT + NG + M + 2] = 0.0;
    }
    __syncthreads();
    double *part = a.partials + size_t(blockIdx.x) * NSTAT;
    for (int j = tid; j < NSTAT; j += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < GW; ++w) s += red[w * GNSTAT + j];
        part[j] = s;
    }
    int row0, nrows;
    if (!finish_ticket(st, a.partials, gridDim.x, NSTAT, &s_last, &row0, &nrows, gsm)) return;
    if (run && st->status == ST_OK) {
        global_update_rt(M, st, a.partials + size_t(row0) * NSTAT, nrows, a, gsm);
    } else if (tid == 0 && a.use_cond) {
        cudaGraphSetConditional(a.cond, 0u);
    }
}

// The same sweep for many profile codes (S >= GROUPED_WIDE_S): lane = code.
// Warp w of the grid takes batches of 32 consecutive codes w, w + W, ...; in a
// batch the low LB = 5 bits of the code (lane) vary and the others, d_S
// included, are the warp's.  So with D_k = d_k - d_S in {-1, 0, 1}:
//   v = L~^T D: the part over k >= LB is the same for the whole batch (lane j
//     forms h_j = sum_{k >= max(j, LB)} L~(k, j) D_k once), the rest is LB
//     terms per lane;  q = |v|^2,  t = kappa~^T D likewise;
//   G = sum gamma D D^T and g = sum w D over the batch: entries (r, c) with
//     r >= LB take D_r (D_c sum gamma or sum gamma D_c) from seven warp sums;
//     the 15 entries with r < LB and g_{j < LB} are accumulated per lane and
//     summed over the warp once at the end.
// About half the FP64 instructions of forming every code's v and adding every
// code into every G entry.
namespace {
constexpr int GNG = GMAX * (GMAX + 1) / 2;                       // packed entries of G at the largest M
constexpr int LB = 5;                                            // code bits that vary within a batch
constexpr int NLL = LB * (LB + 1) / 2;                           // G entries with r < LB (first in the packed order)
constexpr int WIDE_GPL = (GNG - NLL + 31) / 32;                  // entries with r >= LB per lane
constexpr size_t WIDE_PASS_DOUBLES = GNG + 16;                   // L~, kappa~
} // namespace

__global__ void __launch_bounds__(GROUPED_THREADS) grouped_sweep_wide_kernel(GroupArgs ga)
{
    extern __shared__ double gsm[];
    __shared__ int s_last;
    const SweepArgs &a = ga.sa;
    DevState *st = a.st;
    const int S = st->S, M = S - 1;                              // M >= GROUPED_WIDE_S - 1 > LB
    const int NG = M * (M + 1) / 2, NSTAT = NG + M + 3;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool run = (a.mode != MODE_ITER) ||
                     (st->status == ST_OK && !st->converged && st->iter < st->target && st->iter < st->max_iter);

    double *Lf = gsm;                                            // L~ (packed lower, row i at i(i+1)/2), FP64
    double *kf = Lf + GNG;                                       // kappa~
    double *red = gsm + WIDE_PASS_DOUBLES;                       // [warp][NSTAT] partials

    double hacc[WIDE_GPL], llacc[NLL], glow[LB], ghigh = 0.0, t3 = 0.0, t4 = 0.0;
#pragma unroll
    for (int i = 0; i < WIDE_GPL; ++i) hacc[i] = 0.0;
#pragma unroll
    for (int i = 0; i < NLL; ++i) llacc[i] = 0.0;
#pragma unroll
    for (int i = 0; i < LB; ++i) glow[i] = 0.0;
    int er[WIDE_GPL], ec[WIDE_GPL];                              // this lane's entries with r >= LB
#pragma unroll
    for (int i = 0; i < WIDE_GPL; ++i) {
        const int e = NLL + lane + 32 * i;
        int r = 0;
        while ((r + 1) * (r + 2) / 2 <= e) ++r;
        er[i] = (e < NG) ? r : -1;
        ec[i] = e - r * (r + 1) / 2;
    }
    if (run) {
        for (int e = tid; e < NG; e += blockDim.x) Lf[e] = static_cast<double>(st->sw.L[e]);
        for (int i = tid; i < M; i += blockDim.x) kf[i] = static_cast<double>(st->sw.kappa[i]);
        __syncthreads();
        const double erho = static_cast<double>(st->sw.erho);
        const int nbatch = (ga.P + 31) / 32, nw = gridDim.x * GW;
        for (int bt = blockIdx.x * GW + warp; bt < nbatch; bt += nw) {
            const int base = bt * 32, p = base + lane;
            const int bS = (base >> M) & 1;
            auto Dh = [&](int k) -> double {                     // D_k, k >= LB: the batch's
                const int b = (base >> k) & 1;
                return b == bS ? 0.0 : (b ? 1.0 : -1.0);
            };
            auto Dl = [&](int k) -> double {                     // D_k, k < LB: this lane's
                const int b = (lane >> k) & 1;
                return b == bS ? 0.0 : (b ? 1.0 : -1.0);
            };
            // the batch's parts: h_j (lane j), sum_{j >= LB} h_j^2 and sum_{k >= LB} kappa_k D_k
            double hj = 0.0;
            if (lane < M)
                for (int k = (lane > LB ? lane : LB); k < M; ++k) {
                    const double dk = Dh(k);
                    if (dk != 0.0) hj = fma(Lf[k * (k + 1) / 2 + lane], dk, hj);
                }
            const double qh = warp_sum((lane >= LB && lane < M) ? hj * hj : 0.0);
            const double th = warp_sum((lane >= LB && lane < M) ? kf[lane] * Dh(lane) : 0.0);
            // this lane's code: the low parts
            double q = qh, t = th;
#pragma unroll
            for (int j = 0; j < LB; ++j) {
                double v = __shfl_sync(0xffffffffu, hj, j);
#pragma unroll
                for (int k = j; k < LB; ++k) {
                    const double dk = Dl(k);
                    if (dk != 0.0) v = fma(Lf[k * (k + 1) / 2 + j], dk, v);
                }
                q = fma(v, v, q);
                const double dj = Dl(j);
                if (dj != 0.0) t = fma(kf[j], dj, t);
            }
            const bool valid = p < ga.P;
            const double n = valid ? ga.stats[3 * p] : 0.0;
            const double sy = valid ? ga.stats[3 * p + 1] : 0.0, syy = valid ? ga.stats[3 * p + 2] : 0.0;
            const double den = fma(erho, q, 1.0);
            const double inv = 1.0 / den;
            const double c = erho * inv;
            const double se = sy - n * t;
            const double see = syy - 2.0 * t * sy + n * t * t;
            t3 += inv * inv * see + n * q * inv;
            t4 += n * log(den);
            const double sg = c * c * see - n * c, sw = c * se;
            // the batch's sums for the entries with r >= LB and for g_{j >= LB}
            const double S0 = warp_sum(sg), W0 = warp_sum(sw);
            auto sgd = [&](int k) {                               // sum over the batch of gamma D_k, k < LB
                const double dk = Dl(k);
                return warp_sum(dk == 0.0 ? 0.0 : (dk > 0.0 ? sg : -sg));
            };
            const double Sc0 = sgd(0), Sc1 = sgd(1), Sc2 = sgd(2), Sc3 = sgd(3), Sc4 = sgd(4);
            static_assert(LB == 5, "five low bits");
#pragma unroll
            for (int i = 0; i < WIDE_GPL; ++i)
                if (er[i] >= 0) {
                    const double dr = Dh(er[i]);
                    if (dr != 0.0) {
                        double x;
                        if (ec[i] >= LB) {
                            const double dc = Dh(ec[i]);
                            x = dc * S0;
                        } else {
                            const int k = ec[i];
                            x = k == 0 ? Sc0 : k == 1 ? Sc1 : k == 2 ? Sc2 : k == 3 ? Sc3 : Sc4;
                        }
                        hacc[i] = fma(dr, x, hacc[i]);
                    }
                }
            if (lane >= LB && lane < M) {
                const double dj = Dh(lane);
                if (dj != 0.0) ghigh = fma(dj, W0, ghigh);
            }
            // this lane's code into the entries with r < LB and g_{j < LB}
#pragma unroll
            for (int r = 0; r < LB; ++r) {
                const double dr = Dl(r);
                if (dr != 0.0) {
                    const double sgr = dr > 0.0 ? sg : -sg;
#pragma unroll
                    for (int cc = 0; cc <= r; ++cc) {
                        const double dc = Dl(cc);
                        if (dc != 0.0) llacc[r * (r + 1) / 2 + cc] += dc > 0.0 ? sgr : -sgr;
                    }
                    glow[r] += dr > 0.0 ? sw : -sw;
                }
            }
        }
    }
    // per-warp partials -> shared memory [warp][NSTAT] -> this block's partials (fixed order)
    const double t3w = warp_sum(t3), t4w = warp_sum(t4);
#pragma unroll
    for (int i = 0; i < NLL; ++i) {
        const double x = warp_sum(llacc[i]);
        if (lane == 0) red[warp * GNSTAT + i] = x;
    }
#pragma unroll
    for (int j = 0; j < LB; ++j) {
        const double x = warp_sum(glow[j]);
        if (lane == 0) red[warp * GNSTAT + NG + j] = x;
    }
#pragma unroll
    for (int i = 0; i < WIDE_GPL; ++i)
        if (er[i] >= 0) red[warp * GNSTAT + NLL + lane + 32 * i] = hacc[i];
    if (lane >= LB && lane < M) red[warp * GNSTAT + NG + lane] = ghigh;
    if (lane == 0) {
        red[warp * GNSTAT + NG + M] = t3w;
        red[warp * GNSTAT + NG + M + 1] = t4w;
        red[warp * GNSTAT + NG + M + 2] = 0.0;
    }
    __syncthreads();
    double *part = a.partials + size_t(blockIdx.x) * NSTAT;
    for (int j = tid; j < NSTAT; j += blockDim.x) {
        double sum = 0.0;
        for (int w = 0; w < GW; ++w) sum += red[w * GNSTAT + j];
        part[j] = sum;
    }
    int row0, nrows;
    if (!finish_ticket(st, a.partials, gridDim.x, NSTAT, &s_last, &row0, &nrows, gsm)) return;
    if (run && st->status == ST_OK) {
        global_update_rt(M, st, a.partials + size_t(row0) * NSTAT, nrows, a, gsm);
    } else if (tid == 0 && a.use_cond) {
        cudaGraphSetConditional(a.cond, 0u);
    }
}

const void *grouped_sweep_func(int S)
{
    return S >= GROUPED_WIDE_S ? reinterpret_cast<const void *>(&grouped_sweep_wide_kernel)
                               : reinterpret_cast<const void *>(&grouped_sweep_kernel);
}

int grouped_grid(int S, int nsm)
{
    const long long P = 1LL << S;
    long long g = (S >= GROUPED_WIDE_S) ? ((P + 31) / 32 + GW - 1) / GW : (P + GW - 1) / GW;   // warps of 32 codes / one code
    const long long cap = (S >= GROUPED_WIDE_S) ? 2LL * nsm : nsm;            // the wide form: two blocks per SM
    if (g > cap) g = cap;
    return int(g < 1 ? 1 : g);
}

size_t grouped_smem_bytes()
{
    const size_t red = size_t(GW) * GNSTAT * sizeof(double);
    const size_t wide = (WIDE_PASS_DOUBLES + size_t(GW) * GNSTAT) * sizeof(double);
    const size_t ws = size_t(gu_ws_doubles_rt(GMAX)) * sizeof(double);
    size_t m = red > ws ? red : ws;
    return m > wide ? m : wide;
}

int grouped_histogram(const float *r, const float *d, long long V, int S, double *stats,
                      unsigned long long *nonbinary_dev, cudaStream_t stream, int nsm)
{
    if (V == 0) return VBH_OK;
    const int P = 1 << S;
    const size_t smem = (P <= 2048) ? size_t(3) * P * sizeof(double) : 0;
    long long blocks = (V + 255) / 256;
    if (blocks > 4LL * nsm) blocks = 4LL * nsm;
    if (smem > 48 * 1024) VBH_CHECK_CUDA(cudaFuncSetAttribute(grouped_hist_kernel,
                                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    grouped_hist_kernel<<<int(blocks), 256, smem, stream>>>(r, d, V, S, stats, nonbinary_dev);
    VBH_CHECK_CUDA(cudaGetLastError());
    return VBH_OK;
}

} // namespace vbh
