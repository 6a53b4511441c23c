// vbh_tc.cuh -- the fused CAVI sweep for 12 <= S <= 32 on the tcgen05 tensor
// cores (one persistent CTA per SM).
//
// Same sweep as vbh_sweep.cuh (steps (a)-(e), Eq. 16-31); the two contractions
// that grow with M^2 run as BF16 MMAs with FP32 accumulation in tensor memory:
//   MMA1  U = d_tile (128 x 32) . B1 (32 x N1): per observation the vector
//         v = L~^T D_i (so q_i = |v|^2) and t_i = kappa~^T D_i.  The profile
//         column d_S is folded into B1 (row S-1 holds minus the column sums),
//         so the MMA reads the raw profiles; L~ and kappa~ (the FP32 globals
//         of the pass) are split into NSPLIT BF16 parts side by side in N.
//         With binary profiles every product is exact: NSPLIT = 3 reproduces
//         the FP32 values (24 bits), NSPLIT = 2 keeps 16 bits (the BF16 form).
//   MMA2  G' = A2 (128 x 128 obs) . d_tile (128 obs x 32): the rows of A2 are
//         gamma_i d_i (hi and lo BF16 parts of gamma_i = w_i^2 - c_i) and w_i
//         (hi, lo), so G' holds sum gamma d d^T and sum w d in the raw-profile
//         basis; G and g of the sweep follow in FP64 by removing the d_S
//         column (G_jk = G'_jk - G'_jS - G'_Sk + G'_SS, g_j = g'_j - g'_S).
//         G' accumulates in FP32 in tensor memory for an epoch of 64 tiles and
//         is then added into FP64 shared memory.
// The scalar per-observation work (c_i, w_i, S_i, ln(1 + E[rho] q_i)) stays
// on the CUDA cores.  The profile tile (BF16, 64-byte rows, 64-byte swizzle)
// arrives by tensor-map TMA and the r tile by a bulk copy (both from copies
// padded to whole tiles); the same profile tile is MMA1's K-major A operand and
// MMA2's MN-major B operand.
//
// Roles: warp 8 lane 0 issues the TMA loads, warp 9 lane 0 issues the MMAs,
// warps 0-7 are two groups of four consumer warps that take alternate tiles
// (double-buffered U in tensor memory and A2 in shared memory); each warp of a
// group owns one quarter of the tensor-memory lanes (32 observations).  Every
// wait is bounded: on a timeout the kernel records VBH_ETIMEOUT, lets its
// copies and MMAs drain, frees its tensor memory and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "vbh_sweep.cuh"
#include "vbh_tc_host.h"

namespace vbh {

template <int NSPLIT>
struct TcCfg {
    static constexpr int TILE = 128;                                   // observations per tile
    static constexpr int N1 = ((33 * NSPLIT + 15) / 16) * 16;          // MMA1 N: 80 or 112
    static constexpr int STAGES = 4;
    static constexpr uint32_t D_BYTES = TILE * 64;
    static constexpr uint32_t R_BYTES = TILE * 4;
    static constexpr uint32_t A2_ATOM = TILE * 128;                    // one 64-row atom column
    static constexpr uint32_t A2_BYTES = 2 * A2_ATOM;
    static constexpr int EPOCH = 16;                                   // tiles per G' epoch
    static constexpr int NCW = 8;
    static constexpr int THREADS = 32 * (NCW + 2);
    static constexpr int TMEM_COLS = 512;
    static constexpr uint32_t COL_U = 0, COL_U_STRIDE = 128;          // U[b] at column 128 b
    static constexpr uint32_t COL_G = 256, COL_G_STRIDE = 32;          // G'[e] at column 256 + 32 e
    // rows of G': part p of gamma d in rows 32 p .. 32 p + 31, part p of w in row 32 NSPLIT + p
    static constexpr int GROWS = 33 * NSPLIT;
    static constexpr int FLUSH_WARPS = (GROWS + 31) / 32;
    static constexpr int GACC_ROWS = 32 * FLUSH_WARPS;
    static constexpr uint32_t OFF_D = 0;
    static constexpr uint32_t OFF_A2 = OFF_D + STAGES * D_BYTES;
    static constexpr uint32_t OFF_B1 = OFF_A2 + 2 * A2_BYTES;
    static constexpr uint32_t OFF_R = OFF_B1 + 8192;
    static constexpr uint32_t OFF_GACC = OFF_R + STAGES * R_BYTES;     // [group][sum, comp][32 cols][GACC_ROWS] FP32
    static constexpr uint32_t OFF_BAR = OFF_GACC + 2 * 2 * 32 * GACC_ROWS * 4;
    static constexpr uint32_t OFF_MISC = OFF_BAR + 32 * 8;
    static constexpr uint32_t SMEM_BYTES = OFF_MISC + 64 + 1024;       // + slack to align the base to 1 KiB
    static_assert(N1 * 64 <= 8192, "B1 operand region");
    static_assert(32 * NSPLIT + NSPLIT <= 128, "rows of the MMA2 accumulator");
    static_assert(3 * 32 * (NCW + 2) * 8 <= 2 * A2_BYTES, "block reduction scratch");
};

// 16-byte chunk c of row `row` in a tile with 64-byte rows and 64-byte swizzle
__device__ __forceinline__ uint32_t sw64(uint32_t row, uint32_t c) { return row * 64 + ((c ^ ((row >> 1) & 3)) << 4); }
// 16-byte chunk c (0..7) of row `row` in a 128-byte-row atom with 128-byte swizzle,
// rows grouped by 8 (1 KiB per group)
__device__ __forceinline__ uint32_t sw128(uint32_t row, uint32_t c)
{
    return (row >> 3) * 1024 + (row & 7) * 128 + ((c ^ (row & 7)) << 4);
}

__device__ __forceinline__ void bf16_split(double x, int nsplit, __nv_bfloat16 *out)
{
    double rsd = x;
    for (int s = 0; s < nsplit; ++s) {
        const __nv_bfloat16 p = __float2bfloat16_rn(static_cast<float>(rsd));
        out[s] = p;
        rsd -= static_cast<double>(__bfloat162float(p));
    }
}

// NSPLIT BF16 parts of an FP32 value (their sum is x to about 8 NSPLIT bits).
template <int NSPLIT>
__device__ __forceinline__ void f32_split(float x, __nv_bfloat16 (&out)[NSPLIT])
{
    float rsd = x;
#pragma unroll
    for (int s = 0; s < NSPLIT; ++s) {
        out[s] = __float2bfloat16_rn(rsd);
        rsd -= __bfloat162float(out[s]);
    }
}

// Same for two values at once: part s of (x, y) as one bf16x2.
template <int NSPLIT>
__device__ __forceinline__ void f32x2_split(float x, float y, __nv_bfloat162 (&out)[NSPLIT])
{
#pragma unroll
    for (int s = 0; s < NSPLIT; ++s) {
        out[s] = __floats2bfloat162_rn(x, y);
        const float2 f = __bfloat1622float2(out[s]);
        x -= f.x;
        y -= f.y;
    }
}

template <int NSPLIT>
__global__ void __launch_bounds__(TcCfg<NSPLIT>::THREADS, 1)
    tc_sweep_kernel(const __grid_constant__ CUtensorMap tmap_d, TcArgs args)
{
    using C = TcCfg<NSPLIT>;
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_addr(smem_raw);
    unsigned char *base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    unsigned char *dtile = base + C::OFF_D;
    unsigned char *a2 = base + C::OFF_A2;
    unsigned char *b1 = base + C::OFF_B1;
    float *rtile = reinterpret_cast<float *>(base + C::OFF_R);
    float *gacc = reinterpret_cast<float *>(base + C::OFF_GACC);
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + C::OFF_BAR);
    uint64_t *full = bars, *empty = bars + 4, *ufull = bars + 8, *uempty = bars + 10, *a2full = bars + 12;
    uint64_t *a2empty = bars + 14, *gfull = bars + 16, *gempty = bars + 18, *drain = bars + 20;
    volatile uint32_t *tslot = reinterpret_cast<volatile uint32_t *>(base + C::OFF_MISC);
    volatile int *s_abort = reinterpret_cast<volatile int *>(base + C::OFF_MISC + 4);
    volatile int *s_last = reinterpret_cast<volatile int *>(base + C::OFF_MISC + 8);

    const SweepArgs &a = args.sa;
    DevState *st = a.st;
    const int S = args.S, M = S - 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nth = blockDim.x;
    const long long V = a.V;
    const long long ntiles = (V + C::TILE - 1) / C::TILE;
    const long long bid = blockIdx.x, nb = gridDim.x;
    const int nk = (ntiles > bid) ? int((ntiles - bid + nb - 1) / nb) : 0;
    constexpr uint64_t BUDGET = 2000000000ull;

    const bool run = (a.mode != MODE_ITER) ||
                     (st->status == ST_OK && !st->converged && st->iter < st->target && st->iter < st->max_iter);

    double t3_64 = 0.0, t4_64 = 0.0, e4_64 = 0.0;              // consumer sums (FP64)
    uint32_t tbase = 0;
    for (int i = tid; i < 2 * 2 * 32 * C::GACC_ROWS; i += nth) gacc[i] = 0.0f;
    if (run) {
        // ---------------- set-up ----------------
        if (tid == 0) {
            for (int i = 0; i < 4; ++i) {
                mbar_init(&full[i], 1);
                mbar_init(&empty[i], 1);
            }
            for (int i = 0; i < 2; ++i) {
                mbar_init(&ufull[i], 1);
                mbar_init(&uempty[i], 4);
                mbar_init(&a2full[i], 4);
                mbar_init(&a2empty[i], 1);
                mbar_init(&gfull[i], 1);
                mbar_init(&gempty[i], C::FLUSH_WARPS);
            }
            mbar_init(drain, 1);
            *s_abort = 0;
            fence_mbar_init();
        }
        for (int i = tid; i < int(2 * C::A2_BYTES / 16); i += nth) reinterpret_cast<uint4 *>(a2)[i] = make_uint4(0, 0, 0, 0);
        // B1 (N1 rows x 32 components, K-major, 64-byte swizzle): rows 32 s + c hold split s of
        // L'(k, c); rows 32 NSPLIT + s hold split s of kappa'(k); L' and kappa' fold in -d_S.
        const float erho_f = (a.mode == MODE_INIT) ? 0.0f : st->sw.erho;
        for (int idx = tid; idx < C::N1 * 32; idx += nth) {
            const int n = idx >> 5, k = idx & 31;
            double x = 0.0;
            int sp = 0;
            if (n < 32 * NSPLIT) {
                sp = n >> 5;
                const int c = n & 31;
                if (c < M) {
                    if (k < M) {
                        x = (k >= c) ? static_cast<double>(st->sw.L[k * (k + 1) / 2 + c]) : 0.0;
                    } else if (k == M) {
                        double cs = 0.0;
                        for (int kk = c; kk < M; ++kk) cs += static_cast<double>(st->sw.L[kk * (kk + 1) / 2 + c]);
                        x = -cs;
                    }
                }
            } else if (n < 32 * NSPLIT + NSPLIT) {
                sp = n - 32 * NSPLIT;
                if (k < M) {
                    x = static_cast<double>(st->sw.kappa[k]);
                } else if (k == M) {
                    double cs = 0.0;
                    for (int kk = 0; kk < M; ++kk) cs += static_cast<double>(st->sw.kappa[kk]);
                    x = -cs;
                }
            }
            __nv_bfloat16 parts[NSPLIT];
            bf16_split(x, NSPLIT, parts);
            *reinterpret_cast<__nv_bfloat16 *>(b1 + sw64(n, k >> 3) + (k & 7) * 2) = parts[sp];
        }
        if (warp == 0) tmem_alloc<C::TMEM_COLS>(const_cast<uint32_t *>(tslot));
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        tbase = *tslot;

        if (warp == 8 && lane == 0) {
            // ---------------- producer: tensor-map TMA of profile and r tiles ----------------
            int issued = 0;
            for (int k = 0; k < nk; ++k) {
                if (*s_abort) break;
                const int s = k & 3;
                if (k >= 4 && !mbar_wait_bounded(&empty[s], uint32_t(((k >> 2) - 1) & 1), BUDGET)) {
                    *s_abort = 1;
                    break;
                }
                const int tile = int(bid + (long long)k * nb);
                mbar_arrive_expect_tx(&full[s], C::D_BYTES + C::R_BYTES);
                tma_load_2d(dtile + s * C::D_BYTES, &tmap_d, 0, tile * C::TILE, &full[s]);
                bulk_load(rtile + s * C::TILE, a.r + (long long)tile * C::TILE, C::R_BYTES, &full[s]);
                issued = k + 1;
            }
            if (*s_abort) {
                // the last copy of each stage may not have been consumed: let it land (bounded)
                for (int k = (issued > 4 ? issued - 4 : 0); k < issued; ++k)
                    (void)mbar_wait_bounded(&full[k & 3], uint32_t((k >> 2) & 1), 200000000ull);
            }
        } else if (warp == 9 && lane == 0) {
            // ---------------- MMA issuer ----------------
            constexpr uint32_t IDESC1 = umma_idesc_bf16(128, C::N1, 0, 0);
            constexpr uint32_t IDESC2 = umma_idesc_bf16(128, 32, 1, 1);
            const uint32_t b1a = smem_addr(b1), a2a = smem_addr(a2), da = smem_addr(dtile);
            for (int k = 0; k <= nk; ++k) {
                if (*s_abort) break;
                if (k < nk) {
                    const int s = k & 3, b = k & 1;
                    if (!mbar_wait_bounded(&full[s], uint32_t((k >> 2) & 1), BUDGET) ||
                        (k >= 2 && !mbar_wait_bounded(&uempty[b], uint32_t(((k >> 1) - 1) & 1), BUDGET))) {
                        *s_abort = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d0 = da + s * C::D_BYTES;
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk)
                        umma_bf16(tbase + C::COL_U + b * C::COL_U_STRIDE, umma_desc(d0 + kk * 32, 16, 512, 4),
                                  umma_desc(b1a + kk * 32, 16, 512, 4), IDESC1, kk > 0 ? 1u : 0u);
                    umma_commit(&ufull[b]);
                }
                if (k >= 1) {
                    const int j = k - 1, b = j & 1, s = j & 3, e = j / C::EPOCH, eb = e & 1;
                    const bool first = (j % C::EPOCH) == 0;
                    if (!mbar_wait_bounded(&a2full[b], uint32_t((j >> 1) & 1), BUDGET) ||
                        (first && e >= 2 && !mbar_wait_bounded(&gempty[eb], uint32_t(((e >> 1) - 1) & 1), BUDGET))) {
                        *s_abort = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = a2a + b * C::A2_BYTES, d0 = da + s * C::D_BYTES;
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk)
                        umma_bf16(tbase + C::COL_G + eb * C::COL_G_STRIDE, umma_desc(a0 + kk * 16 * 128, C::A2_ATOM, 1024, 2),
                                  umma_desc(d0 + kk * 16 * 64, 1024, 512, 4), IDESC2, (first && kk == 0) ? 0u : 1u);
                    umma_commit(&a2empty[b]);
                    umma_commit(&empty[s]);
                    if ((j % C::EPOCH) == C::EPOCH - 1 || j == nk - 1) umma_commit(&gfull[eb]);
                }
            }
            umma_commit(drain);                 // arrives once every MMA issued above has completed
            if (!mbar_wait_bounded(drain, 0u, BUDGET)) *s_abort = 1;
        } else if (warp < 8) {
            // ---------------- consumers ----------------
            // group g takes tiles k = g (mod 2) and flushes the G' epochs e = g (mod 2)
            const int g = warp >> 2, q = warp & 3;
            const int row = 32 * q + lane;
            const uint32_t lanebase = uint32_t(32 * q) << 16;
            const bool flusher = q < C::FLUSH_WARPS;
            int next_e = g;
            float t3 = 0.0f, prod = 1.0f;
            int ex = 0, cnt = 0;
            // adds epoch e of G' (FP32, tensor memory) into this group's compensated FP32 sums
            auto flush_epoch = [&](int e) -> bool {
                const int eb = e & 1;
                const bool okg = mbar_wait_bounded(&gfull[eb], uint32_t((e >> 1) & 1), BUDGET);
                if (__any_sync(0xffffffffu, !okg)) return false;
                tc_fence_after();
                float v[32];
                tmem_ld32(tbase + lanebase + C::COL_G + eb * C::COL_G_STRIDE, v);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&gempty[eb]);
                float *sum = gacc + (g * 2) * 32 * C::GACC_ROWS + row;
                float *cmp = sum + 32 * C::GACC_ROWS;
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const float s0 = sum[c * C::GACC_ROWS];
                    const float y = v[c] - cmp[c * C::GACC_ROWS];
                    const float t = s0 + y;
                    cmp[c * C::GACC_ROWS] = (t - s0) - y;
                    sum[c * C::GACC_ROWS] = t;
                }
                return true;
            };
            const float erho = erho_f;
            const bool binary = args.binary != 0;
            constexpr int WATOM = (32 * NSPLIT) / 64, WCHUNK = ((32 * NSPLIT) % 64) / 8;
            for (int k = g; k < nk; k += 2) {
                if (__any_sync(0xffffffffu, *s_abort)) break;
                if (flusher) {
                    bool ok = true;
                    while (ok && (next_e + 1) * C::EPOCH <= k) {
                        ok = flush_epoch(next_e);
                        next_e += 2;
                    }
                    if (!ok) {
                        *s_abort = 1;
                        break;
                    }
                }
                const int s = k & 3, b = k & 1;
                const long long obs = (bid + (long long)k * nb) * C::TILE + row;
                const bool valid = obs < V;
                const bool okw = mbar_wait_bounded(&full[s], uint32_t((k >> 2) & 1), BUDGET) &&
                                 mbar_wait_bounded(&ufull[b], uint32_t((k >> 1) & 1), BUDGET);
                if (__any_sync(0xffffffffu, !okw)) {
                    *s_abort = 1;
                    break;
                }
                tc_fence_after();
                // v = L~^T D and t = kappa~^T D: sum of the NSPLIT BF16 parts
                float v[32], w32[32], tv[4];
                const uint32_t tu = tbase + lanebase + C::COL_U + b * C::COL_U_STRIDE;
                tmem_ld32(tu, v);
#pragma unroll
                for (int sp = 1; sp < NSPLIT; ++sp) {
                    tmem_ld32(tu + 32 * sp, w32);
#pragma unroll
                    for (int c = 0; c < 32; ++c) v[c] += w32[c];
                }
                tmem_ld4(tu + 32 * NSPLIT, tv);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&uempty[b]);
                float qv = 0.0f, t = 0.0f;
#pragma unroll
                for (int c = 0; c < 32; ++c) qv = fmaf(v[c], v[c], qv);
#pragma unroll
                for (int sp = 0; sp < NSPLIT; ++sp) t += tv[sp];
                // the observation: r and the profile row from the stage
                const unsigned char *drow = dtile + s * C::D_BYTES;
                uint4 ch[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) ch[c] = *reinterpret_cast<const uint4 *>(drow + sw64(row, c));
                const __nv_bfloat16 *dv = reinterpret_cast<const __nv_bfloat16 *>(ch);
                const float dS = __bfloat162float(dv[M]);
                const float rr = rtile[s * C::TILE + row];
                const float e = (rr - dS) - t;
                const float den = fmaf(erho, qv, 1.0f);
                float inv = rcp_approx(den);
                inv = fmaf(inv, fmaf(-den, inv, 1.0f), inv);
                const float c_ = erho * inv;
                float w = c_ * e;
                float gam = fmaf(w, w, -c_);
                if (valid) {
                    const float ei = e * inv;
                    t3 += fmaf(ei, ei, qv * inv);
                    prod *= den;
                    peel_exponent(prod, ex);
                    if (++cnt == 32) {
                        t3_64 += static_cast<double>(t3);
                        t4_64 += static_cast<double>(logf(prod));
                        e4_64 += static_cast<double>(ex);
                        t3 = 0.0f;
                        prod = 1.0f;
                        ex = 0;
                        cnt = 0;
                    }
                } else {
                    w = 0.0f;
                    gam = 0.0f;
                }
                // A2 row of this observation (MN-major, 128-byte swizzle): the NSPLIT parts of
                // gamma d, then the NSPLIT parts of w
                const bool oka = (k < 2) || mbar_wait_bounded(&a2empty[b], uint32_t(((k >> 1) - 1) & 1), BUDGET);
                if (__any_sync(0xffffffffu, !oka)) {
                    *s_abort = 1;
                    break;
                }
                unsigned char *arow = a2 + b * C::A2_BYTES;
                if (binary) {
                    // d in {0, 1}: each part of gamma times d is exact in BF16
                    __nv_bfloat16 gp[NSPLIT];
                    f32_split<NSPLIT>(gam, gp);
#pragma unroll
                    for (int p = 0; p < NSPLIT; ++p) {
                        const __nv_bfloat162 g2 = __halves2bfloat162(gp[p], gp[p]);
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const __nv_bfloat162 *dp = reinterpret_cast<const __nv_bfloat162 *>(&ch[c]);
                            uint4 o;
                            __nv_bfloat162 *op = reinterpret_cast<__nv_bfloat162 *>(&o);
#pragma unroll
                            for (int u = 0; u < 4; ++u) op[u] = __hmul2(g2, dp[u]);
                            *reinterpret_cast<uint4 *>(arow + (p >> 1) * C::A2_ATOM + sw128(row, 4 * (p & 1) + c)) = o;
                        }
                    }
                } else {
                    // general d (exact in BF16): gamma d_x in FP32, then its parts
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const __nv_bfloat162 *dp = reinterpret_cast<const __nv_bfloat162 *>(&ch[c]);
                        uint4 o[NSPLIT];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const float2 df = __bfloat1622float2(dp[u]);
                            __nv_bfloat162 pp[NSPLIT];
                            f32x2_split<NSPLIT>(gam * df.x, gam * df.y, pp);
#pragma unroll
                            for (int p = 0; p < NSPLIT; ++p) reinterpret_cast<__nv_bfloat162 *>(&o[p])[u] = pp[p];
                        }
#pragma unroll
                        for (int p = 0; p < NSPLIT; ++p)
                            *reinterpret_cast<uint4 *>(arow + (p >> 1) * C::A2_ATOM + sw128(row, 4 * (p & 1) + c)) = o[p];
                    }
                }
                {
                    __nv_bfloat16 wp[NSPLIT];
                    f32_split<NSPLIT>(w, wp);
                    uint4 wv = make_uint4(0, 0, 0, 0);
                    __nv_bfloat16 *wq = reinterpret_cast<__nv_bfloat16 *>(&wv);
#pragma unroll
                    for (int p = 0; p < NSPLIT; ++p) wq[p] = wp[p];
                    *reinterpret_cast<uint4 *>(arow + WATOM * C::A2_ATOM + sw128(row, WCHUNK)) = wv;
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&a2full[b]);
            }
            t3_64 += static_cast<double>(t3);
            t4_64 += static_cast<double>(logf(prod));
            e4_64 += static_cast<double>(ex);
            if (flusher && !*s_abort) {
                bool ok = true;
                while (ok && next_e * C::EPOCH < nk) {
                    ok = flush_epoch(next_e);
                    next_e += 2;
                }
                if (!ok) *s_abort = 1;
            }
        }
        // ---------------- every MMA done (issuer's drain wait), every copy landed ----------------
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (warp == 0) tmem_dealloc<C::TMEM_COLS>(tbase);
        if (tid == 0 && *s_abort) atomicCAS(&st->status, ST_OK, ST_ETIMEOUT);
    }
    __syncthreads();

    // ---------------- this block's partial statistics (FP64) ----------------
    const int NG = M * (M + 1) / 2;
    const int NSTAT = NG + M + 3;
    double *red = reinterpret_cast<double *>(base + C::OFF_A2);          // the pipeline is idle
    red[3 * tid + 0] = t3_64;
    red[3 * tid + 1] = t4_64;
    red[3 * tid + 2] = e4_64;
    __syncthreads();
    // G'(x, y) summed over the two groups and the NSPLIT parts (compensated sums: sum - comp)
    auto gval = [&](int x, int y) {
        double v = 0.0;
#pragma unroll
        for (int gg = 0; gg < 2; ++gg) {
            const float *sum = gacc + (gg * 2) * 32 * C::GACC_ROWS;
            const float *cmp = sum + 32 * C::GACC_ROWS;
            v += static_cast<double>(sum[y * C::GACC_ROWS + x]) - static_cast<double>(cmp[y * C::GACC_ROWS + x]);
        }
        return v;
    };
    auto Graw = [&](int x, int y) {
        double v = 0.0;
#pragma unroll
        for (int p = 0; p < NSPLIT; ++p) v += gval(32 * p + x, y);
        return v;
    };
    auto graw = [&](int y) {
        double v = 0.0;
#pragma unroll
        for (int p = 0; p < NSPLIT; ++p) v += gval(32 * NSPLIT + p, y);
        return v;
    };
    double *part = a.partials + size_t(blockIdx.x) * NSTAT;
    for (int j = tid; j < NSTAT; j += nth) {
        double v = 0.0;
        if (j < NG) {                                                     // packed lower G, row r col c
            int r = 0;
            while ((r + 1) * (r + 2) / 2 <= j) ++r;
            const int c = j - r * (r + 1) / 2;
            v = Graw(r, c) - Graw(r, M) - Graw(M, c) + Graw(M, M);
        } else if (j < NG + M) {
            v = graw(j - NG) - graw(M);
        } else {
            const int which = j - NG - M;                                  // T3, T4, E4
            for (int t = 0; t < 32 * C::NCW; ++t) v += red[3 * t + which];
        }
        part[j] = v;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) *s_last = (atomicAdd(&st->ticket, 1u) == gridDim.x - 1) ? 1 : 0;
    __syncthreads();
    if (!*s_last) return;
    __threadfence();
    if (run && st->status == ST_OK) {
        global_update_rt(M, st, a.partials, gridDim.x, a, reinterpret_cast<double *>(base));
    } else if (tid == 0 && a.use_cond) {
        cudaGraphSetConditional(a.cond, 0u);
    }
    if (tid == 0) st->ticket = 0u;
}

// Inputs of the tensor-core sweep, padded to whole tiles of 128 observations:
// profiles (V x S FP32, row-major) -> BF16 rows of 32 components (zero padded,
// Vp rows), r -> r_pad (Vp floats, zero padded).  counts[0] += profile values
// that BF16 does not represent exactly, counts[1] += values other than 0 and 1.
__global__ void tc_inputs_kernel(const float *__restrict__ d, const float *__restrict__ r, long long V, long long Vp,
                                 int S, __nv_bfloat16 *__restrict__ out, float *__restrict__ r_pad,
                                 unsigned long long *counts)
{
    unsigned long long bad = 0, nonbin = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < Vp * 32; i += stride) {
        const long long o = i >> 5;
        const int j = int(i & 31);
        const float x = (j < S && o < V) ? d[o * S + j] : 0.0f;
        const __nv_bfloat16 b = __float2bfloat16_rn(x);
        if (__bfloat162float(b) != x) ++bad;
        if (x != 0.0f && x != 1.0f) ++nonbin;
        out[i] = b;
    }
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < Vp; i += stride)
        r_pad[i] = (i < V) ? r[i] : 0.0f;
    if (bad) atomicAdd(&counts[0], bad);
    if (nonbin) atomicAdd(&counts[1], nonbin);
}

} // namespace vbh
