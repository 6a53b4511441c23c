// vbh_tc.cuh -- the fused CAVI sweep for 12 <= S <= 32 on the tcgen05 tensor
// cores (one persistent CTA per SM).
//
// Same sweep as vbh_sweep.cuh (steps (a)-(e), Eq. 16-31); the two contractions
// that grow with M^2 run as BF16 MMAs with FP32 accumulation in tensor memory:
//   MMA1  U = d_tile (128 x 32) . B1 (32 x 48): per observation the vector
//         v = L~^T D_i (columns 0..31, so q_i = |v|^2) and t_i = kappa~^T D_i
//         (column 32).  The profile column d_S is folded into B1 (row S-1
//         holds minus the column sums), so the MMA reads the raw profiles.  L~
//         and kappa~ (the FP32 globals of the pass) are split into NSPLIT BF16
//         parts, one B1 operand each, and the NSPLIT MMAs accumulate into the
//         same columns.  With binary profiles every product is exact: NSPLIT = 3
//         carries the FP32 values (24 bits), NSPLIT = 2 keeps 16 bits (the BF16
//         form).
//   MMA2  G' = A2 (128 x 128 obs) . d_tile (128 obs x 32): the rows of A2 are
//         the NSPLIT BF16 parts of gamma_i d_i (gamma_i = w_i^2 - c_i) and of
//         w_i, so G' holds sum gamma d d^T and sum w d in the raw-profile basis;
//         G and g of the sweep follow in FP64 by removing the d_S column
//         (G_jk = G'_jk - G'_jS - G'_Sk + G'_SS, g_j = g'_j - g'_S).  G'
//         accumulates in FP32 in tensor memory over an epoch of 16 tiles and is
//         then added into compensated FP32 sums (sum and lost low part).
// The scalar per-observation work (c_i, w_i, S_i, ln(1 + E[rho] q_i)) stays
// on the CUDA cores.  The inputs are repacked once per fit into tiles of 128
// observations, each 8,704 contiguous bytes: the BF16 profiles as the
// 64-byte-swizzled shared-memory image the MMAs read (64-byte rows), then the
// 128 r values.  One bulk copy per tile lands it in a pipeline stage (a
// tensor-map load of the same box moved only ~11 GB/s per SM); the profile tile
// is MMA1's K-major A operand and MMA2's MN-major B operand.
//
// Roles (14 warps): warps 0-7 are two groups of four consumer warps that take
// alternate tiles, each warp owning one quarter of the tensor-memory lanes (32
// observations); warps 8-11 flush the G' epochs (one lane quarter each); warp
// 12 lane 0 issues the loads and warp 13 lane 0 the MMAs.  MMA1 runs two tiles
// ahead of MMA2 (four U buffers in tensor memory, four A2 buffers in shared
// memory), so a consumer group never waits for the MMA of its own previous
// tile.  Every wait is bounded: on a timeout the kernel records VBH_ETIMEOUT,
// lets its copies and MMAs drain, frees its tensor memory and returns.
#pragma once

#include <cuda_bf16.h>

#include "vbh_sweep.cuh"
#include "vbh_tc_host.h"

namespace vbh {

template <int NSPLIT>
struct TcCfg {
    static constexpr int TILE = 128;                                   // observations per tile
    static constexpr int N1 = 48;                                      // MMA1 N: v (32 columns), t (column 32)
    static constexpr int STAGES = 10;                                  // input tiles in flight
    static constexpr int NBUF = 4;                                     // U and A2 buffers (tile k uses k & 3)
    static constexpr uint32_t D_BYTES = TILE * 64;                     // swizzled BF16 profiles
    static constexpr uint32_t STAGE_BYTES = TC_TILE_BYTES;             // + 128 r values
    static constexpr uint32_t B1_PART = N1 * 64;                       // one split of the MMA1 B operand
    static constexpr uint32_t A2_ATOM = TILE * 128;                    // one 64-row atom column
    static constexpr uint32_t A2_BYTES = 2 * A2_ATOM;
    static constexpr int EPOCH = 16;                                   // tiles per G' epoch
    static constexpr int NCW = 8;                                      // consumer warps
    static constexpr int FLUSH_WARP0 = NCW;                            // warps 8..11
    static constexpr int PRODUCER_WARP = NCW + 4;
    static constexpr int MMA_WARP = NCW + 5;
    static constexpr int THREADS = 32 * (NCW + 6);
    static constexpr int TMEM_COLS = 512;
    static constexpr uint32_t COL_U = 0, COL_U_STRIDE = 64;           // U[u] at column 64 u
    static constexpr uint32_t COL_G = 256, COL_G_STRIDE = 32;          // G'[e & 1] at column 256 + 32 (e & 1)
    // rows of G': part p of gamma d in rows 32 p .. 32 p + 31, part p of w in row 32 NSPLIT + p
    static constexpr int GROWS = 33 * NSPLIT;
    static constexpr uint32_t OFF_D = 0;                                // stage s at s * STAGE_BYTES (512-byte aligned)
    static constexpr uint32_t OFF_A2 = ((OFF_D + STAGES * STAGE_BYTES + 1023) / 1024) * 1024;
    static constexpr uint32_t OFF_B1 = OFF_A2 + NBUF * A2_BYTES;
    static constexpr uint32_t OFF_BAR = OFF_B1 + ((NSPLIT * B1_PART + 1023) / 1024) * 1024;
    // mbarrier slots (8 bytes each) from OFF_BAR
    static constexpr int BAR_FULL = 0, BAR_EMPTY = BAR_FULL + STAGES, BAR_UFULL = BAR_EMPTY + STAGES;
    static constexpr int BAR_UEMPTY = BAR_UFULL + NBUF, BAR_A2FULL = BAR_UEMPTY + NBUF;
    static constexpr int BAR_A2EMPTY = BAR_A2FULL + NBUF, BAR_GFULL = BAR_A2EMPTY + NBUF;
    static constexpr int BAR_GEMPTY = BAR_GFULL + 2, BAR_DRAIN = BAR_GEMPTY + 2, NBARS = BAR_DRAIN + 1;
    static constexpr uint32_t OFF_MISC = OFF_BAR + 64 * 8;
    static_assert(NBARS <= 64, "mbarrier slots");
    static constexpr uint32_t SMEM_BYTES = OFF_MISC + 64 + 1024;       // + slack to align the base to 1 KiB
    // end-of-kernel scratch, once the pipeline is idle
    static constexpr uint32_t OFF_GACC = OFF_D;                        // [sum, comp][32 columns][128 rows] FP32
    static constexpr uint32_t OFF_RED = OFF_A2;                        // 3 doubles per thread
    static_assert(GROWS <= 128, "rows of the MMA2 accumulator");
    static_assert(2 * 32 * 128 * 4 <= STAGES * STAGE_BYTES, "G' totals scratch");
    static_assert(STAGE_BYTES % 512 == 0 && D_BYTES + TILE * 4 == STAGE_BYTES, "stage layout");
    static_assert(3 * THREADS * 8 <= NBUF * A2_BYTES, "reduction scratch");
    static_assert(SMEM_BYTES <= 227 * 1024, "shared memory per block");
};

// 16-byte chunk c of row `row` in a tile with 64-byte rows and 64-byte swizzle
__device__ __forceinline__ uint32_t sw64(uint32_t row, uint32_t c) { return row * 64 + ((c ^ ((row >> 1) & 3)) << 4); }
// 16-byte chunk c (0..7) of row `row` in a 128-byte-row atom with 128-byte swizzle,
// rows grouped by 8 (1 KiB per group)
__device__ __forceinline__ uint32_t sw128(uint32_t row, uint32_t c)
{
    return (row >> 3) * 1024 + (row & 7) * 128 + ((c ^ (row & 7)) << 4);
}

// Part `part` of the split of x into BF16 parts (x ~ part 0 + part 1 + ...).
__device__ __forceinline__ __nv_bfloat16 bf16_part(double x, int part)
{
    double rsd = x;
    __nv_bfloat16 p = __float2bfloat16_rn(static_cast<float>(rsd));
    for (int s = 0; s < part; ++s) {
        rsd -= static_cast<double>(__bfloat162float(p));
        p = __float2bfloat16_rn(static_cast<float>(rsd));
    }
    return p;
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
    tc_sweep_kernel(TcArgs args)
{
    using C = TcCfg<NSPLIT>;
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_addr(smem_raw);
    unsigned char *base = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    unsigned char *dtile = base + C::OFF_D;
    unsigned char *a2 = base + C::OFF_A2;
    unsigned char *b1 = base + C::OFF_B1;
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + C::OFF_BAR);
    uint64_t *full = bars + C::BAR_FULL, *empty = bars + C::BAR_EMPTY, *ufull = bars + C::BAR_UFULL;
    uint64_t *uempty = bars + C::BAR_UEMPTY, *a2full = bars + C::BAR_A2FULL, *a2empty = bars + C::BAR_A2EMPTY;
    uint64_t *gfull = bars + C::BAR_GFULL, *gempty = bars + C::BAR_GEMPTY, *drain = bars + C::BAR_DRAIN;
    volatile uint32_t *tslot = reinterpret_cast<volatile uint32_t *>(base + C::OFF_MISC);
    volatile int *s_abort = reinterpret_cast<volatile int *>(base + C::OFF_MISC + 4);
    volatile int *s_last = reinterpret_cast<volatile int *>(base + C::OFF_MISC + 8);
    float *gsum = reinterpret_cast<float *>(base + C::OFF_GACC);
    float *gcmp = gsum + 32 * 128;

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
    if (run) {
        // ---------------- set-up ----------------
        if (tid == 0) {
            for (int i = 0; i < C::STAGES; ++i) {
                mbar_init(&full[i], 1);
                mbar_init(&empty[i], 1);
            }
            for (int i = 0; i < C::NBUF; ++i) {
                mbar_init(&ufull[i], 1);
                mbar_init(&uempty[i], 4);
                mbar_init(&a2full[i], 4);
                mbar_init(&a2empty[i], 1);
            }
            for (int i = 0; i < 2; ++i) {
                mbar_init(&gfull[i], 1);
                mbar_init(&gempty[i], 4);
            }
            mbar_init(drain, 1);
            *s_abort = 0;
            fence_mbar_init();
        }
        for (int i = tid; i < int(C::NBUF * C::A2_BYTES / 16); i += nth)
            reinterpret_cast<uint4 *>(a2)[i] = make_uint4(0, 0, 0, 0);
        // B1 part p (48 rows x 32 components, K-major, 64-byte swizzle): row c < 32 holds split p
        // of L'(k, c), row 32 split p of kappa'(k); L' and kappa' fold in -d_S.
        const float erho_f = (a.mode == MODE_INIT) ? 0.0f : st->sw.erho;
        for (int idx = tid; idx < NSPLIT * C::N1 * 32; idx += nth) {
            const int p = idx / (C::N1 * 32), n = (idx >> 5) % C::N1, k = idx & 31;
            double x = 0.0;
            if (n < M) {
                if (k < M) {
                    x = (k >= n) ? static_cast<double>(st->sw.L[k * (k + 1) / 2 + n]) : 0.0;
                } else if (k == M) {
                    double cs = 0.0;
                    for (int kk = n; kk < M; ++kk) cs += static_cast<double>(st->sw.L[kk * (kk + 1) / 2 + n]);
                    x = -cs;
                }
            } else if (n == 32) {
                if (k < M) {
                    x = static_cast<double>(st->sw.kappa[k]);
                } else if (k == M) {
                    double cs = 0.0;
                    for (int kk = 0; kk < M; ++kk) cs += static_cast<double>(st->sw.kappa[kk]);
                    x = -cs;
                }
            }
            *reinterpret_cast<__nv_bfloat16 *>(b1 + p * C::B1_PART + sw64(n, k >> 3) + (k & 7) * 2) = bf16_part(x, p);
        }
        if (warp == 0) tmem_alloc<C::TMEM_COLS>(const_cast<uint32_t *>(tslot));
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        const uint32_t tbase = *tslot;

        if (warp == C::PRODUCER_WARP) {
            // ---------------- producer: profile tiles (tensor map) and r tiles (bulk copies) ----------------
            if (lane == 0) {
                int issued = 0;
                for (int k = 0; k < nk; ++k) {
                    if (*s_abort) break;
                    const int s = k % C::STAGES;
                    if (k >= C::STAGES &&
                        !mbar_wait_bounded(&empty[s], uint32_t(((k / C::STAGES) - 1) & 1), BUDGET)) {
                        *s_abort = 1;
                        break;
                    }
                    const int tile = int(bid + (long long)k * nb);
                    mbar_arrive_expect_tx(&full[s], C::STAGE_BYTES);
                    bulk_load(dtile + s * C::STAGE_BYTES, args.tiles + (long long)tile * C::STAGE_BYTES, C::STAGE_BYTES,
                              &full[s]);
                    issued = k + 1;
                }
                if (*s_abort) {
                    // the last copy of each stage may not have been consumed: let it land (bounded)
                    for (int k = (issued > C::STAGES ? issued - C::STAGES : 0); k < issued; ++k)
                        (void)mbar_wait_bounded(&full[k % C::STAGES], uint32_t((k / C::STAGES) & 1), BUDGET);
                }
            }
        } else if (warp == C::MMA_WARP) {
            // ---------------- MMA issuer: MMA1 of tile k, then MMA2 of tile k - 2 ----------------
            if (lane == 0) {
                constexpr uint32_t IDESC1 = umma_idesc_bf16(128, C::N1, 0, 0);
                constexpr uint32_t IDESC2 = umma_idesc_bf16(128, 32, 1, 1);
                const uint32_t b1a = smem_addr(b1), a2a = smem_addr(a2), da = smem_addr(dtile);
                for (int k = 0; k < nk + 2; ++k) {
                    if (*s_abort) break;
                    if (k < nk) {
                        const int s = k % C::STAGES, u = k & 3;
                        if (!mbar_wait_bounded(&full[s], uint32_t((k / C::STAGES) & 1), BUDGET) ||
                            (k >= 4 && !mbar_wait_bounded(&uempty[u], uint32_t(((k >> 2) - 1) & 1), BUDGET))) {
                            *s_abort = 1;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t d0 = da + s * C::STAGE_BYTES;
#pragma unroll
                        for (int p = 0; p < NSPLIT; ++p)
#pragma unroll
                            for (int kk = 0; kk < 2; ++kk)
                                umma_bf16(tbase + C::COL_U + u * C::COL_U_STRIDE, umma_desc(d0 + kk * 32, 16, 512, 4),
                                          umma_desc(b1a + p * C::B1_PART + kk * 32, 16, 512, 4), IDESC1,
                                          (p | kk) ? 1u : 0u);
                        umma_commit(&ufull[u]);
                    }
                    if (k >= 2) {
                        const int j = k - 2, b = j & 3, s = j % C::STAGES, e = j / C::EPOCH, eb = e & 1;
                        const bool first = (j % C::EPOCH) == 0;
                        if (!mbar_wait_bounded(&a2full[b], uint32_t((j >> 2) & 1), BUDGET) ||
                            (first && e >= 2 &&
                             !mbar_wait_bounded(&gempty[eb], uint32_t(((e >> 1) - 1) & 1), BUDGET))) {
                            *s_abort = 1;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a0 = a2a + b * C::A2_BYTES, d0 = da + s * C::STAGE_BYTES;
#pragma unroll
                        for (int kk = 0; kk < 8; ++kk)
                            umma_bf16(tbase + C::COL_G + eb * C::COL_G_STRIDE,
                                      umma_desc(a0 + kk * 16 * 128, C::A2_ATOM, 1024, 2),
                                      umma_desc(d0 + kk * 16 * 64, 1024, 512, 4), IDESC2,
                                      (first && kk == 0) ? 0u : 1u);
                        umma_commit(&a2empty[b]);
                        umma_commit(&empty[s]);
                        if ((j % C::EPOCH) == C::EPOCH - 1 || j == nk - 1) umma_commit(&gfull[eb]);
                    }
                }
                umma_commit(drain);             // arrives once every MMA issued above has completed
                if (!mbar_wait_bounded(drain, 0u, BUDGET)) *s_abort = 1;
            }
        } else if (warp >= C::FLUSH_WARP0) {
            // ---------------- flushers: G' epochs -> compensated FP32 sums (one row per lane) ----------------
            const int q = warp - C::FLUSH_WARP0;
            const int row = 32 * q + lane;
            float gs[32], gc[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) gs[c] = gc[c] = 0.0f;
            bool ok = true;
            for (int e = 0; e * C::EPOCH < nk; ++e) {
                if (__any_sync(0xffffffffu, *s_abort)) {
                    ok = false;
                    break;
                }
                const int eb = e & 1;
                const bool okg = mbar_wait_bounded(&gfull[eb], uint32_t((e >> 1) & 1), BUDGET);
                if (__any_sync(0xffffffffu, !okg)) {
                    *s_abort = 1;
                    ok = false;
                    break;
                }
                tc_fence_after();
                float v[32];
                tmem_ld32(tbase + (uint32_t(32 * q) << 16) + C::COL_G + eb * C::COL_G_STRIDE, v);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&gempty[eb]);
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const float y = v[c] - gc[c];
                    const float t = gs[c] + y;
                    gc[c] = (t - gs[c]) - y;
                    gs[c] = t;
                }
            }
            // after the last epoch every MMA has completed and every copy has been consumed, so the
            // stage buffers are free
            if (ok) {
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    gsum[c * 128 + row] = gs[c];
                    gcmp[c * 128 + row] = gc[c];
                }
            }
        } else {
            // ---------------- consumers ----------------
            // group g takes tiles k = g (mod 2); tile k uses U and A2 buffer k & 3
            const int g = warp >> 2, q = warp & 3;
            const int row = 32 * q + lane;
            const uint32_t lanebase = uint32_t(32 * q) << 16;
            const uint32_t ds_off = sw64(row, uint32_t(M) >> 3) + (M & 7) * 2;
            float t3 = 0.0f, prod = 1.0f;
            int ex = 0, cnt = 0;
            const float erho = erho_f;
            const bool binary = args.binary != 0;
            constexpr int WATOM = (32 * NSPLIT) / 64, WCHUNK = ((32 * NSPLIT) % 64) / 8;
            for (int k = g; k < nk; k += 2) {
                if (__any_sync(0xffffffffu, *s_abort)) break;
                const int s = k % C::STAGES, u = k & 3;
                const long long obs = (bid + (long long)k * nb) * C::TILE + row;
                const bool valid = obs < V;
                const bool okw = mbar_wait_bounded(&full[s], uint32_t((k / C::STAGES) & 1), BUDGET) &&
                                 mbar_wait_bounded(&ufull[u], uint32_t((k >> 2) & 1), BUDGET);
                if (__any_sync(0xffffffffu, !okw)) {
                    *s_abort = 1;
                    break;
                }
                tc_fence_after();
                float v[32], t;
                const uint32_t tu = tbase + lanebase + C::COL_U + u * C::COL_U_STRIDE;
                tmem_ld32_1(tu, v, tu + 32, t);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&uempty[u]);
                float q0 = 0.0f, q1 = 0.0f, q2 = 0.0f, q3 = 0.0f;
#pragma unroll
                for (int c = 0; c < 32; c += 4) {
                    q0 = fmaf(v[c], v[c], q0);
                    q1 = fmaf(v[c + 1], v[c + 1], q1);
                    q2 = fmaf(v[c + 2], v[c + 2], q2);
                    q3 = fmaf(v[c + 3], v[c + 3], q3);
                }
                const float qv = (q0 + q1) + (q2 + q3);
                // the observation: r and the profile row from the stage
                const unsigned char *drow = dtile + s * C::STAGE_BYTES;
                uint4 ch[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) ch[c] = *reinterpret_cast<const uint4 *>(drow + sw64(row, c));
                const float dS = __bfloat162float(*reinterpret_cast<const __nv_bfloat16 *>(drow + ds_off));
                const float rr = reinterpret_cast<const float *>(drow + C::D_BYTES)[row];
                const float e = (rr - dS) - t;
                const float den = fmaf(erho, qv, 1.0f);
                float inv = rcp_approx(den);
                inv = fmaf(inv, fmaf(-den, inv, 1.0f), inv);
                const float c_ = erho * inv;
                const float ei = e * inv;
                const float w = valid ? c_ * e : 0.0f;
                const float gam = valid ? fmaf(c_ * e, c_ * e, -c_) : 0.0f;
                t3 += valid ? fmaf(ei, ei, qv * inv) : 0.0f;
                prod *= valid ? den : 1.0f;
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
                // A2 row of this observation (MN-major, 128-byte swizzle): the NSPLIT parts of
                // gamma d, then the NSPLIT parts of w
                const bool oka = (k < 4) || mbar_wait_bounded(&a2empty[u], uint32_t(((k >> 2) - 1) & 1), BUDGET);
                if (__any_sync(0xffffffffu, !oka)) {
                    *s_abort = 1;
                    break;
                }
                unsigned char *arow = a2 + u * C::A2_BYTES;
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
                            for (int h = 0; h < 4; ++h) op[h] = __hmul2(g2, dp[h]);
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
                        for (int h = 0; h < 4; ++h) {
                            const float2 df = __bfloat1622float2(dp[h]);
                            __nv_bfloat162 pp[NSPLIT];
                            f32x2_split<NSPLIT>(gam * df.x, gam * df.y, pp);
#pragma unroll
                            for (int p = 0; p < NSPLIT; ++p) reinterpret_cast<__nv_bfloat162 *>(&o[p])[h] = pp[p];
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
                if (lane == 0) mbar_arrive(&a2full[u]);
            }
            t3_64 += static_cast<double>(t3);
            t4_64 += static_cast<double>(logf(prod));
            e4_64 += static_cast<double>(ex);
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
    double *red = reinterpret_cast<double *>(base + C::OFF_RED);
    red[3 * tid + 0] = t3_64;
    red[3 * tid + 1] = t4_64;
    red[3 * tid + 2] = e4_64;
    __syncthreads();
    // G'(x, y) as sum - comp; summed over the NSPLIT parts
    auto gval = [&](int x, int y) {
        return static_cast<double>(gsum[y * 128 + x]) - static_cast<double>(gcmp[y * 128 + x]);
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
    const bool have = run && *s_abort == 0;
    for (int j = tid; j < NSTAT; j += nth) {
        double v = 0.0;
        if (!have) {
            v = 0.0;
        } else if (j < NG) {                                              // packed lower G, row r col c
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

// Inputs of the tensor-core sweep, repacked into tiles of 128 observations
// (TC_TILE_BYTES each): the profiles (V x S FP32, row-major) as BF16 rows of 32
// components (zero padded) in the 64-byte-swizzled order of the kernel's shared
// memory (16-byte chunk c of row j at j * 64 + ((c ^ ((j >> 1) & 3)) << 4)),
// then the tile's r values (FP32); rows past V are zero.  counts[0] += profile
// values that BF16 does not represent exactly, counts[1] += values other than
// 0 and 1.
__global__ void tc_inputs_kernel(const float *__restrict__ d, const float *__restrict__ r, long long V, int S,
                                 unsigned char *__restrict__ out, unsigned long long *counts)
{
    unsigned long long bad = 0, nonbin = 0;
    const long long ntiles = (V + 127) / 128;
    const long long stride = (long long)gridDim.x * blockDim.x;
    // one thread per (observation, 8-component chunk)
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ntiles * 128 * 4; i += stride) {
        const long long o = i >> 2;
        const int c = int(i & 3);
        const uint32_t j = uint32_t(o & 127);
        __align__(16) __nv_bfloat16 b[8];
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            const int col = 8 * c + h;
            const float x = (col < S && o < V) ? d[o * S + col] : 0.0f;
            b[h] = __float2bfloat16_rn(x);
            if (__bfloat162float(b[h]) != x) ++bad;
            if (x != 0.0f && x != 1.0f) ++nonbin;
        }
        unsigned char *tile = out + (o >> 7) * (long long)TC_TILE_BYTES;
        *reinterpret_cast<uint4 *>(tile + j * 64 + ((uint32_t(c) ^ ((j >> 1) & 3)) << 4)) =
            *reinterpret_cast<const uint4 *>(b);
        if (c == 0) reinterpret_cast<float *>(tile + 128 * 64)[j] = (o < V) ? r[o] : 0.0f;
    }
    if (bad) atomicAdd(&counts[0], bad);
    if (nonbin) atomicAdd(&counts[1], nonbin);
}

} // namespace vbh
