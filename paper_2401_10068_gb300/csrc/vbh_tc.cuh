// vbh_tc.cuh -- the fused CAVI sweep for 12 <= S <= 32 on the tcgen05 tensor
// cores (one persistent CTA per SM).
//
// Same sweep as vbh_sweep.cuh (steps (a)-(e), Eq. 16-31); the two contractions
// that grow with M^2 run as BF16 MMAs with FP32 accumulation in tensor memory.
// The inputs are repacked once per fit into tiles of 128 observations in the
// basis of Eq. 3: per observation the M differences D_ij = d_ij - d_iS as BF16
// in slots 0..M-1 of 32 slots, the constant 1 in slot 31 (free for S <= 32,
// since D has M <= 31 entries) and y_i = r_i - d_iS in FP32.  The BF16 part of
// a tile is slot-major ("comp-major"): for each slot, the tile's observations
// are contiguous, so that both operands of MMA2 are K-major.
//   MMA1  U = [D~_tile .. D~_tile] (128 x 32 NSPLIT) . [B1_0; ..; B1_{NSPLIT-1}]
//         (32 NSPLIT x 32): per observation v = L~^T D_i in columns 0..30
//         (q_i = |v|^2) and t_i = kappa~^T D_i in column 31.  L~ and kappa~
//         (the FP32 globals of the pass) are split into NSPLIT BF16 parts; the
//         parts are stacked along K (part p meets the tile's slots in K steps
//         2p, 2p + 1), so the tensor core adds them in its FP32 accumulator.
//         With D in {-1, 0, 1} every product is exact: NSPLIT = 3 carries the
//         FP32 values (24 bits), NSPLIT = 2 keeps 16 bits (the BF16 form).
//   MMA2  G'' = A2 . D~_tile^T: row (p, j) of A2 holds part p of
//         gamma_i D_ij (gamma_i = w_i^2 - c_i) for j < 31 and part p of w_i in
//         slot 31, with the observations along K; against the D~ rows this
//         gives sum gamma D D^T and, in row (p, 31), sum w D (slot 31 of D~ is
//         1).  In the BF16 form two sets of 64 observations share one MMA: A2
//         rows 0-63 belong to observations 0-63 and rows 64-127 to 64-127, B is
//         the 64 slot rows of both sets, so each MMA covers 32 observations (the
//         cross blocks of the output are not read).  G'' accumulates in FP32 in
//         tensor memory over an epoch of 16 tiles and is then added into
//         compensated FP32 sums (sum and lost low part).
// The scalar per-observation work (c_i, w_i, S_i, ln(1 + E[rho] q_i)) stays
// on the CUDA cores; the consumer threads then stage the BF16 parts of gamma
// and build A2: in the FP32 form in shared memory, in chunks of 8
// observations; in the BF16 form in tensor memory, each consumer thread
// forming one A2 row (set, part, slot) over its set's 64 observations and
// storing it with tcgen05.st, MMA2 then taking its A operand from tensor
// memory.  Two tiles (17,408 contiguous bytes) land in a pipeline stage by one
// bulk copy.
//
// Roles (15 warps): warps 0-7 are two groups of four consumer warps that take
// alternate tiles, each warp owning one quarter of the tensor-memory lanes (32
// observations); warps 8-11 flush the G'' epochs (one lane quarter each); lane
// 0 of warp 12 issues the loads, of warp 13 the MMA1s and of warp 14 the
// MMA2s.  MMA1 runs ahead of the consumers into one U buffer per consumer
// group in tensor memory, and four A2 buffers decouple the consumers from
// MMA2.  Every buffer is assigned so that all tiles using it belong to one
// consumer group, so each mbarrier parity wait follows its waiter's wait of
// the previous phase (static assertions below).  Every wait is bounded: on a
// timeout the kernel records VBH_ETIMEOUT, lets its copies and MMAs drain,
// frees its tensor memory and returns.
#pragma once

#include <cuda_bf16.h>

#include "vbh_sweep.cuh"
#include "vbh_tc_host.h"

namespace vbh {

// 16 consecutive 32-bit columns of this thread's TMEM lane (32x32b shape, x16),
// without the wait.
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(taddr));
}

// Layout of the BF16 part of a tile (8 KiB, two 4 KiB blocks j of 64 rows x 64
// bytes, 64-byte swizzle): observation o of slot x sits in block (o >> 5) & 1,
// row 32 (o >> 6) + x, element o & 31.
__host__ __device__ constexpr uint32_t tc_slot_byte(uint32_t o, uint32_t x)
{
    return ((o >> 5) & 1u) * 4096u + (32u * (o >> 6) + x) * 64u +
           ((((o & 31u) >> 3) ^ (((32u * (o >> 6) + x) >> 1) & 3u)) << 4) + (o & 7u) * 2u;
}

template <int NSPLIT>
struct TcCfg {
    static constexpr int TILE = 128;                                   // observations per tile
    static constexpr int SETS = (NSPLIT == 2) ? 2 : 1;                 // observation sets per MMA2
    static constexpr int N1 = 32;                                      // MMA1 N: v (31 columns), then t
    static constexpr int N2 = 32 * SETS;                               // MMA2 N
    static constexpr int NK2 = 8 / SETS;                               // MMA2 instructions per tile (K = 16)
    static constexpr int NCG = 2;                                      // consumer groups (tile k: group k % NCG)
    static constexpr int STAGES = (NSPLIT == 2) ? 8 : 4;               // pipeline stages of two tiles
    static constexpr int NUBUF = NCG;                                  // U buffers (tile k uses k % NUBUF)
    static constexpr int NBUF = 4;                                     // A2 buffers (tile k uses k % NBUF)
    static constexpr uint32_t D_BYTES = TILE * 64;                     // BF16 slots of a tile
    static constexpr uint32_t TILE_BYTES = TC_TILE_BYTES;              // + 128 y values
    static constexpr uint32_t STAGE_BYTES = 2 * TILE_BYTES;
    static constexpr uint32_t B1_BYTES = NSPLIT * 32 * 64;             // NSPLIT blocks of 32 rows x 32 slots
    static constexpr uint32_t A2_BLOCK = 128 * 64;                     // 128 rows x 32 observations (or pairs)
    static constexpr uint32_t A2_BYTES = (TILE / SETS / 32) * A2_BLOCK;
    static constexpr bool TMEM_A2 = (NSPLIT == 2);                     // A2 in tensor memory (BF16 form)
    static constexpr uint32_t GAM_BYTES = (TMEM_A2 ? 2 : 1) * NSPLIT * TILE * 2;   // staged BF16 parts of gamma (and w)
    static constexpr int EPOCH = 16;                                   // tiles per G'' epoch
    static constexpr int NCW = 4 * NCG;                                // consumer warps
    static constexpr int FLUSH_WARP0 = NCW;                            // four flusher warps
    static constexpr int PRODUCER_WARP = NCW + 4;
    static constexpr int MMA1_WARP = NCW + 5;                          // issues MMA1 (runs ahead)
    static constexpr int MMA2_WARP = NCW + 6;                          // issues MMA2
    static constexpr int THREADS = 32 * (NCW + 7);
    static constexpr int TMEM_COLS = 512;
    static constexpr uint32_t COL_U = 0, COL_U_STRIDE = TMEM_A2 ? N1 : 128;   // U[u] at column COL_U_STRIDE u
    static constexpr uint32_t COL_A2 = NUBUF * COL_U_STRIDE, A2_COLS = 32;      // TMEM A2[b] at COL_A2 + 32 b
    static constexpr uint32_t COL_G = 384, COL_G_STRIDE = N2;          // G''[e & 1] at column 384 + N2 (e & 1)
    static constexpr int NTASK = 31 * (TILE / 8);                     // A2 chunks (8 observations) per part
    static constexpr uint32_t OFF_D = 0;                                // stage s at s * STAGE_BYTES (512-byte aligned)
    static constexpr uint32_t OFF_A2 = ((OFF_D + STAGES * STAGE_BYTES + 1023) / 1024) * 1024;
    // A2 in shared memory, or (A2 in tensor memory) only the end-of-kernel reduction scratch
    static constexpr uint32_t A2_REGION = TMEM_A2 ? ((3 * THREADS * 8 + 1023) / 1024) * 1024 : NBUF * A2_BYTES;
    static constexpr uint32_t OFF_B1 = OFF_A2 + A2_REGION;
    static constexpr uint32_t OFF_GAM = OFF_B1 + ((B1_BYTES + 1023) / 1024) * 1024;
    // the flushers' compensation terms (3-group form: kept out of registers) [32 columns][128 rows]
    static constexpr uint32_t GC_BYTES = (NCG == 3) ? 32 * 128 * 4 : 0;
    static constexpr uint32_t OFF_GC = OFF_GAM + ((NBUF * GAM_BYTES + 1023) / 1024) * 1024;
    static constexpr uint32_t OFF_BAR = OFF_GC + GC_BYTES;
    // mbarrier slots (8 bytes each) from OFF_BAR
    static constexpr int BAR_FULL = 0, BAR_EMPTY = BAR_FULL + STAGES, BAR_UFULL = BAR_EMPTY + STAGES;
    static constexpr int BAR_UEMPTY = BAR_UFULL + NUBUF, BAR_A2FULL = BAR_UEMPTY + NUBUF;
    static constexpr int BAR_A2EMPTY = BAR_A2FULL + NBUF, BAR_STAGED = BAR_A2EMPTY + NBUF;
    static constexpr int BAR_GFULL = BAR_STAGED + NBUF, BAR_GEMPTY = BAR_GFULL + 2, BAR_DRAIN = BAR_GEMPTY + 2;
    static constexpr int NBARS = BAR_DRAIN + 2;                        // one drain barrier per MMA issuer
    static constexpr uint32_t OFF_MISC = OFF_BAR + 64 * 8;
    static constexpr uint32_t SMEM_BYTES = OFF_MISC + 64 + 1024;       // + slack to align the base to 1 KiB
    // end-of-kernel scratch, once the pipeline is idle
    static constexpr uint32_t OFF_GACC = OFF_D;                        // [sum, comp][32 columns][128 rows] FP32
    static constexpr uint32_t OFF_RED = OFF_A2;                        // 3 doubles per thread
    static_assert(NBARS <= 64, "mbarrier slots");
    static_assert(SETS * 32 * NSPLIT <= 128 && (SETS == 1 || 32 * NSPLIT <= 64), "rows of the MMA2 accumulator");
    static_assert(COL_U + NUBUF * COL_U_STRIDE <= COL_G && COL_G + 2 * COL_G_STRIDE <= TMEM_COLS, "tensor memory");
    static_assert(N1 <= COL_U_STRIDE && N1 * 64 <= 8192, "MMA1 shape");
    static_assert(2 * 32 * 128 * 4 <= STAGES * STAGE_BYTES, "G'' totals scratch");
    static_assert(TILE_BYTES % 512 == 0 && D_BYTES + TILE * 4 == TILE_BYTES, "tile layout");
    static_assert(3 * THREADS * 8 <= A2_REGION, "reduction scratch");
    // An mbarrier parity wait is only sound when the waiter has waited for the barrier's previous
    // phase too (a wait for parity 1 passes while phase 0 is still open).  So every buffer is
    // used by one consumer group only: the tiles sharing a U buffer, an A2 buffer or a stage
    // (k and k + NUBUF, k + NBUF, k + 2 STAGES) belong to the same group, and each group waits
    // the phases of its buffers in order.
    static_assert(NUBUF % NCG == 0 && NBUF % NCG == 0 && (2 * STAGES) % NCG == 0,
                  "buffers shared across consumer groups");
    static_assert(SMEM_BYTES <= 227 * 1024, "shared memory per block");
    static_assert(!TMEM_A2 || (SETS == 2 && COL_A2 % 16 == 0 && COL_A2 + NBUF * A2_COLS <= COL_G),
                  "tensor memory of the A2 buffers");
    static_assert(D_BYTES <= 8192 && A2_BYTES <= 32768 && TILE / 8 <= 16, "packed chunk offsets (13 + 15 + 4 bits)");
    static_assert(size_t(gu_ws_doubles_rt(MMAX)) * 8 <= OFF_MISC, "workspace of the global update");
};

// 16-byte chunk c of row `row` in a region with 64-byte rows and 64-byte swizzle
__device__ __forceinline__ uint32_t sw64(uint32_t row, uint32_t c) { return row * 64 + ((c ^ ((row >> 1) & 3)) << 4); }

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

// Byte offset in an A2 buffer of element (row m, observation o) for the given
// number of sets: K-major, 64-byte swizzle, blocks of 32 observations (pairs)
// of 128 rows x 64 bytes.
template <int SETS>
__device__ __forceinline__ uint32_t a2_byte(uint32_t m, uint32_t o)
{
    const uint32_t k = (SETS == 2) ? (o & 63u) : o;                    // K index: pair or observation
    return (k >> 5) * 8192u + sw64(m, (k & 31u) >> 3) + (k & 7u) * 2u;
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
    __nv_bfloat16 *gam = reinterpret_cast<__nv_bfloat16 *>(base + C::OFF_GAM);
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + C::OFF_BAR);
    uint64_t *full = bars + C::BAR_FULL, *empty = bars + C::BAR_EMPTY, *ufull = bars + C::BAR_UFULL;
    uint64_t *uempty = bars + C::BAR_UEMPTY, *a2full = bars + C::BAR_A2FULL, *a2empty = bars + C::BAR_A2EMPTY;
    uint64_t *staged = bars + C::BAR_STAGED, *gfull = bars + C::BAR_GFULL, *gempty = bars + C::BAR_GEMPTY;
    uint64_t *drain = bars + C::BAR_DRAIN;
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
    // this block's tiles: pairs of consecutive tiles (one stage each) taken round robin
    const long long npairs = ((V + C::TILE - 1) / C::TILE + 1) / 2;
    const long long bid = blockIdx.x, nb = gridDim.x;
    const int npb = (npairs > bid) ? int((npairs - bid + nb - 1) / nb) : 0;
    const int nk = 2 * npb;
    constexpr uint64_t BUDGET = 2000000000ull;

    const bool run = (a.mode != MODE_ITER) ||
                     (st->status == ST_OK && !st->converged && st->iter < st->target && st->iter < st->max_iter);

    double t3_64 = 0.0, t4_64 = 0.0, e4_64 = 0.0;              // consumer sums (FP64)
    if (run) {
        // ---------------- set-up ----------------
        if (tid == 0) {
            for (int i = 0; i < C::STAGES; ++i) {
                mbar_init(&full[i], 1);
                mbar_init(&empty[i], 2);                        // both tiles' MMA2
            }
            for (int i = 0; i < C::NUBUF; ++i) {
                mbar_init(&ufull[i], 1);
                mbar_init(&uempty[i], 4);
            }
            for (int i = 0; i < C::NBUF; ++i) {
                mbar_init(&a2full[i], 4);
                mbar_init(&a2empty[i], 1);
                mbar_init(&staged[i], 4);
            }
            for (int i = 0; i < 2; ++i) {
                mbar_init(&gfull[i], 1);
                mbar_init(&gempty[i], 4);
            }
            mbar_init(&drain[0], 1);
            mbar_init(&drain[1], 1);
            *s_abort = 0;
            fence_mbar_init();
        }
        for (int i = tid; i < int(C::A2_REGION / 16); i += nth)
            reinterpret_cast<uint4 *>(a2)[i] = make_uint4(0, 0, 0, 0);
        // B1: NSPLIT blocks of 32 rows x 32 slots (K-major, 64-byte swizzle, 2 KiB each); row c < 31
        // of block p holds part p of column c of L~ (L~(k, c) at slot k), row 31 part p of kappa~;
        // slot 31 (the constant 1 of the tile rows) meets zeros.
        const float erho_f = st->sw.erho;       // 0 in sweep 0 of a CAVI fit from the paper's start
        for (int idx = tid; idx < NSPLIT * 32 * 32; idx += nth) {
            const int n = idx >> 5, k = idx & 31;
            const int p = n >> 5, c = n & 31;
            double x = 0.0;
            if (c < 31) {
                if (c < M && k < M && k >= c) x = static_cast<double>(st->sw.L[k * (k + 1) / 2 + c]);
            } else if (k < M) {
                x = static_cast<double>(st->sw.kappa[k]);
            }
            *reinterpret_cast<__nv_bfloat16 *>(b1 + sw64(n, k >> 3) + (k & 7) * 2) = bf16_part(x, p);
        }
        if (warp == 0) tmem_alloc<C::TMEM_COLS>(const_cast<uint32_t *>(tslot));
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        const uint32_t tbase = *tslot;

        if (warp == C::PRODUCER_WARP) {
            // ---------------- producer: one bulk copy of two tiles per stage ----------------
            if (lane == 0) {
                int issued = 0;
                for (int i = 0; i < npb; ++i) {
                    if (*s_abort) break;
                    const int s = i % C::STAGES;
                    if (i >= C::STAGES &&
                        !mbar_wait_bounded(&empty[s], uint32_t(((i / C::STAGES) - 1) & 1), BUDGET)) {
                        *s_abort = 1;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[s], C::STAGE_BYTES);
                    bulk_load(dtile + s * C::STAGE_BYTES, args.tiles + (bid + (long long)i * nb) * C::STAGE_BYTES,
                              C::STAGE_BYTES, &full[s]);
                    issued = i + 1;
                }
                if (*s_abort) {
                    // the last copy of each stage may not have been consumed: let it land (bounded)
                    for (int i = (issued > C::STAGES ? issued - C::STAGES : 0); i < issued; ++i)
                        (void)mbar_wait_bounded(&full[i % C::STAGES], uint32_t((i / C::STAGES) & 1), BUDGET);
                }
            }
        } else if (warp == C::MMA1_WARP) {
            // ---------------- MMA1 issuer: U of tile k as soon as its inputs and a U buffer are there ----------------
            if (lane == 0) {
                constexpr uint32_t IDESC1 = umma_idesc_bf16(128, C::N1, 1, 0);
                const uint32_t b1a = smem_addr(b1), da = smem_addr(dtile);
                for (int k = 0; k < nk; ++k) {
                    if (*s_abort) break;
                    const int i = k >> 1, s = i % C::STAGES, u = k % C::NUBUF;
                    if (!mbar_wait_bounded(&full[s], uint32_t((i / C::STAGES) & 1), BUDGET) ||
                        (k >= C::NUBUF &&
                         !mbar_wait_bounded(&uempty[u], uint32_t(((k / C::NUBUF) - 1) & 1), BUDGET))) {
                        *s_abort = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d0 = da + s * C::STAGE_BYTES + (k & 1) * C::TILE_BYTES;
                    // A = the tile's slots as an MN-major operand: four atoms of 32 observations
                    // (2 KiB apart), K step 16 slots = 1 KiB; the same two K steps once per part
                    // of B1 (block p, 2 KiB apart), all accumulating into one U
#pragma unroll
                    for (int p = 0; p < NSPLIT; ++p)
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk)
                            umma_bf16(tbase + C::COL_U + u * C::COL_U_STRIDE, umma_desc(d0 + kk * 1024, 2048, 512, 4),
                                      umma_desc(b1a + p * 2048 + kk * 32, 16, 512, 4), IDESC1, (p | kk) ? 1u : 0u);
                    umma_commit(&ufull[u]);
                }
                umma_commit(&drain[0]);         // arrives once every MMA issued above has completed
                if (!mbar_wait_bounded(&drain[0], 0u, BUDGET)) *s_abort = 1;
            }
        } else if (warp == C::MMA2_WARP) {
            // ---------------- MMA2 issuer: G'' += A2 . D~ of tile j once its A2 is built ----------------
            if (lane == 0) {
                constexpr uint32_t IDESC2 = umma_idesc_bf16(128, C::N2, 0, 0);
                const uint32_t a2a = smem_addr(a2), da = smem_addr(dtile);
                for (int j = 0; j < nk; ++j) {
                    if (*s_abort) break;
                    const int b = j % C::NBUF, i = j >> 1, s = i % C::STAGES;
                    const int e = j / C::EPOCH, eb = e & 1;
                    const bool first = (j % C::EPOCH) == 0;
                    if (!mbar_wait_bounded(&full[s], uint32_t((i / C::STAGES) & 1), BUDGET) ||
                        !mbar_wait_bounded(&a2full[b], uint32_t((j / C::NBUF) & 1), BUDGET) ||
                        (first && e >= 2 &&
                         !mbar_wait_bounded(&gempty[eb], uint32_t(((e >> 1) - 1) & 1), BUDGET))) {
                        *s_abort = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = a2a + b * C::A2_BYTES;
                    const uint32_t d0 = da + s * C::STAGE_BYTES + (j & 1) * C::TILE_BYTES;
#pragma unroll
                    for (int kk = 0; kk < C::NK2; ++kk) {
                        // K step kk: 16 observations (pairs) = half of a 32-wide block
                        const uint32_t blk = uint32_t(kk >> 1), half = uint32_t(kk & 1) * 32;
                        const uint32_t boff = (C::SETS == 2) ? blk * 4096 + half
                                                             : (blk & 1) * 4096 + (blk >> 1) * 2048 + half;
                        if constexpr (C::TMEM_A2)
                            umma_bf16_ts(tbase + C::COL_G + eb * C::COL_G_STRIDE,
                                         tbase + C::COL_A2 + C::A2_COLS * uint32_t(b) + 8 * uint32_t(kk),
                                         umma_desc(d0 + boff, 16, 512, 4), IDESC2, (first && kk == 0) ? 0u : 1u);
                        else
                            umma_bf16(tbase + C::COL_G + eb * C::COL_G_STRIDE,
                                      umma_desc(a0 + blk * 8192 + half, 16, 512, 4), umma_desc(d0 + boff, 16, 512, 4),
                                      IDESC2, (first && kk == 0) ? 0u : 1u);
                    }
                    umma_commit(&a2empty[b]);
                    umma_commit(&empty[s]);
                    if ((j % C::EPOCH) == C::EPOCH - 1 || j == nk - 1) umma_commit(&gfull[eb]);
                }
                umma_commit(&drain[1]);
                if (!mbar_wait_bounded(&drain[1], 0u, BUDGET)) *s_abort = 1;
            }
        } else if (warp >= C::FLUSH_WARP0 && warp < C::FLUSH_WARP0 + 4) {
            // ---------------- flushers: G'' epochs -> compensated FP32 sums (one row per lane) ----------------
            const int q = warp - C::FLUSH_WARP0;
            const int row = 32 * q + lane;
            float gs[32], gc[(C::NCG == 3) ? 1 : 32];
            float *gcs = reinterpret_cast<float *>(base + C::OFF_GC);   // used by the 3-group form
            // compensation term of column c of this thread's row
            auto gcr = [&](int c) -> float & {
                if constexpr (C::NCG == 3) return gcs[c * 128 + row];
                else return gc[c];
            };
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                gs[c] = 0.0f;
                gcr(c) = 0.0f;
            }
            bool ok = true;
            for (int e = 0; e * C::EPOCH < nk; ++e) {
                if (__any_sync(0xffffffffu, *s_abort)) {
                    ok = false;
                    break;
                }
                const int eb = e & 1;
                const bool okg = mbar_wait_backoff(&gfull[eb], uint32_t((e >> 1) & 1), BUDGET);
                if (__any_sync(0xffffffffu, !okg)) {
                    *s_abort = 1;
                    ok = false;
                    break;
                }
                tc_fence_after();
                // rows 0..63 read the first 32 columns; with two sets rows 64..127 read the next 32;
                // two halves of 16 columns (fewer live registers next to the 64 running sums)
                const uint32_t colset = (C::SETS == 2 && q >= 2) ? 32u : 0u;
                const uint32_t tg = tbase + (uint32_t(32 * q) << 16) + C::COL_G + eb * C::COL_G_STRIDE + colset;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint32_t vr[16];
                    tmem_ld16_nowait(tg + 16 * h, vr);
                    tmem_wait_regs(vr);
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        float &cc = gcr(16 * h + c);
                        const float y = __uint_as_float(vr[c]) - cc;
                        const float t = gs[16 * h + c] + y;
                        cc = (t - gs[16 * h + c]) - y;
                        gs[16 * h + c] = t;
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&gempty[eb]);
            }
            // after the last epoch every MMA has completed and every copy has been consumed, so the
            // stage buffers are free
            if (ok) {
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    gsum[c * 128 + row] = gs[c];
                    gcmp[c * 128 + row] = gcr(c);
                }
            }
        } else {
            // ---------------- consumers ----------------
            // group g takes tiles k = g (mod NCG); tile k uses U buffer k % NUBUF, A2 buffer k % NBUF
            const int g = warp >> 2, q = warp & 3;
            const int row = 32 * q + lane;                       // tensor-memory lane
            // U row `row` belongs to observation obs_row of the tile: the MMA1 atoms are the
            // 32-observation runs 0, 64, 32, 96 (bits 5 and 6 of the row swapped)
            const uint32_t o_r = (uint32_t(row) & 31u) | ((uint32_t(row) & 32u) << 1) | ((uint32_t(row) & 64u) >> 1);
            const uint32_t lanebase = uint32_t(32 * q) << 16;
            const int gt = tid & 127;                            // thread within the group
            // this thread's A2 chunk tasks (slot x < 31 of 8 observations), the same in every
            // tile: source byte in the tile's BF16 part (13 bits), destination byte of part 0 in
            // an A2 buffer (15 bits; part p is 2048 p further) and the chunk (4 bits), packed
            constexpr int TPT = (C::NTASK + 127) / 128;
            uint32_t tpk[TPT];
#pragma unroll
            for (int i = 0; i < TPT; ++i) {
                const int task = gt + 128 * i;
                const uint32_t x = uint32_t(task % 31), ch = uint32_t(task / 31) & 15u, o0 = 8u * ch;
                const uint32_t set = (C::SETS == 2) ? (o0 >> 6) : 0u;
                tpk[i] = tc_slot_byte(o0, x) | (a2_byte<C::SETS>(64 * set + x, o0) << 13) | (ch << 28);
            }
            float t3 = 0.0f, prod = 1.0f;
            int ex = 0, cnt = 0;
            const float erho = erho_f;
            const bool binary = args.binary != 0;
            for (int k = g; k < nk; k += C::NCG) {
                if (__any_sync(0xffffffffu, *s_abort)) break;
                const int i = k >> 1, s = i % C::STAGES, u = k % C::NUBUF, b = k % C::NBUF;
                const long long tile = 2 * (bid + (long long)i * nb) + (k & 1);
                const bool valid = tile * C::TILE + o_r < V;
                const bool okw = mbar_wait_backoff(&full[s], uint32_t((i / C::STAGES) & 1), BUDGET) &&
                                 mbar_wait_backoff(&ufull[u], uint32_t((k / C::NUBUF) & 1), BUDGET);
                if (__any_sync(0xffffffffu, !okw)) {
                    *s_abort = 1;
                    break;
                }
                tc_fence_after();
                // v = L~^T D (columns 0..30, q = |v|^2) and t = kappa~^T D (column 31), the parts
                // already added by MMA1: one tensor-memory round trip of 32 columns
                const uint32_t tu = tbase + lanebase + C::COL_U + u * C::COL_U_STRIDE;
                float q0 = 0.0f, q1 = 0.0f, q2 = 0.0f, q3 = 0.0f, t;
                {
                    uint32_t ua[16], ub[16];
                    tmem_ld16_nowait(tu, ua);
                    tmem_ld16_nowait(tu + 16, ub);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        asm volatile("" : "+r"(ua[c]));
                        asm volatile("" : "+r"(ub[c]));
                    }
#pragma unroll
                    for (int c = 0; c < 16; c += 4) {
                        const float v0 = __uint_as_float(ua[c]), v1 = __uint_as_float(ua[c + 1]);
                        const float v2 = __uint_as_float(ua[c + 2]), v3 = __uint_as_float(ua[c + 3]);
                        q0 = fmaf(v0, v0, q0);
                        q1 = fmaf(v1, v1, q1);
                        q2 = fmaf(v2, v2, q2);
                        q3 = fmaf(v3, v3, q3);
                    }
#pragma unroll
                    for (int c = 0; c < 12; c += 4) {
                        const float v0 = __uint_as_float(ub[c]), v1 = __uint_as_float(ub[c + 1]);
                        const float v2 = __uint_as_float(ub[c + 2]), v3 = __uint_as_float(ub[c + 3]);
                        q0 = fmaf(v0, v0, q0);
                        q1 = fmaf(v1, v1, q1);
                        q2 = fmaf(v2, v2, q2);
                        q3 = fmaf(v3, v3, q3);
                    }
                    const float v12 = __uint_as_float(ub[12]), v13 = __uint_as_float(ub[13]);
                    const float v14 = __uint_as_float(ub[14]);
                    q0 = fmaf(v12, v12, q0);
                    q1 = fmaf(v13, v13, q1);
                    q2 = fmaf(v14, v14, q2);
                    t = __uint_as_float(ub[15]);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&uempty[u]);
                const float qv = (q0 + q1) + (q2 + q3);
                const unsigned char *dt = dtile + s * C::STAGE_BYTES + (k & 1) * C::TILE_BYTES;
                const float yv = reinterpret_cast<const float *>(dt + C::D_BYTES)[o_r];
                const float e = yv - t;
                const float den = fmaf(erho, qv, 1.0f);
                float inv = rcp_approx(den);
                inv = fmaf(inv, fmaf(-den, inv, 1.0f), inv);
                const float c_ = erho * inv;
                const float ei = e * inv;
                const float w = valid ? c_ * e : 0.0f;
                const float gm = valid ? fmaf(c_ * e, c_ * e, -c_) : 0.0f;
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
                if constexpr (C::TMEM_A2) {
                    // stage this observation's parts of gamma and w for the A2 row builders
                    const bool oka = (k < C::NBUF) || mbar_wait_backoff(&a2empty[b], uint32_t(((k / C::NBUF) - 1) & 1), BUDGET);
                    if (__any_sync(0xffffffffu, !oka)) {
                        *s_abort = 1;
                        break;
                    }
                    __nv_bfloat16 *gb = gam + b * (2 * NSPLIT * C::TILE);
                    {
                        __nv_bfloat16 gp[NSPLIT], wp[NSPLIT];
                        f32_split<NSPLIT>(gm, gp);
                        f32_split<NSPLIT>(w, wp);
#pragma unroll
                        for (int p = 0; p < NSPLIT; ++p) {
                            gb[p * C::TILE + o_r] = gp[p];
                            gb[(NSPLIT + p) * C::TILE + o_r] = wp[p];
                        }
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&staged[b]);
                    const bool oks = mbar_wait_backoff(&staged[b], uint32_t((k / C::NBUF) & 1), BUDGET);
                    if (__any_sync(0xffffffffu, !oks)) {
                        *s_abort = 1;
                        break;
                    }
                    tc_fence_after();                   // after MMA2's reads of A2[b] (a2empty) and the staging
                    // this thread's A2 row: tensor-memory lane 32 q + lane = (set q >> 1, part q & 1,
                    // slot lane); K = the set's 64 observations, two per column.  Slot 31 of the tile
                    // rows is 1, and row (set, part, 31) holds part `part` of w.
                    const uint32_t set = uint32_t(q >> 1), part = uint32_t(q & 1), x = uint32_t(lane);
                    uint32_t row[32];
                    const uint32_t ta2 = tbase + lanebase + C::COL_A2 + C::A2_COLS * uint32_t(b);
                    const __nv_bfloat16 *wsrc = gb + (NSPLIT + part) * C::TILE + 64 * set;
                    if (binary) {                       // warp-uniform: every tensor-memory store below is converged
                        const __nv_bfloat16 *src = (x == 31) ? wsrc : gb + part * C::TILE + 64 * set;
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            if (j == 4) tmem_st16(ta2, row);          // first half on its way
                            // 8 observations 64 set + 8 j ..: D in {-1, 0, 1} (or the constant 1 of slot
                            // 31), so each product is exact in BF16
                            const uint4 dv = *reinterpret_cast<const uint4 *>(dt + tc_slot_byte(64 * set + 8 * j, x));
                            const uint4 gv = *reinterpret_cast<const uint4 *>(src + 8 * j);
                            const __nv_bfloat162 *dp = reinterpret_cast<const __nv_bfloat162 *>(&dv);
                            const __nv_bfloat162 *gq = reinterpret_cast<const __nv_bfloat162 *>(&gv);
#pragma unroll
                            for (int h = 0; h < 4; ++h)
                                reinterpret_cast<__nv_bfloat162 *>(&row[4 * j + h])[0] = __hmul2(gq[h], dp[h]);
                        }
                        tmem_st16(ta2 + 16, row + 16);
                    } else {
                        // general D (exact in BF16): gamma (the sum of its parts) times D_x in FP32,
                        // then part `part` of the product; slot 31 takes part `part` of w as staged
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const uint4 dv = *reinterpret_cast<const uint4 *>(dt + tc_slot_byte(64 * set + 8 * j, x));
                            const uint4 wv = *reinterpret_cast<const uint4 *>(wsrc + 8 * j);
                            const __nv_bfloat162 *dp = reinterpret_cast<const __nv_bfloat162 *>(&dv);
                            const uint32_t *wq = reinterpret_cast<const uint32_t *>(&wv);
                            float g8[8];
#pragma unroll
                            for (int h = 0; h < 8; ++h) g8[h] = 0.0f;
#pragma unroll
                            for (int p = 0; p < NSPLIT; ++p) {
                                const uint4 gv = *reinterpret_cast<const uint4 *>(gb + p * C::TILE + 64 * set + 8 * j);
                                const __nv_bfloat16 *gq = reinterpret_cast<const __nv_bfloat16 *>(&gv);
#pragma unroll
                                for (int h = 0; h < 8; ++h) g8[h] += __bfloat162float(gq[h]);
                            }
#pragma unroll
                            for (int h = 0; h < 4; ++h) {
                                const float2 df = __bfloat1622float2(dp[h]);
                                __nv_bfloat162 pp[NSPLIT];
                                f32x2_split<NSPLIT>(g8[2 * h] * df.x, g8[2 * h + 1] * df.y, pp);
                                uint32_t u0, u1;
                                memcpy(&u0, &pp[0], 4);
                                memcpy(&u1, &pp[1], 4);
                                row[4 * j + h] = (x == 31) ? wq[h] : (part ? u1 : u0);
                            }
                        }
                        tmem_st32(ta2, row);
                    }
                    tmem_wait_st();
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&a2full[b]);
                    continue;
                } else {
                // stage this observation's parts: gamma for the chunk builders, w straight into
                // A2 row (set, p, 31)
                const bool oka = (k < C::NBUF) || mbar_wait_backoff(&a2empty[b], uint32_t(((k / C::NBUF) - 1) & 1), BUDGET);
                if (__any_sync(0xffffffffu, !oka)) {
                    *s_abort = 1;
                    break;
                }
                unsigned char *abuf = a2 + b * C::A2_BYTES;
                __nv_bfloat16 *gb = gam + b * (NSPLIT * C::TILE);
                {
                    __nv_bfloat16 gp[NSPLIT], wp[NSPLIT];
                    f32_split<NSPLIT>(gm, gp);
                    f32_split<NSPLIT>(w, wp);
                    const uint32_t set = (C::SETS == 2) ? (o_r >> 6) : 0u;
#pragma unroll
                    for (int p = 0; p < NSPLIT; ++p) {
                        gb[p * C::TILE + o_r] = gp[p];
                        *reinterpret_cast<__nv_bfloat16 *>(abuf + a2_byte<C::SETS>(64 * set + 32 * p + 31, o_r)) = wp[p];
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&staged[b]);
                const bool oks = mbar_wait_backoff(&staged[b], uint32_t((k / C::NBUF) & 1), BUDGET);
                if (__any_sync(0xffffffffu, !oks)) {
                    *s_abort = 1;
                    break;
                }
                // A2 chunks: slot x < 31 of 8 observations (pairs) -> part p of gamma D_x; each
                // thread takes up to TPT chunks, loading all operands before the products
                if (binary) {
                    uint4 dch[TPT], gch[TPT][NSPLIT];
#pragma unroll
                    for (int i = 0; i < TPT; ++i) {
                        if (gt + 128 * i < C::NTASK) {
                            const uint32_t pk = tpk[i], o0 = (pk >> 28) << 3;
                            dch[i] = *reinterpret_cast<const uint4 *>(dt + (pk & 0x1FFFu));
#pragma unroll
                            for (int p = 0; p < NSPLIT; ++p)
                                gch[i][p] = *reinterpret_cast<const uint4 *>(gb + p * C::TILE + o0);
                        }
                    }
#pragma unroll
                    for (int i = 0; i < TPT; ++i) {
                        if (gt + 128 * i < C::NTASK) {
                            unsigned char *dst = abuf + ((tpk[i] >> 13) & 0x7FFFu);
                            const __nv_bfloat162 *dp = reinterpret_cast<const __nv_bfloat162 *>(&dch[i]);
#pragma unroll
                            for (int p = 0; p < NSPLIT; ++p) {
                                // D in {-1, 0, 1}: each part of gamma times D is exact in BF16
                                const __nv_bfloat162 *gq = reinterpret_cast<const __nv_bfloat162 *>(&gch[i][p]);
                                uint4 o;
                                __nv_bfloat162 *op = reinterpret_cast<__nv_bfloat162 *>(&o);
#pragma unroll
                                for (int h = 0; h < 4; ++h) op[h] = __hmul2(gq[h], dp[h]);
                                *reinterpret_cast<uint4 *>(dst + 2048 * p) = o;
                            }
                        }
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < TPT; ++i) {
                        if (gt + 128 * i >= C::NTASK) continue;
                        const uint32_t pk = tpk[i], o0 = (pk >> 28) << 3;
                        unsigned char *dst = abuf + ((pk >> 13) & 0x7FFFu);
                        const uint4 dch = *reinterpret_cast<const uint4 *>(dt + (pk & 0x1FFFu));
                        const __nv_bfloat162 *dp = reinterpret_cast<const __nv_bfloat162 *>(&dch);
                        // general D (exact in BF16): gamma (the sum of its parts) times D_x in FP32,
                        // then the parts of the product
                        float gsum8[8];
#pragma unroll
                        for (int h = 0; h < 8; ++h) gsum8[h] = 0.0f;
#pragma unroll
                        for (int p = 0; p < NSPLIT; ++p) {
                            const uint4 gch = *reinterpret_cast<const uint4 *>(gb + p * C::TILE + o0);
                            const __nv_bfloat16 *gq = reinterpret_cast<const __nv_bfloat16 *>(&gch);
#pragma unroll
                            for (int h = 0; h < 8; ++h) gsum8[h] += __bfloat162float(gq[h]);
                        }
                        uint4 o[NSPLIT];
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            const float2 df = __bfloat1622float2(dp[h]);
                            __nv_bfloat162 pp[NSPLIT];
                            f32x2_split<NSPLIT>(gsum8[2 * h] * df.x, gsum8[2 * h + 1] * df.y, pp);
#pragma unroll
                            for (int p = 0; p < NSPLIT; ++p) reinterpret_cast<__nv_bfloat162 *>(&o[p])[h] = pp[p];
                        }
#pragma unroll
                        for (int p = 0; p < NSPLIT; ++p) *reinterpret_cast<uint4 *>(dst + 2048 * p) = o[p];
                    }
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&a2full[b]);
                }
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
    // G''(m, y) as sum - comp; G(x, y) sums rows (set, part, x), g(y) rows (set, part, 31)
    auto gval = [&](int m, int y) {
        return static_cast<double>(gsum[y * 128 + m]) - static_cast<double>(gcmp[y * 128 + m]);
    };
    auto Gsum = [&](int x, int y) {
        double v = 0.0;
#pragma unroll
        for (int set = 0; set < C::SETS; ++set)
#pragma unroll
            for (int p = 0; p < NSPLIT; ++p) v += gval(64 * set + 32 * p + x, y);
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
            v = Gsum(r, c);
        } else if (j < NG + M) {
            v = Gsum(31, j - NG);
        } else {
            const int which = j - NG - M;                                  // T3, T4, E4
            for (int t = 0; t < 32 * C::NCW; ++t) v += red[3 * t + which];
        }
        part[j] = v;
    }
    int row0, nrows;
    if (!finish_ticket(st, a.partials, gridDim.x, NSTAT, s_last, &row0, &nrows, reinterpret_cast<double *>(base)))
        return;
    if (run && st->status == ST_OK) {
        global_update_rt(M, st, a.partials + size_t(row0) * NSTAT, nrows, a, reinterpret_cast<double *>(base));
    } else if (tid == 0 && a.use_cond) {
        cudaGraphSetConditional(a.cond, 0u);
    }
}

// Inputs of the tensor-core sweep, repacked into tiles of 128 observations
// (TC_TILE_BYTES each; an even number of tiles) in the basis of Eq. 3: the
// BF16 slots D_ij = d_ij - d_iS (j < M), 0 (M <= j < 31) and 1 (j = 31) in the
// slot-major layout of tc_slot_byte, then y_i = r_i - d_iS (FP32).  Rows past V
// are zero.  counts[0] += D values that BF16 does not represent exactly,
// counts[1] += D values other than -1, 0, 1.  One thread per (8 observations,
// slot).
__global__ void tc_inputs_kernel(const float *__restrict__ d, const float *__restrict__ r, long long V, int S,
                                 long long ntiles, unsigned char *__restrict__ out, unsigned long long *counts)
{
    unsigned long long bad = 0, nonunit = 0;
    const int M = S - 1;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ntiles * 16 * 32; i += stride) {
        const int x = int(i & 31);
        const long long oct = i >> 5;                                  // global octet of observations
        const long long o0 = oct * 8;
        unsigned char *tile = out + (o0 >> 7) * (long long)TC_TILE_BYTES;
        const uint32_t ot = uint32_t(o0 & 127);
        __align__(16) __nv_bfloat16 b[8];
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            const long long o = o0 + h;
            float v = 0.0f;
            if (o < V) {
                const float dS = d[o * S + M];
                if (x < M) {
                    v = d[o * S + x] - dS;
                    if (v != 0.0f && v != 1.0f && v != -1.0f) ++nonunit;
                } else if (x == 31) {
                    v = 1.0f;
                }
                if (x == 0) reinterpret_cast<float *>(tile + 128 * 64)[ot + h] = r[o] - dS;
            } else if (x == 0) {
                reinterpret_cast<float *>(tile + 128 * 64)[ot + h] = 0.0f;
            }
            b[h] = __float2bfloat16_rn(v);
            if (__bfloat162float(b[h]) != v) ++bad;
        }
        *reinterpret_cast<uint4 *>(tile + tc_slot_byte(ot, uint32_t(x))) = *reinterpret_cast<const uint4 *>(b);
    }
    if (bad) atomicAdd(&counts[0], bad);
    if (nonunit) atomicAdd(&counts[1], nonunit);
}

} // namespace vbh
