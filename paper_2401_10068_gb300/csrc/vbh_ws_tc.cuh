// vbh_ws_tc.cuh -- the contractions of the learned warm start's set encoder
// on the tcgen05 tensor cores: C = A B^T with BF16 operands and FP32
// accumulation in tensor memory, and epilogues that apply the encoder's
// elementwise steps to the accumulator before anything goes back to memory.
//
// Operand layout ("tile layout").  A matrix X with `rows` rows and `cols`
// columns (cols a multiple of 32) is stored as blocks of RB rows x 32 columns,
// block (rb, a) at element offset (rb * cols / 32 + a) * RB * 32; inside a
// block row r occupies 64 bytes and its 16-byte chunk c (columns 8c .. 8c+7)
// sits at chunk position c ^ ((r >> 1) & 3) (the 64-byte swizzle of the MMA's
// shared-memory descriptors).  One block of the A operand (RB = 128) and one
// of the B operand (RB = the N tile) are each one contiguous bulk copy, and a
// 32-column step of K is two MMAs of K = 16 on them.  The epilogues write the
// encoder's activations directly in this layout, in the orientation the next
// contraction needs: K-major (rows = observations) for the next layer, and
// transposed (rows = features, columns = observations) for the weight
// gradients, whose K is the observation index.
//
// Roles (12 warps, one persistent block per SM): lane 0 of warp 0 issues the
// bulk copies into a 4-stage ring, lane 0 of warp 1 issues the MMAs of one
// output tile (128 rows x NT columns, FP32) into one of two tensor-memory
// accumulators while the epilogue drains the other, warp 2 allocates and
// frees the tensor memory, and warps 4-11 run the epilogue: warp 4 + e reads
// tensor-memory lanes 32 (e % 4) .. + 31 (rows of the tile) and columns of
// half e / 4.  Every wait is bounded; on a timeout the block records the
// failure in *err, lets its copies and MMAs drain and skips its writes.
#pragma once

#include <cuda_bf16.h>

#include "vbh_internal.cuh"

namespace vbh {

// Element offset of (row, col) in the tile layout (cols columns, row blocks of RB).
__host__ __device__ __forceinline__ long long tl_index(long long row, int col, long long cols, int RB)
{
    const long long rb = row / RB;
    const int r = int(row - rb * RB), a = col >> 5, c = col & 31;
    const long long block = (rb * (cols >> 5) + a) * (long long)RB * 32;
    return block + r * 32 + ((((c >> 3) ^ ((r >> 1) & 3)) << 3) | (c & 7));
}

// GELU in the tanh form, z (1 + tanh(k0 (z + k1 z^3))) / 2 (Hendrycks and
// Gimpel, 2016), evaluated as z sigma(2 k0 (z + k1 z^3)) with sigma(x) = 1 /
// (1 + e^{-x}) (the same function: (1 + tanh(x/2)) / 2 = sigma(x)), one
// exponential and one approximate reciprocal; and its derivative
// sigma + z sigma (1 - sigma) 2 k0 (1 + 3 k1 z^2).
constexpr float WS_K0 = 0.7978845608028654f, WS_K1 = 0.044715f;
constexpr float WS_NEG2K0_LOG2E = -2.0f * 0.7978845608028654f * 1.4426950408889634f;

__device__ __forceinline__ float ws_ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float ws_rcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float ws_sigma2(float z)
{
    // sigma(2 k0 (z + k1 z^3)); the exponent is clamped so that 1 + e stays finite
    const float w = fmaf(WS_K1 * z * z, z, z);
    return ws_rcp(1.0f + ws_ex2(fminf(WS_NEG2K0_LOG2E * w, 126.0f)));
}

__device__ __forceinline__ float ws_gelu(float z) { return z * ws_sigma2(z); }

__device__ __forceinline__ float ws_gelu_grad(float z)
{
    const float sg = ws_sigma2(z);
    return fmaf(z * sg * (1.0f - sg), 2.0f * WS_K0 * fmaf(3.0f * WS_K1, z * z, 1.0f), sg);
}

enum WsEpi : int {
    EPI_PLAIN = 0,   // out[split][m][n] = acc (+ bias[n])
    EPI_FWD = 1,     // z = acc + bias; a = GELU(z): Z (FP32 rows), A (K-major), A^T, column sums of a
    EPI_DZ2 = 2,     // z = acc + bias (layer 2 again); dz = dpool[set] / count[set] * GELU'(z): dZ (K-major), dZ^T,
                     // column sums of dz
    EPI_BWD = 3,     // dz = acc * GELU'(Zin): dZ^T, column sums of dz
};

struct WsGemmArgs {
    const __nv_bfloat16 *A;        // tile layout, RB = 128, cols = K
    const __nv_bfloat16 *B;        // tile layout, RB = NT, cols = K
    int M, N, K;                   // M % 128 == 0, N % NT == 0, K % 32 == 0
    int kchunk;                    // K per split (blockIdx.z), a multiple of 32
    const float *bias;             // [N] or null
    float *out;                    // EPI_PLAIN: [splits][M][N]
    float *Z;                      // EPI_FWD: pre-activations [M][N] (optional)
    __nv_bfloat16 *Aout;           // EPI_FWD / EPI_DZ2: tile layout RB = 128, cols = N (optional)
    __nv_bfloat16 *ATout;          // transposed: tile layout RB = rbt, rows = N, cols = Mt (optional)
    int rbt;
    long long Mt;
    float *colsum;                 // [M / 128][N] sums over the valid rows of each row tile (optional)
    const int *valid;              // [M / 128] valid rows per row tile (null: 128)
    const int *tile_set;           // EPI_DZ2: set of each row tile
    const float *dpool;            // EPI_DZ2: [sets][N]
    const float *inv_count;        // EPI_DZ2: [sets] 1 / observations pooled
    const float *Zin;              // EPI_BWD: [M][N] pre-activations of the forward pass
    int *err;                      // set to ST_ETIMEOUT by a block whose wait ran out
};

template <int NT>
struct WsGemmCfg {
    static constexpr int STAGES = 4;
    static constexpr int THREADS = 384;               // warps 0-3: copies, MMAs, tensor memory; 4-11: epilogue
    static constexpr int EPI_WARPS = 8;
    static constexpr uint32_t A_BYTES = 128u * 64u, B_BYTES = uint32_t(NT) * 64u;
    static constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr uint32_t TMEM_COLS = 2 * NT;     // two accumulators: the MMAs of a tile overlap the
                                                      // epilogue of the one before
    static constexpr size_t SMEM_BYTES = size_t(STAGES) * STAGE_BYTES + 1024 /* alignment */ + 256 /* barriers */;
    static_assert((2 * STAGES + 7) * 8 <= 256, "mbarrier slots");
    static_assert(NT == 64 || NT == 128 || NT == 256, "N tile");
};

// Column sums over the 32 rows of a warp: a butterfly reduce-scatter leaves
// lane l with the sum of column l of the 32 values each lane holds.
__device__ __forceinline__ float warp_colsum32(float (&v)[32], int lane)
{
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
    return v[0];
}

// Store the 32 BF16 values of row `row` (columns n0 .. n0 + 31) into a K-major
// tile-layout matrix with `cols` columns: four 16-byte chunks at their
// swizzled positions.
__device__ __forceinline__ void store_row32_bf16(__nv_bfloat16 *dst, long long row, int n0, long long cols,
                                                 const float (&v)[32])
{
    const long long rb = row >> 7;
    const int r = int(row & 127);
    __nv_bfloat16 *blk = dst + (rb * (cols >> 5) + (n0 >> 5)) * 128 * 32 + r * 32;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uint4 w;
        __nv_bfloat162 p0 = __floats2bfloat162_rn(v[8 * c + 0], v[8 * c + 1]);
        __nv_bfloat162 p1 = __floats2bfloat162_rn(v[8 * c + 2], v[8 * c + 3]);
        __nv_bfloat162 p2 = __floats2bfloat162_rn(v[8 * c + 4], v[8 * c + 5]);
        __nv_bfloat162 p3 = __floats2bfloat162_rn(v[8 * c + 6], v[8 * c + 7]);
        w.x = *reinterpret_cast<uint32_t *>(&p0);
        w.y = *reinterpret_cast<uint32_t *>(&p1);
        w.z = *reinterpret_cast<uint32_t *>(&p2);
        w.w = *reinterpret_cast<uint32_t *>(&p3);
        *reinterpret_cast<uint4 *>(blk + ((c ^ ((r >> 1) & 3)) << 3)) = w;
    }
}

__device__ __forceinline__ void ws_named_sync(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Persistent: block b takes work items b, b + gridDim.x, ... (an item is one
// output tile of one split); the producer and the MMA issuer run ahead across
// items through the stage ring and the two accumulators.
template <int NT, int EPI>
__global__ void __launch_bounds__(WsGemmCfg<NT>::THREADS, 1) ws_gemm_kernel(WsGemmArgs g)
{
    using C = WsGemmCfg<NT>;
    constexpr int STAGES = C::STAGES;
    extern __shared__ unsigned char ws_smem_raw[];
    // stages on 1024-byte boundaries of the shared address space (the swizzle atoms)
    unsigned char *smem = ws_smem_raw + ((1024u - (smem_addr(ws_smem_raw) & 1023u)) & 1023u);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * C::STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;        // [2] accumulator ready for the epilogue
    uint64_t *tempty = tfull + 2;            // [2] accumulator drained by the epilogue
    uint64_t *drain = tempty + 2;            // the MMAs issued have completed
    uint64_t *csready = drain + 1;           // [2] every epilogue warp has written its column sums
    __shared__ uint32_t s_tmem;
    __shared__ int s_bad, s_issued, s_consumed;
    __shared__ float s_cs[2][4][NT];
    __shared__ __align__(16) float s_bias[256];        // the bias of the N range (N <= 256 where one is given)

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int MT = g.M / 128, NTT = g.N / NT;
    const int nsplit = (g.K + g.kchunk - 1) / g.kchunk;
    const long long items = (long long)MT * NTT * nsplit;
    const long long kblocks = g.K >> 5;
    constexpr uint64_t BUDGET = 2000000000ull;
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], C::EPI_WARPS);
            mbar_init(&csready[a], C::EPI_WARPS);
        }
        mbar_init(drain, 1);
        fence_mbar_init();
        s_bad = 0;
        s_issued = 0;
        s_consumed = 0;
    }
    if (warp == 2) tmem_alloc<C::TMEM_COLS>(&s_tmem);
    for (int n = tid; n < 256; n += C::THREADS) s_bias[n] = (g.bias && n < g.N) ? g.bias[n] : 0.0f;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = s_tmem;

    auto item_of = [&](long long it, int &tm, int &tn, int &split) {
        tm = int(it % MT);
        tn = int((it / MT) % NTT);
        split = int(it / ((long long)MT * NTT));
    };

    if (warp == 0 && lane == 0) {
        // producer: A block (tm, a) and B block (tn, a) per 32-column step, over all items
        int cnt = 0;
        for (long long it = blockIdx.x; it < items && !s_bad; it += gridDim.x) {
            int tm, tn, split;
            item_of(it, tm, tn, split);
            const int k0 = split * g.kchunk, k1 = min(g.K, k0 + g.kchunk);
            for (int kb = 0; kb < (k1 - k0) >> 5; ++kb, ++cnt) {
                const int s = cnt % STAGES;
                if (cnt >= STAGES && !mbar_wait_bounded(&empty[s], uint32_t(((cnt / STAGES) - 1) & 1), BUDGET)) {
                    atomicExch(&s_bad, 1);
                    break;
                }
                const long long a = (k0 >> 5) + kb;
                unsigned char *st = smem + size_t(s) * C::STAGE_BYTES;
                mbar_arrive_expect_tx(&full[s], C::STAGE_BYTES);
                bulk_load(st, g.A + (tm * kblocks + a) * 128 * 32, C::A_BYTES, &full[s]);
                bulk_load(st + C::A_BYTES, g.B + (tn * kblocks + a) * (long long)NT * 32, C::B_BYTES, &full[s]);
                s_issued = cnt + 1;
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issue: D[acc] (128 x NT, FP32) += A_tile (128 x 32) B_tile (NT x 32)^T per step
        constexpr uint32_t IDESC = umma_idesc_bf16(128, NT, 0, 0);
        int cnt = 0, li = 0;
        for (long long it = blockIdx.x; it < items && !s_bad; it += gridDim.x, ++li) {
            int tm, tn, split;
            item_of(it, tm, tn, split);
            const int k0 = split * g.kchunk, k1 = min(g.K, k0 + g.kchunk);
            const int acc = li & 1;
            if (li >= 2 && !mbar_wait_bounded(&tempty[acc], uint32_t(((li >> 1) - 1) & 1), BUDGET)) {
                atomicExch(&s_bad, 1);
                break;
            }
            tc_fence_after();
            const uint32_t td = tbase + uint32_t(acc * NT);
            bool ok = true;
            for (int kb = 0; kb < (k1 - k0) >> 5; ++kb, ++cnt) {
                const int s = cnt % STAGES;
                if (!mbar_wait_bounded(&full[s], uint32_t((cnt / STAGES) & 1), BUDGET)) {
                    atomicExch(&s_bad, 1);
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t sa = smem_addr(smem + size_t(s) * C::STAGE_BYTES);
                const uint32_t sb = sa + C::A_BYTES;
#pragma unroll
                for (int kk = 0; kk < 2; ++kk)
                    umma_bf16(td, umma_desc(sa + kk * 32, 16, 512, 4), umma_desc(sb + kk * 32, 16, 512, 4), IDESC,
                              (kb | kk) ? 1u : 0u);
                umma_commit(&empty[s]);
                s_consumed = cnt + 1;
            }
            if (!ok) break;
            umma_commit(&tfull[acc]);
        }
        umma_commit(drain);                      // after every MMA issued above (also on a timeout)
        (void)mbar_wait_bounded(drain, 0u, BUDGET);
    } else if (warp >= 4) {
        const int ew = warp - 4, q = ew & 3, half = ew >> 2;   // lane quarter q, column half
        const int row = q * 32 + lane;
        int li = 0;
        for (long long it = blockIdx.x; it < items; it += gridDim.x, ++li) {
            int tm, tn, split;
            item_of(it, tm, tn, split);
            const int acc = li & 1;
            const bool okw = mbar_wait_backoff(&tfull[acc], uint32_t((li >> 1) & 1), 2 * BUDGET);
            if (__any_sync(0xffffffffu, !okw)) {
                atomicExch(&s_bad, 1);
                break;
            }
            tc_fence_after();
            const long long m = (long long)tm * 128 + row;
            const bool good = !s_bad;
            const int nvalid = g.valid ? g.valid[tm] : 128;
            const bool vrow = row < nvalid;
            int set = 0;
            float dps = 0.0f;
            if constexpr (EPI == EPI_DZ2) {
                set = g.tile_set[tm];
                dps = g.inv_count[set];
            }
#pragma unroll 1
            for (int c0 = half * (NT / 2); c0 < (half + 1) * (NT / 2); c0 += 32) {
                float v[32];
                tmem_ld32(tbase + uint32_t(acc * NT) + (uint32_t(q * 32) << 16) + uint32_t(c0), v);
                const int n0 = tn * NT + c0;
                const float4 *bq = reinterpret_cast<const float4 *>(s_bias + n0);
                if constexpr (EPI == EPI_PLAIN) {
                    if (!good) continue;
                    float *o = g.out + ((size_t)split * g.M + m) * g.N + n0;
#pragma unroll
                    for (int j = 0; j < 32; j += 4) {
                        const float4 bb = bq[j / 4];
                        *reinterpret_cast<float4 *>(o + j) =
                            make_float4(v[j] + bb.x, v[j + 1] + bb.y, v[j + 2] + bb.z, v[j + 3] + bb.w);
                    }
                } else {
                    float a[32];
                    if constexpr (EPI != EPI_BWD) {
#pragma unroll
                        for (int j = 0; j < 32; j += 4) {           // v = z
                            const float4 bb = bq[j / 4];
                            v[j] += bb.x;
                            v[j + 1] += bb.y;
                            v[j + 2] += bb.z;
                            v[j + 3] += bb.w;
                        }
                    }
                    if constexpr (EPI == EPI_FWD) {
                        if (g.Z && good) {
                            float *o = g.Z + (size_t)m * g.N + n0;
#pragma unroll
                            for (int j = 0; j < 32; j += 4)
                                *reinterpret_cast<float4 *>(o + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                        }
#pragma unroll
                        for (int j = 0; j < 32; ++j) a[j] = vrow ? ws_gelu(v[j]) : 0.0f;
                    } else if constexpr (EPI == EPI_DZ2) {
                        const float *dp = g.dpool + (size_t)set * g.N + n0;
#pragma unroll
                        for (int j = 0; j < 32; ++j) a[j] = vrow ? dp[j] * dps * ws_gelu_grad(v[j]) : 0.0f;
                    } else {                                        // EPI_BWD
                        const float *zi = g.Zin + (size_t)m * g.N + n0;
#pragma unroll
                        for (int j = 0; j < 32; j += 4) {
                            const float4 zz = *reinterpret_cast<const float4 *>(zi + j);
                            a[j] = vrow ? v[j] * ws_gelu_grad(zz.x) : 0.0f;
                            a[j + 1] = vrow ? v[j + 1] * ws_gelu_grad(zz.y) : 0.0f;
                            a[j + 2] = vrow ? v[j + 2] * ws_gelu_grad(zz.z) : 0.0f;
                            a[j + 3] = vrow ? v[j + 3] * ws_gelu_grad(zz.w) : 0.0f;
                        }
                    }
                    if (g.colsum && EPI == EPI_FWD) {
                        // the forward pool sums the FP32 activations (a copy: the butterfly consumes it)
                        float cs[32];
#pragma unroll
                        for (int j = 0; j < 32; ++j) cs[j] = a[j];
                        s_cs[acc][q][c0 + lane] = warp_colsum32(cs, lane);
                    }
                    if (g.Aout || g.ATout || (g.colsum && EPI != EPI_FWD)) {
                        // the BF16 values the next contraction reads; the backward column sums
                        // (bias gradients) take the same rounded values
#pragma unroll
                        for (int j = 0; j < 32; ++j) a[j] = __bfloat162float(__float2bfloat16_rn(a[j]));
                        if (g.Aout && good) store_row32_bf16(g.Aout, m, n0, g.N, a);
                        if (g.ATout && good) {
                            // column m of the transposed matrix: rows n0 .. n0 + 31 of one row block
                            const long long rb = n0 / g.rbt;
                            const int r0 = n0 - int(rb) * g.rbt, cc = int(m & 31);
                            __nv_bfloat16 *blk = g.ATout + (rb * (g.Mt >> 5) + (m >> 5)) * (long long)g.rbt * 32;
#pragma unroll
                            for (int j = 0; j < 32; ++j) {
                                const int r = r0 + j;
                                blk[r * 32 + ((((cc >> 3) ^ ((r >> 1) & 3)) << 3) | (cc & 7))] = __float2bfloat16_rn(a[j]);
                            }
                        }
                        if (g.colsum && EPI != EPI_FWD) s_cs[acc][q][c0 + lane] = warp_colsum32(a, lane);
                    }
                }
            }
            // this accumulator may take the next MMAs
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[acc]);
            if constexpr (EPI != EPI_PLAIN) {
                if (g.colsum) {
                    // every epilogue warp's column sums are in s_cs[acc] (a bounded wait: a
                    // named barrier could not give up); the buffer is written again two items
                    // later, after every warp has passed this item's wait
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&csready[acc]);
                    const bool okc = mbar_wait_bounded(&csready[acc], uint32_t((li >> 1) & 1), BUDGET);
                    if (__any_sync(0xffffffffu, !okc)) {
                        atomicExch(&s_bad, 1);
                        break;
                    }
                    for (int n = tid - 128; n < NT; n += 32 * C::EPI_WARPS)
                        if (good)
                            g.colsum[(size_t)tm * g.N + tn * NT + n] =
                                (s_cs[acc][0][n] + s_cs[acc][1][n]) + (s_cs[acc][2][n] + s_cs[acc][3][n]);
                }
            }
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 0 && lane == 0 && s_bad) {
        // a wait ran out: let the copies issued but not consumed land before the block exits
        for (int kb = s_consumed; kb < s_issued; ++kb)
            (void)mbar_wait_bounded(&full[kb % STAGES], uint32_t((kb / STAGES) & 1), 100000000ull);
    }
    if (tid == 0 && s_bad && g.err) atomicExch(g.err, ST_ETIMEOUT);
    if (warp == 2) {
        tc_fence_after();
        tmem_dealloc<C::TMEM_COLS>(tbase);
    }
}

} // namespace vbh
