// vbh_internal.cuh -- device-side state and helpers shared by the kernels of
// libvbh (the CUDA path).  Nothing here is used by the CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vbh {

constexpr int MMAX = 31;             // largest M = S - 1
// Block partials are reduced in one level up to TICKET_SINGLE_MAX blocks (the
// block that finishes the launch sums all rows) and in two levels above: the
// last block of each group of TICKET_GROUP consecutive blocks sums the group's
// rows, the last group's reducer runs the global update over the group sums.
constexpr int TICKET_SINGLE_MAX = 128;
constexpr int TICKET_GROUP = 32;
constexpr int TICKET_GROUPS_MAX = 40;
constexpr int GRID_MAX = TICKET_GROUP * TICKET_GROUPS_MAX;  // largest sweep grid
// rows of the partials buffer for a grid of nblk blocks: one per block, then one per group
__host__ __device__ constexpr long long partial_rows(long long nblk)
{
    return nblk <= TICKET_SINGLE_MAX ? nblk : nblk + (nblk + TICKET_GROUP - 1) / TICKET_GROUP;
}
constexpr int SMAX = 32;
constexpr int S_FP32_MAX = 11;       // largest S of the register-resident FP32 sweep

// Launch modes of the fused sweep kernel.
enum SweepMode : int {
    MODE_INIT = 0,   // sweep 0: Q(beta_i) = N(K0, Lambda_0^{-1}); then Q(rho), Q(K,Lambda), ELBO
    MODE_ITER = 1,   // Q(beta) (Eq. 19-21) -> Q(rho) (Eq. 16-18) -> Q(K,Lambda) (Eq. 22-25) -> ELBO
    MODE_ELBO = 2,   // Q(beta) from the current globals, ELBO only, no global update
};

// Status codes (same values as the public header).
enum : int { ST_OK = 0, ST_ENONFINITE = -4, ST_ETIMEOUT = -5 };

constexpr int NG_COMP_MAX = (S_FP32_MAX - 1) * S_FP32_MAX / 2;   // packed entries of Sigma0 at S <= 11

// What one data pass reads: the FP32 form of Sigma0 = W^{-1}/nu (its packed
// lower Cholesky factor, row i at offset i(i+1)/2), kappa and E[rho].  For
// the compensated statistics (S <= 11) also Sigma0~ = L~ L~^T, off-diagonal
// entries doubled, and kappa~, each split into a part on a coarse grid
// (Sh, kh) and the rest (Sl, kl), so that for profiles with entries in
// {0, 1} the sums of the grid parts over D_j D_k (or D_j) are exact in FP32.
struct SweepGlobalsF32 {
    float L[MMAX * (MMAX + 1) / 2];
    float kappa[MMAX];
    float erho;
    int pad;
    float Sh[NG_COMP_MAX], Sl[NG_COMP_MAX];
    float kh[S_FP32_MAX - 1], kl[S_FP32_MAX - 1];
};

// Functions of (a_rho, nu, lambda) that the ELBO needs.  In a fit these are
// fixed by V (Eq. 16, 22, 23), so they are evaluated once per fit by the
// set-up kernel instead of once per sweep.
struct ElboConst {
    double a_rho, nu, lam;
    double lgamma_a, psi_a;          // lnGamma(a_rho), psi(a_rho)
    double sum_psi_nu;               // sum_{j=1..M} psi((nu + 1 - j)/2)
    double sum_lgamma_nu;            // sum_{j=1..M} lnGamma((nu + 1 - j)/2)
    double log_lam;
    double log_nu, rs_nu;            // ln nu, 1/sqrt(nu)
    double inv_lam, inv_V;           // 1/lambda, 1/V (0 when V = 0)
    // the ELBO of Eq. 11 as an affine function of what a sweep changes:
    //   L = e0 + e_logb ln b_rho - e_ldw ln|W^{-1}| - tr(E[Lambda] X)/2 - T4/2
    //       + V ln|Sigma0~|/2 - E[rho] (b0 + T3/2)
    // (X = C + Lambda_0^{-1} + q0 (kappa - K0)(kappa - K0)^T, C as in the update)
    double e0, e_logb, e_ldw;
};

// FP64 state of one fit, resident in device memory.
struct DevState {
    // prior, Eq. 5-7
    int S, M;
    double V;
    double q0, n0, a0, b0;
    double lndetL0inv;
    double K0[MMAX];
    double L0inv[MMAX * MMAX];
    // global factors: Q(rho) = Gamma(a_rho, b_rho); Q(K, Lambda) = N(kappa, (lam Lambda)^-1) Wish(W, nu)
    double a_rho, b_rho, nu, lam;
    double kappa[MMAX];
    double Winv[MMAX * MMAX];
    // the Q(beta)-defining quantities of the next data pass
    double Sigma0[MMAX * MMAX];      // E[Lambda]^{-1} = W^{-1} / nu
    double lndetSigma0;
    double erho;                     // E[rho], Eq. 29
    // lower bound and control
    double elbo, elbo_prev, tol;
    int iter, target, max_iter, converged, status, const_dropped;
    unsigned int ticket;             // last-block-done counter of a sweep launch
    unsigned int gticket[TICKET_GROUPS_MAX];   // per-group counters of the two-level reduction
    int em;                          // 1: expectation maximisation (Eq. 42-47) instead of CAVI
    int comp;                        // 1: the data pass adds the compensated statistics U and T4 (one more
                                     //    column of partials) and the ELBO takes their first-order correction
    double *trace;                   // device array [max_iter + 1] (may be null)
    // per-fit constants: kc_upd for (a0 + V/2, n0 + V, q0 + V), kc_given for
    // the factors a fit or vbh_elbo starts from; prior_const collects the
    // prior-only terms of the ELBO (dropping ln B(Lambda_0, n0) when improper)
    ElboConst kc_upd, kc_given;
    double prior_const;
    int prior_dropped, pad1;
    SweepGlobalsF32 sw;
    // ln|W^{-1}| and the Cholesky pivots of W^{-1} behind the current pass
    // factors (S <= 11), left by the last update for the resident loop's ELBO
    // of the next sweep; carry_ok = 0 after a set-up (the factors were given)
    double carry_ldw;
    double carry_piv[S_FP32_MAX - 1];
    int carry_ok, pad2;
};

// Arguments of one launch of the fused sweep kernel.
struct SweepArgs {
    const float *r;
    const float *d;
    long long V;
    DevState *st;
    double *partials;                 // [gridDim.x][statistics per block]
    cudaGraphConditionalHandle cond;  // while-loop condition of the sweep graph
    int use_cond;
    int mode;
};

// Arguments of the resident sweep loop (every sweep of a step in one
// cooperative launch, the observations held in shared memory).
struct ResidentArgs {
    const float *r;
    const float *d;
    long long V;
    DevState *st;        // the fit's state (block 0)
    DevState *priv;      // [gridDim.x - 1] private state copies (blocks 1 ..)
    double *partials;    // [2][gridDim.x][statistics per block], zero at launch
    int per_block;       // observations of every block but the last (a multiple of 4)
};

// ---------------------------------------------------------------------------
// mbarrier / bulk-copy (TMA) helpers, PTX ISA 8.x forms valid on sm_100+.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of an mbarrier, giving up after budget_ns of wall
// time (or 2^28 polls).  Returns false on timeout; never traps.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t budget_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1; it < (1u << 28); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 31u) == 0 && global_ns() - t0 > budget_ns) return false;
    }
    return false;
}

// Same wait with a short sleep between polls, for warps that may wait long
// (keeps the polling traffic off the shared-memory barrier unit).
__device__ __forceinline__ bool mbar_wait_backoff(uint64_t *bar, uint32_t parity, uint64_t budget_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1; it < (1u << 28); ++it) {
        __nanosleep(64);
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 15u) == 0 && global_ns() - t0 > budget_ns) return false;
    }
    return false;
}

// 1-D bulk copy global -> shared memory, completing on an mbarrier.  Both
// addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src_gmem, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// ---------------------------------------------------------------------------
// Tensor-memory (tcgen05) helpers.
// ---------------------------------------------------------------------------
// Shared-memory matrix descriptor of tcgen05.mma: start address, leading and
// stride byte offsets (16-byte units), descriptor version 1, layout (0 none,
// 2 = 128-byte swizzle, 4 = 64-byte swizzle).  K-major swizzled operands use
// SBO = bytes between 8-row groups; MN-major ones use LBO = bytes between
// 64-element (128-byte swizzle) atoms along M/N and SBO = bytes between
// 8-row groups along K.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t layout)
{
    uint64_t d = 0;
    d |= uint64_t((saddr & 0x3FFFFu) >> 4);
    d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
    d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
    d |= uint64_t(1) << 46;
    d |= uint64_t(layout & 7u) << 61;
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: BF16 A and B, FP32 D,
// operand majors (0 = K-major, 1 = MN-major), shape M x N.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N, int a_mn, int b_mn)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(a_mn) << 15) | (uint32_t(b_mn) << 16) |
           (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// Same MMA with the A operand in tensor memory (M rows = TMEM lanes, K
// elements two per 32-bit column, starting at column tmem_a).
__device__ __forceinline__ void umma_bf16_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t idesc,
                                             uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem_d),
        "r"(tmem_a), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <int NCOLS>
__device__ __forceinline__ void tmem_alloc(uint32_t *slot)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "n"(NCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

template <int NCOLS>
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "n"(NCOLS));
}

// 32 consecutive FP32 columns of this thread's TMEM lane (32x32b shape, x32);
// the wait is in the same statement, so no use of the registers can be
// scheduled before the load has completed.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                   "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                   "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 4 consecutive FP32 columns (x4), load and wait in one statement.
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4])
{
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive FP32 columns at taddr and one column at taddr1, one wait for both.
__device__ __forceinline__ void tmem_ld32_1(uint32_t taddr, float (&v)[32], uint32_t taddr1, float &x)
{
    uint32_t r[32], r1;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%33];\n\t"
                 "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%32}, [%34];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                   "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                   "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r1)
                 : "r"(taddr), "r"(taddr1));
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
    x = __uint_as_float(r1);
}

// 32 consecutive 32-bit columns of this thread's TMEM lane from registers
// (32x32b shape, x32); tmem_wait_st must follow before the columns are used.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
                 "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
                 "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
                 "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
                 "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
                 "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
                 : "memory");
}

// 16 consecutive 32-bit columns (x16), no wait.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t *r)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
                     taddr),
                 "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
                 "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Loads without the wait (tcgen05.wait::ld must follow before the registers are used).
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                   "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                   "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld4_nowait(uint32_t taddr, uint32_t (&r)[4])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
}

// The wait for the loads above; the registers are passed through so that no use
// can be scheduled before it.
template <int N>
__device__ __forceinline__ void tmem_wait_regs(uint32_t (&r)[N])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < N; ++i) asm volatile("" : "+r"(r[i]));
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// ---------------------------------------------------------------------------
// Natural logarithm of a positive normal double by the table-driven method of
// P. T. P. Tang ("Table-driven implementation of the logarithm function in
// IEEE floating-point arithmetic", ACM TOMS 16(4), 1990): x = 2^e m with m in
// [1, 2); F = 1 + j/128 from the leading seven fraction bits of m, f = m - F
// (exact), u = f / F in [0, 2^-7) (as f times a tabulated 1/F); then
//   ln x = e ln 2 + ln F + ln(1 + u),
// ln(1 + u) = sum_{i=1..8} (-1)^(i+1) u^i / i (truncation below 2^-59),
// evaluated in Estrin's scheme (dependency depth 6 instead of 9).  ln F and
// 1/F are tabulated by the block at start-up (ln F by the library logarithm).
// The absolute error is within a few units in the last place of
// max(|ln x|, ln 2); zero, negative, subnormal and non-finite x take the
// library path.
// ---------------------------------------------------------------------------
constexpr double LN2_HI = 0.6931471805599453094;      // ln 2 rounded to double
constexpr double LN2_LO = 2.319046813846299558e-17;   // ln 2 - LN2_HI

__device__ inline void log_tang_table(double *tab, int t0, int nt)
{
    for (int j = t0; j < 128; j += nt) {
        const double F = 1.0 + double(j) * (1.0 / 128.0);
        tab[j] = 1.0 / F;
        tab[128 + j] = log(F);
    }
}

__device__ __forceinline__ double log_tang(double x, const double *tab)
{
    const long long b = __double_as_longlong(x);
    const int eb = int((b >> 52) & 0x7ff);
    if (b <= 0 || eb == 0 || eb == 0x7ff) return log(x);      // <= 0, -0, subnormal, inf, nan
    const int j = int((b >> 45) & 127);
    const double m = __longlong_as_double((b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
    const double F = __longlong_as_double((b & 0x000fe00000000000LL) | 0x3ff0000000000000LL);
    const double u = (m - F) * tab[j];
    const double u2 = u * u;
    const double u4 = u2 * u2;
    const double p01 = fma(-0.5, u, 1.0);
    const double p23 = fma(-0.25, u, 1.0 / 3.0);
    const double p45 = fma(-1.0 / 6.0, u, 0.2);
    const double p67 = fma(-0.125, u, 1.0 / 7.0);
    const double q = fma(u4, fma(u2, p67, p45), fma(u2, p23, p01));
    const double e = double(eb - 1023);
    return fma(e, LN2_HI, tab[128 + j]) + fma(e, LN2_LO, u * q);
}


// ---------------------------------------------------------------------------
// 1/sqrt(p) for positive normal p with a short dependency chain: the PTX
// approximation rsqrt.approx.f64 as the seed, then one step of the
// third-order iteration y' = y (1 + e/2 + 3e^2/8), e = 1 - p y^2 (the
// binomial series of (1 - e)^(-1/2) to second order), which takes a seed
// error of 2^-20 below 2^-59 before the final rounding.  Zero, negative,
// subnormal and non-finite p take the library path.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double rsqrt_fast(double p)
{
    const long long b = __double_as_longlong(p);
    const int eb = int((b >> 52) & 0x7ff);
    if (b <= 0 || eb == 0 || eb == 0x7ff) return rsqrt(p);
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(p));
    const double e = fma(-(p * y), y, 1.0);
    return fma(y, e * fma(0.375, e, 0.5), y);
}

// ---------------------------------------------------------------------------
// Digamma for x > 0 (FP64): shift the argument up to x >= 8 with
// psi(x) = psi(x + 1) - 1/x, then the Stirling-type asymptotic series
// psi(x) = ln x - 1/(2x) - sum_{k=1..7} B_{2k} / (2k x^{2k}) with the
// Bernoulli numbers B_2 .. B_14 (Abramowitz & Stegun 6.3.18).  Truncation
// error below 3e-14 at x = 8.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double digamma_d(double x)
{
    double shift = 0.0;
    while (x < 8.0) {
        shift += 1.0 / x;
        x += 1.0;
    }
    const double r = 1.0 / x;
    const double r2 = r * r;
    // coefficients B_{2k}/(2k): 1/12, -1/120, 1/252, -1/240, 1/132, -691/32760, 1/12
    double p = 1.0 / 12.0;
    p = -691.0 / 32760.0 + r2 * p;
    p = 1.0 / 132.0 + r2 * p;
    p = -1.0 / 240.0 + r2 * p;
    p = 1.0 / 252.0 + r2 * p;
    p = -1.0 / 120.0 + r2 * p;
    p = 1.0 / 12.0 + r2 * p;
    return log(x) - 0.5 * r - r2 * p - shift;
}

} // namespace vbh
