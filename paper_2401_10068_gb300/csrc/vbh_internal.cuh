// vbh_internal.cuh -- device-side state and helpers shared by the kernels of
// libvbh (the CUDA path).  Nothing here is used by the CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vbh {

constexpr int MMAX = 31;             // largest M = S - 1
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

// What one data pass reads: the FP32 form of Sigma0 = W^{-1}/nu (its packed
// lower Cholesky factor, row i at offset i(i+1)/2), kappa and E[rho].
struct SweepGlobalsF32 {
    float L[MMAX * (MMAX + 1) / 2];
    float kappa[MMAX];
    float erho;
    int pad;
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
    int pad0;
    double *trace;                   // device array [max_iter + 1] (may be null)
    // per-fit constants: kc_upd for (a0 + V/2, n0 + V, q0 + V), kc_given for
    // the factors a fit or vbh_elbo starts from; prior_const collects the
    // prior-only terms of the ELBO (dropping ln B(Lambda_0, n0) when improper)
    ElboConst kc_upd, kc_given;
    double prior_const;
    int prior_dropped, pad1;
    SweepGlobalsF32 sw;
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
