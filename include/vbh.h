/*
 * vbh.h -- C ABI of the GB300 (sm_103a) implementation of the mean-field
 * variational-Bayes (CAVI) iteration for the conjugate-exponential model of
 * cancer-tissue heterogeneity (arXiv 2401.10068, Sections 3.3-3.5).
 *
 * Model (Section 3.3).  There are V observations r_i (one gene-expression ratio
 * each) with known expression profiles d_i in R^S over S subpopulations (the
 * paper's N).  With M = S - 1, mu_i = d_{i,S}, D_i = d_{i,1:M} - d_{i,S}:
 *   r_i    ~ N(D_i^T beta_i + mu_i, 1/rho)             Eq. 3
 *   beta_i ~ N(K, Lambda^{-1})                         Eq. 4
 *   rho ~ Gamma(a0, b0),  K | Lambda ~ N(K0, (q0 Lambda)^{-1}),
 *   Lambda ~ Wishart(n0, scale Lambda_0)               Eq. 5-7
 * The posterior is approximated by Q(rho) Q(beta) Q(K, Lambda) (Eq. 13) and
 * fitted by coordinate ascent: Q(beta) (Eq. 19-21), Q(rho) (Eq. 16-18),
 * Q(K, Lambda) (Eq. 22-25), with the expectations of Eq. 26-31 and the lower
 * bound L_Q of Eq. 10-11 as the convergence monitor.
 *
 * Conventions for every entry point:
 *   - Return 0 (VBH_OK) or a negative VBH_E* code; vbh_strerror() names it.
 *   - Calls are synchronous on the handle's stream: when a call returns, its
 *     results are in host memory and no work of the call is in flight.
 *   - The caller owns every buffer it passes; the library only reads r and d.
 *   - A handle is not thread-safe; use one handle per host thread.
 *   - r and d may be device pointers (any CUDA allocation on the handle's
 *     device) or host pointers (pageable or pinned); host inputs are copied to
 *     a device buffer owned by the handle, inside the call.
 *   - r: V floats.  d: V x S floats, row-major (the S entries of profile d_i
 *     are contiguous).  Device pointers must be 16-byte aligned.
 *   - The sweep is FP32 per observation with FP64 accumulation across blocks
 *     and FP64 global updates; non-finite results return VBH_ENONFINITE.
 *     With a stopping test (tol > 0) the CUDA-core sweeps (S <= 11) also
 *     carry the compensated statistics of the ELBO (vbh_opts.stats).
 *   - For 12 <= S <= 32 the two contractions per observation that grow with
 *     M^2 (q_i = D_i^T Sigma0 D_i of Eq. 20-21 and the sum of
 *     (w_i^2 - c_i) D_i D_i^T that enters Eq. 25) run on the tensor cores:
 *     the profiles are converted once per fit to BF16 (a device buffer of
 *     V x 64 bytes owned by the handle) and every FP32 operand is split into
 *     BF16 parts, three for VBH_FP32 (the FP32 values) and two for VBH_BF16
 *     (16 significant bits).  VBH_FP32 then needs profiles that BF16 holds
 *     exactly (binary profiles, as in the paper, do) and returns
 *     VBH_EUNSUPPORTED otherwise; VBH_BF16 rounds any profile to BF16.
 *     Accumulation is FP32 over 16 tiles of 128 observations, compensated FP32
 *     across tiles, FP64 across blocks.  These fits need V < 2^31.
 */
#ifndef VBH_H
#define VBH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VBH_SMAX 32              /* largest number of subpopulations S */
#define VBH_MMAX 31              /* largest M = S - 1 */

/* status codes */
#define VBH_OK 0
#define VBH_EINVAL (-1)          /* invalid argument (null pointer, size, alignment, S) */
#define VBH_ENOMEM (-2)          /* device or host allocation failed */
#define VBH_ECUDA (-3)           /* a CUDA runtime call failed */
#define VBH_ENONFINITE (-4)      /* a global update or the ELBO became NaN/Inf */
#define VBH_ETIMEOUT (-5)        /* a bounded device wait ran out (the kernel returned early) */
#define VBH_ESTATE (-6)          /* call out of order (e.g. vbh_fit_step before vbh_fit_begin) */
#define VBH_EUNSUPPORTED (-7)    /* valid request this build does not implement (e.g. S above the FP32 sweep limit) */

/* precision of the per-observation sweep */
#define VBH_FP32 0               /* FP32 products and sums per observation */
#define VBH_BF16 1               /* 12 <= S <= 32: 16-bit tensor-core operands for all but the last
                                    vbh_opts.refine_iters sweeps, which run as VBH_FP32; S <= 11 runs VBH_FP32 */

/* method of a fit */
#define VBH_CAVI 0               /* variational Bayes: Q(rho) Q(beta) Q(K, Lambda) by coordinate ascent (Section 3.5) */
#define VBH_EM 1                 /* expectation maximisation: point estimates of K, Lambda, rho (Section 4.2,
                                    Eq. 42-47); see vbh_opts.method */

/* statistics of the per-observation sweep, S <= 11 (vbh_opts.stats) */
#define VBH_STATS_AUTO 0         /* VBH_STATS_COMPENSATED when the fit has a stopping test (tol > 0), else plain */
#define VBH_STATS_COMPENSATED 1  /* the pass also carries U = sum c_i e_i^2 and sum ln(1 + E[rho] q_i) in
                                    two-part FP32 arithmetic (~2^-40), which replace the first-order part of the
                                    FP32 sums in the ELBO: its rounding noise between sweeps drops from ~1e-8 |L|
                                    (binary profiles repeat the same FP32 rounding in every observation of a
                                    profile) to ~1e-11 |L|, so a relative stopping tolerance of 1e-8 is met by
                                    convergence, not by noise.  About 1.5x the arithmetic per observation. */
#define VBH_STATS_PLAIN 2        /* FP32 statistics only (the fastest pass; ELBO noise ~1e-8 |L|) */

/* sweep loop of the per-observation FP32 sweep, S <= 11, not grouped (vbh_opts.loop) */
#define VBH_LOOP_AUTO 0          /* VBH_LOOP_RESIDENT when the data set fits, else VBH_LOOP_STREAM */
#define VBH_LOOP_STREAM 1        /* one launch per sweep, reading (r, d) from device memory (the sweep loop of
                                    vbh_create's note) */
#define VBH_LOOP_RESIDENT 2      /* one cooperative launch per vbh_fit_step call runs all its sweeps: every block
                                    keeps a slice of (r, d) in shared memory, and the blocks meet at one grid
                                    barrier per sweep, after which each runs the FP64 global update on the same
                                    partial sums (identical results in every block).  The data set must fit in
                                    the shared memory of one block per SM: about 14,000 observations per SM at
                                    S = 3, 3,000 at S = 11 with the compensated statistics (VBH_EUNSUPPORTED
                                    otherwise).  Same arithmetic per observation as the streaming sweep; the
                                    sums are taken over other blocks, so results agree to FP32 rounding.  A
                                    barrier wait that runs out (2 s) ends the fit with VBH_ETIMEOUT. */

/* initial state of a fit */
#define VBH_INIT_PAPER 0         /* Q(beta_i) = N(K0, Lambda_0^{-1}) before sweep 0 (Section 3.5) */
#define VBH_INIT_GIVEN 1         /* start from the global factors in vbh_opts.init_state (warm start / resume) */

typedef struct vbh_handle vbh_handle;

/* Prior constants of Eq. 5-7.  vbh_prior_default() fills the paper's values
 * (Section 3.5): K0 = (1/S, ..., 1/S), q0 = 0.001, n0 = 1, a0 = b0 = 0.5 and
 * Lambda_0^{-1} = 0.005 * 1 1^T + diag(0.005, 0.003, 0.005, 0.003, ...),
 * which is the paper's [[0.01, 0.005], [0.005, 0.008]] for S = 3. */
typedef struct {
    int S;                       /* 1 .. VBH_SMAX */
    const double *K0;            /* M entries (host memory), or NULL for 1/S each */
    double q0, n0, a0, b0;       /* q0 > 0, n0 > 0, a0 > 0, b0 > 0 */
    const double *Lambda0_inv;   /* M x M row-major symmetric positive definite (host), or NULL for the default */
} vbh_prior;

/* Posterior summary, also usable as a checkpoint (vbh_opts.init_state). */
typedef struct {
    int S, iters, converged, status, elbo_const_dropped;
    double kappa[VBH_MMAX];      /* E[K] = K_{0K}, Eq. 24/30 */
    double weights[VBH_SMAX];    /* (kappa, 1 - sum kappa): all S subpopulation weights (Section 3.3) */
    double W_inv[VBH_MMAX * VBH_MMAX]; /* Lambda_{0Lambda}^{-1}, Eq. 25 (M x M row-major) */
    double nu, lambda;           /* n0 + V (Eq. 23), q0 + V (Eq. 22) */
    double a_rho, b_rho;         /* Q(rho) = Gamma(a_rho, b_rho), Eq. 16-18 */
    double rho_mean, rho_mode;   /* a_rho / b_rho (Eq. 29), (a_rho - 1) / b_rho */
    double elbo;                 /* L_Q of Eq. 11 after the last sweep */
} vbh_result;

typedef struct {
    double tol;                  /* stop after sweep t >= 1 when |L_t - L_{t-1}| < tol |L_t|; 0 runs max_iter sweeps */
    int max_iter;                /* sweeps after sweep 0, >= 0 */
    int precision;               /* VBH_FP32 or VBH_BF16 */
    int init;                    /* VBH_INIT_PAPER or VBH_INIT_GIVEN */
    int refine_iters;            /* VBH_BF16 only: the last sweeps (>= 0, of max_iter) run as VBH_FP32;
                                    after the 16-bit sweeps stop (tolerance or count) the FP32 sweeps
                                    continue with the same tolerance test */
    const vbh_result *init_state;/* global factors to start from when init == VBH_INIT_GIVEN */
    double *elbo_trace;          /* optional host array of max_iter + 1 doubles: L_0 .. L_iters */
    int method;                  /* VBH_CAVI or VBH_EM.  EM maximises ln p(r | K, Lambda, rho) (beta_i
                                    integrated out; Eq. 45-47 carry no prior terms).  Iteration n evaluates
                                    ln p(r | theta^(n)) -- the "elbo" of the trace and result -- and forms
                                    theta^(n+1), which the result holds: kappa = K, W_inv = Lambda^{-1},
                                    a_rho = rho_mean = rho_mode = rho, b_rho = nu = 1, lambda = V.  Start:
                                    VBH_INIT_PAPER takes K0, Lambda_0^{-1} and rho = a0 / b0 from the prior;
                                    VBH_INIT_GIVEN takes kappa, W_inv and a_rho / b_rho of init_state.
                                    vbh_fit_batched and vbh_fit_static run VBH_CAVI only. */
    int grouped;                 /* 1: exact profile-grouped sweeps for binary profiles (every d_ij 0 or 1;
                                    otherwise VBH_EINVAL), S <= 16: one pass histograms (count, sum y,
                                    sum y^2) per profile, y = r - d_S (FP64), and every sweep then runs over
                                    the 2^S profiles in FP64 at a cost independent of V.  Same schedule,
                                    methods and results as the per-observation sweeps (up to their FP32
                                    rounding); the histogram's FP64 atomic sums make the last bits depend on
                                    the order of the additions.  Ignores precision. */
    int stats;                   /* VBH_STATS_AUTO (0), VBH_STATS_COMPENSATED or VBH_STATS_PLAIN; only the
                                    CUDA-core sweeps (S <= 11, not grouped) have the compensated form, the
                                    others ignore it.  vbh_elbo always uses the compensated form there. */
    int loop;                    /* VBH_LOOP_AUTO (0), VBH_LOOP_STREAM or VBH_LOOP_RESIDENT: how vbh_fit and
                                    vbh_fit_step run the sweeps (sweep 0 of a fit always streams) */
} vbh_opts;

/* Fill *p with the paper's prior for S subpopulations (Section 3.5). */
void vbh_prior_default(int S, vbh_prior *p);

/* Fill *o with tol = 1e-8, max_iter = 200, VBH_FP32, VBH_INIT_PAPER, refine_iters = 10, no trace,
 * VBH_CAVI, not grouped, VBH_STATS_AUTO, VBH_LOOP_AUTO. */
void vbh_opts_default(vbh_opts *o);

/* Create a handle on CUDA device `device` that issues all work on `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The stream is borrowed:
 * it must outlive the handle.  Returns VBH_EINVAL for a bad device.
 * The streaming sweep loop (VBH_LOOP_STREAM) runs as a CUDA graph with a
 * conditional while node; with the environment variable VBH_LAUNCH=direct at
 * creation the handle instead issues one kernel launch per sweep (same kernels
 * and results; for profilers that cannot look inside conditional graphs).  The
 * resident loop (VBH_LOOP_RESIDENT) sizes its blocks for about
 * VBH_RESIDENT_OBS (environment, default 2) observations per thread and sweep. */
int vbh_create(vbh_handle **h, int device, void *stream);

/* Release every resource of the handle (NULL is allowed). */
void vbh_destroy(vbh_handle *h);

/* Name of a status code (static string). */
const char *vbh_strerror(int status);

/* Detail of the last failed CUDA call behind a VBH_ECUDA or VBH_ENOMEM status
 * returned to the calling host thread ("<call> at <file>:<line>: <error>"),
 * or "" if there was none.  Thread-local static storage: valid until the
 * thread's next failing call. */
const char *vbh_last_error_detail(void);

/* Diagnostic of the bounded device waits.  Every kernel of the library waits
 * on mbarriers through waits that give up after a wall-time budget, after
 * which the kernel records VBH_ETIMEOUT, lets its own copies land and returns
 * (no trap, the CUDA context stays usable).  This runs those waits in one
 * block on `stream` of `device`: on a barrier phase that nothing completes
 * (status[0]: polling wait, status[1]: wait with a sleep between polls; both
 * must be VBH_ETIMEOUT after budget_ns, 0 < budget_ns <= 1e9) and on a phase
 * that a 1 KiB bulk copy completes (status[2]: VBH_OK; status[3]: VBH_OK when
 * the copied bytes are right).  *waited_ns receives the time the first wait
 * took.  Allocates and frees about 1 KiB of device memory; synchronous. */
int vbh_selftest_wait(int device, void *stream, uint64_t budget_ns, int *status, uint64_t *waited_ns);

/* Diagnostic of two short-latency FP64 functions of the global updates, out[i]
 * = f(x[i]) for n (1 .. 2^24) host doubles:
 *   fn 0: the natural logarithm the resident sweep loop's ELBO uses (Tang's
 *         table-driven method: 128 tabulated ln F and 1/F, F = 1 + j/128, and
 *         a degree-8 series of ln(1 + u), |u| < 2^-7); absolute error a few
 *         units in the last place of max(|ln x|, ln 2);
 *   fn 1: the reciprocal square root of the Cholesky factorisations (the
 *         PTX approximation as the seed and one third-order correction);
 *         within about an ulp.
 * Allocates and frees 16 n bytes of device memory; synchronous. */
int vbh_selftest_math(int device, void *stream, int fn, const double *x, double *out, int n);

/* Bytes of the device-resident fit state that each vbh_fit_begin,
 * vbh_fit_step and vbh_fit_result call copies back to the host (a vbh_fit
 * call copies it three times); for accounting of host<->device traffic. */
size_t vbh_state_bytes(void);

/* Fit Q(rho) Q(beta) Q(K, Lambda) to (r, d): sweep 0 from the initial state,
 * then up to o->max_iter sweeps of Q(beta) -> Q(rho) -> Q(K, Lambda) -> ELBO
 * (Section 3.5), run on the device as one CUDA graph with a conditional while
 * loop.  out receives the final global factors; out->converged = 0 when the
 * sweep limit was reached first (not an error).  V = 0 is allowed: the
 * posterior is then the prior. */
int vbh_fit(vbh_handle *h, const float *r, const float *d, int64_t V, int S, const vbh_prior *p,
            const vbh_opts *o, vbh_result *out);

/* Step-wise form of vbh_fit.  vbh_fit_begin validates, stages the inputs and
 * runs sweep 0; vbh_fit_step runs up to nsweeps further sweeps (fewer if the
 * fit converges or reaches o->max_iter) and reports the convergence flag;
 * vbh_fit_result copies the current global factors out.  The inputs must stay
 * valid and unchanged until the next vbh_fit_begin / vbh_fit / vbh_destroy. */
int vbh_fit_begin(vbh_handle *h, const float *r, const float *d, int64_t V, int S, const vbh_prior *p,
                  const vbh_opts *o);
int vbh_fit_step(vbh_handle *h, int nsweeps, int *converged);
int vbh_fit_result(vbh_handle *h, vbh_result *out);

/* Fit B independent data sets in one device loop (the batched form).  Data
 * set b has V[b] observations and S[b] subpopulations (1 .. 11), inputs r[b]
 * (V[b] floats) and d[b] (V[b] x S[b] floats, row-major): for each b both
 * device pointers (16-byte aligned) or both host pointers (staged by the call).
 * p: B priors, or NULL for vbh_prior_default(S[b]) each.  o: one set of options
 * for all data sets; with o->init == VBH_INIT_GIVEN, o->init_state points to B
 * results; o->elbo_trace, if set, holds B * (o->max_iter + 1) doubles (row b
 * is L_0 .. L_iters of data set b).  out: B results.
 * Each data set follows exactly the schedule of vbh_fit (sweep 0, then sweeps
 * until its own convergence test or o->max_iter) and retires when done; one
 * batched sweep is, per class of equal S, a persistent data-pass kernel over
 * chunks of contiguous observations taken from a work queue and one FP64
 * update per data set, and the loop is a CUDA graph with a conditional while
 * node.  For batches of at least 2^26 observations the pass shape of each
 * class (tiles per chunk and pipeline stages) is autotuned by timing one data
 * pass per candidate; vbh_batched_plan reports the choice.
 * Returns the first non-zero per-data-set status (also in out[b].status). */
int vbh_fit_batched(vbh_handle *h, int B, const int64_t *V, const int *S, const float *const *r,
                    const float *const *d, const vbh_prior *p, const vbh_opts *o, vbh_result *out);

/* The data-pass shape of one class (equal S) in the last vbh_fit_batched call. */
typedef struct vbh_batch_plan {
    int S;
    int tile;                    /* observations per tile (one bulk copy per tile) */
    int chunk_tiles;             /* tiles per chunk (work-queue unit) */
    int stages;                  /* pipeline stages of the shared-memory ring */
    int blocks_per_sm;           /* resident pass blocks per SM at that ring */
    float pass_ms;               /* the autotuner's time of one data pass of the class with that shape
                                    (0 when the batch was too small to tune) */
} vbh_batch_plan;

/* Copy up to `cap` class plans of the last vbh_fit_batched call on h (classes
 * in increasing S) into out (may be NULL when cap is 0) and their number into
 * *n.  Returns VBH_EINVAL for a NULL h or n. */
int vbh_batched_plan(vbh_handle *h, vbh_batch_plan *out, int cap, int *n);

/* ELBO (Eq. 11) of the global factors in *q (kappa, W_inv, nu, lambda,
 * a_rho, b_rho) with Q(beta) set from them by Eq. 19-21: one data pass and no
 * update of *q. */
int vbh_elbo(vbh_handle *h, const float *r, const float *d, int64_t V, int S, const vbh_prior *p,
             const vbh_result *q, double *elbo);

/* ---------------------------------------------------------------------------
 * vbh_fit_static: the same fit as vbh_fit, for callers that cannot allocate
 * device memory.  The paper has no counterpart of this entry point.
 *
 * vbh_fit and the other entry points work through a handle, which allocates
 * device buffers (cudaMalloc) and builds a CUDA graph.  Some callers cannot
 * allow that: cudaMalloc and cudaFree synchronise the whole device and stall
 * latency-sensitive work on other streams; frameworks that serve all device
 * memory from their own pool may leave a foreign cudaMalloc without memory;
 * plug-in hosts and fixed-budget deployments forbid allocations beyond the
 * budget fixed when the library is loaded.  vbh_fit_static needs no handle
 * and performs no allocation (no cudaMalloc, cudaFree, graph or pool call):
 * its scratch -- the fit state, the per-block partial sums and the ELBO
 * trace -- is one statically sized __device__ array of
 * VBH_STATIC_SCRATCH_BYTES that every GPU loading the library holds from load
 * until process exit.
 *
 *   r, d:    device pointers on `device` (16-byte aligned), layout as for
 *            vbh_fit; host pointers are rejected (staging them would allocate).
 *   p, o:    as for vbh_fit; with o->elbo_trace set, o->max_iter + 1 must not
 *            exceed VBH_STATIC_TRACE_MAX (else VBH_EINVAL).  S > 11 returns
 *            VBH_EUNSUPPORTED (vbh_fit runs it on the tensor-core path, which
 *            this entry point lacks); so do o->method = VBH_EM and
 *            o->grouped = 1.
 *   out:     the result, as for vbh_fit.
 *   stream:  a cudaStream_t on `device` (NULL = legacy default stream); the
 *            call is synchronous on it.
 * The sweeps run as one kernel launch each, issued in batches of 64; between
 * batches the call reads the fit's control fields back and issues no more
 * launches once the fit has stopped.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress, with that device
 * current) and loads every kernel this entry point can launch, for every S:
 * under CUDA's lazy module loading the first use of a kernel loads its
 * module, which allocates device memory, so this first call per device is
 * the only one that may load code or allocate.  Make it before any stream
 * capture and before the caller's device memory is fully committed.  All
 * calls on a device share the one array
 * and every call rewrites the whole fit state before its first kernel, so
 * nothing of an earlier call carries over; but calls whose work overlaps on
 * the GPU (other host threads, other streams) race on the array and must be
 * serialised by the caller. */
#define VBH_STATIC_SCRATCH_BYTES (512 * 1024)
#define VBH_STATIC_TRACE_MAX 4097
int vbh_fit_static(const float *r, const float *d, int64_t V, int S, const vbh_prior *p, const vbh_opts *o,
                   vbh_result *out, int device, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* VBH_H */
