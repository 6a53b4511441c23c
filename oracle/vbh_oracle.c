/*
 * vbh_oracle.c -- plain FP64 CPU oracle of the mean-field variational-Bayes
 * (CAVI) iteration for the conjugate-exponential cancer-tissue model of
 * Sections 3.3-3.5 (Eq. 2-31), and of its expectation-maximisation variant
 * (Section 4.2, Eq. 42-47).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call this library.
 * It shares no code, header, helper or constant with the CUDA path.  It is
 * deliberately slow and direct: every Q(beta_i) is formed and inverted
 * explicitly (Eq. 20-21), exactly as the paper states it, so that a reader can
 * check each line against the equations.
 *
 * Notation (paper -> here):
 *   N subpopulations          -> S, with M = S - 1
 *   mu_i = d_{i,N}            -> dS
 *   D_i = d_{i,1:N-1} - d_{i,N}-> D[M]
 *   K_{0K}                    -> kappa
 *   Lambda_{0Lambda}^{-1}     -> Winv   (so E[Lambda] = nu * inv(Winv), Eq. 28)
 *   n0 + V                    -> nu      (Eq. 23)
 *   q0 + V                    -> lam     (Eq. 22)
 *   Lambda_0^{-1}             -> L0inv   (prior inverse scale of the Wishart, Eq. 7)
 *
 * Readings of the paper that this file takes (each also listed in the design
 * notes of the repository):
 *   - Gamma(a, b) has shape a and rate ("inverse scale") b (Eq. 5, 16-18).
 *   - In Wish(Lambda | n, X) (Eq. 7, 23) n is the number of degrees of
 *     freedom and X is the INVERSE of the scale matrix: that is the only
 *     reading under which Eq. 28 (E[Lambda] = (n0 + V) Lambda_{0Lambda}) is
 *     the Wishart mean.  So the prior scale is Lambda_0, and the posterior
 *     scale W satisfies W^{-1} = Eq. 25.
 *   - Sweep order: Q(beta) -> Q(rho) -> Q(K,Lambda) -> ELBO.  Sweep 0 starts
 *     from Q(beta_i) = N(K0, Lambda_0^{-1}) (the initialisation paragraph of
 *     Section 3.5) and runs only the Q(rho), Q(K,Lambda) updates and the ELBO.
 *   - The ELBO (Eq. 11) is expanded with the standard Gamma / Gaussian /
 *     Wishart expectations and entropies; the log normaliser of the Wishart
 *     prior is dropped (and *const_dropped set) when n0 <= M - 1, where the
 *     prior is improper.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define VBO_MMAX 31
#define VBO_LN2PI 1.83787706640934548356065947281
#define VBO_LNPI 1.14472988584940017414342735135
#define VBO_LN2 0.693147180559945309417232121458

/* Prior constants of Eq. 5-7. */
typedef struct {
    int S;                              /* number of subpopulations (paper: N) */
    double K0[VBO_MMAX];                /* prior mean of K, Eq. 6 */
    double q0, n0, a0, b0;              /* Eq. 5-7 */
    double L0inv[VBO_MMAX * VBO_MMAX];  /* Lambda_0^{-1}, Eq. 7, row-major M x M */
} vbo_prior;

/* Parameters of the global factors Q(rho) and Q(K, Lambda). */
typedef struct {
    double a_rho, b_rho;                /* Q(rho) = Gamma(a_rho, b_rho), Eq. 16-18 */
    double nu;                          /* Wishart degrees of freedom n0 + V, Eq. 23 */
    double lam;                         /* q0 + V, Eq. 22 */
    double kappa[VBO_MMAX];             /* K_{0K}, Eq. 24 */
    double Winv[VBO_MMAX * VBO_MMAX];   /* Lambda_{0Lambda}^{-1}, Eq. 25 */
} vbo_glob;

/* The sums over observations that Eq. 17, 24, 25 and the ELBO consume. */
typedef struct {
    double V;                           /* number of observations summed */
    double sum_S;                       /* sum_i {braces of Eq. 17} */
    double sum_mu[VBO_MMAX];            /* sum_i E[beta_i], Eq. 24 */
    double sum_Ebb[VBO_MMAX * VBO_MMAX];/* sum_i E[beta_i beta_i^T], Eq. 25, 27 */
    double sum_logdet;                  /* sum_i ln|Lambda_{beta_i}^{-1}| (entropy of Q(beta)) */
} vbo_sums;

/* ------------------------------------------------------------------------ */
/* Small dense linear algebra, row-major M x M.                              */
/* ------------------------------------------------------------------------ */

/* A = L L^T with L lower triangular.  Returns 0, or -1 if A is not positive
 * definite. */
static int chol(int M, const double *A, double *L)
{
    for (int i = 0; i < M * M; ++i) L[i] = 0.0;
    for (int j = 0; j < M; ++j) {
        double s = A[j * M + j];
        for (int k = 0; k < j; ++k) s -= L[j * M + k] * L[j * M + k];
        if (!(s > 0.0)) return -1;
        double ljj = sqrt(s);
        L[j * M + j] = ljj;
        for (int i = j + 1; i < M; ++i) {
            double t = A[i * M + j];
            for (int k = 0; k < j; ++k) t -= L[i * M + k] * L[j * M + k];
            L[i * M + j] = t / ljj;
        }
    }
    return 0;
}

/* Inverse and log-determinant of a symmetric positive-definite matrix, by
 * solving A x = e_c for every column c through the Cholesky factor. */
static int spd_inverse(int M, const double *A, double *Ainv, double *logdet)
{
    double L[VBO_MMAX * VBO_MMAX];
    if (chol(M, A, L)) return -1;
    if (logdet) {
        double s = 0.0;
        for (int j = 0; j < M; ++j) s += 2.0 * log(L[j * M + j]);
        *logdet = s;
    }
    for (int c = 0; c < M; ++c) {
        double y[VBO_MMAX], x[VBO_MMAX];
        for (int i = 0; i < M; ++i) {          /* L y = e_c */
            double t = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) t -= L[i * M + k] * y[k];
            y[i] = t / L[i * M + i];
        }
        for (int i = M - 1; i >= 0; --i) {     /* L^T x = y */
            double t = y[i];
            for (int k = i + 1; k < M; ++k) t -= L[k * M + i] * x[k];
            x[i] = t / L[i * M + i];
        }
        for (int i = 0; i < M; ++i) Ainv[i * M + c] = x[i];
    }
    for (int i = 0; i < M; ++i)                /* exact symmetry */
        for (int j = 0; j < i; ++j) {
            double a = 0.5 * (Ainv[i * M + j] + Ainv[j * M + i]);
            Ainv[i * M + j] = a;
            Ainv[j * M + i] = a;
        }
    return 0;
}

static int spd_logdet(int M, const double *A, double *logdet)
{
    double L[VBO_MMAX * VBO_MMAX];
    if (chol(M, A, L)) return -1;
    double s = 0.0;
    for (int j = 0; j < M; ++j) s += 2.0 * log(L[j * M + j]);
    *logdet = s;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Special functions.                                                        */
/* ------------------------------------------------------------------------ */

/* Digamma psi(x), x > 0.  The recurrence psi(x) = psi(x + 1) - 1/x moves the
 * argument to x >= 10; there the asymptotic expansion
 *   psi(x) ~ ln x - 1/(2x) - sum_k B_{2k} / (2k x^{2k})
 * (Abramowitz & Stegun 6.3.18, Bernoulli numbers B_2..B_10) is accurate to
 * about 2e-14. */
double vbo_digamma(double x)
{
    double acc = 0.0;
    while (x < 10.0) {
        acc -= 1.0 / x;
        x += 1.0;
    }
    double z = 1.0 / (x * x);
    double tail = z * (1.0 / 12.0 - z * (1.0 / 120.0 - z * (1.0 / 252.0 - z * (1.0 / 240.0 - z * (1.0 / 132.0)))));
    return acc + log(x) - 0.5 / x - tail;
}

/* ln B(W, nu), the log normaliser of the Wishart density with scale W and nu
 * degrees of freedom (Bishop, PRML B.79), written with ln|W|. */
static double wishart_lnB(int M, double lndetW, double nu)
{
    double s = -0.5 * nu * lndetW - 0.5 * nu * M * VBO_LN2 - 0.25 * M * (M - 1) * VBO_LNPI;
    for (int j = 1; j <= M; ++j) s -= lgamma(0.5 * (nu + 1.0 - j));
    return s;
}

/* E[ln|Lambda|] under Wish(W, nu) (PRML B.81). */
static double wishart_Elndet(int M, double lndetW, double nu)
{
    double s = M * VBO_LN2 + lndetW;
    for (int j = 1; j <= M; ++j) s += vbo_digamma(0.5 * (nu + 1.0 - j));
    return s;
}

/* ------------------------------------------------------------------------ */
/* Per-observation reparametrisation (Section 3.3, text before Eq. 3).       */
/* ------------------------------------------------------------------------ */

/* mu_i = d_{i,S}; D_i = d_{i,1:M} - d_{i,S}; ytilde_i = r_i - mu_i. */
static void observation(int S, const float *r, const float *d, int64_t i, double *D, double *yt)
{
    int M = S - 1;
    double dS = (double)d[i * S + M];
    for (int j = 0; j < M; ++j) D[j] = (double)d[i * S + j] - dS;
    *yt = (double)r[i] - dS;
}

/* ------------------------------------------------------------------------ */
/* Q(beta) -- initialisation and Eq. 19-21.                                  */
/* ------------------------------------------------------------------------ */

/* Initial Q(beta_i): mean K0, covariance Lambda_0^{-1} (Section 3.5, the
 * paragraph that initialises Lambda_{beta_i} to Lambda_0). */
void vbo_beta_init(const vbo_prior *p, int64_t V, double *mu, double *Sig)
{
    int M = p->S - 1;
    for (int64_t i = 0; i < V; ++i) {
        for (int j = 0; j < M; ++j) mu[i * M + j] = p->K0[j];
        for (int j = 0; j < M * M; ++j) Sig[i * M * M + j] = p->L0inv[j];
    }
}

/* Eq. 19-21 with the expectations of Eq. 28, 29, 31:
 *   Lambda_{beta_i} = E[Lambda] + E[rho] D_i D_i^T
 *   mu_{beta_i}     = Lambda_{beta_i}^{-1} (E[Lambda K] + E[rho] D_i (r_i - mu_i))
 * Stores mu_{beta_i} and Sigma_i = Lambda_{beta_i}^{-1} (explicit inverse).
 * Returns 0, or -1 if a matrix is not positive definite. */
int vbo_beta_update(const vbo_prior *p, int64_t V, const float *r, const float *d,
                    const vbo_glob *g, double *mu, double *Sig)
{
    int S = p->S, M = S - 1;
    double EL[VBO_MMAX * VBO_MMAX], ELK[VBO_MMAX];
    if (M > 0 && spd_inverse(M, g->Winv, EL, NULL)) return -1;
    for (int j = 0; j < M * M; ++j) EL[j] *= g->nu;                 /* Eq. 28 */
    for (int j = 0; j < M; ++j) {                                    /* Eq. 31 */
        double t = 0.0;
        for (int k = 0; k < M; ++k) t += EL[j * M + k] * g->kappa[k];
        ELK[j] = t;
    }
    double Erho = g->a_rho / g->b_rho;                               /* Eq. 29 */
    for (int64_t i = 0; i < V; ++i) {
        double D[VBO_MMAX], yt, Lb[VBO_MMAX * VBO_MMAX], rhs[VBO_MMAX];
        observation(S, r, d, i, D, &yt);
        for (int j = 0; j < M; ++j)
            for (int k = 0; k < M; ++k) Lb[j * M + k] = EL[j * M + k] + Erho * D[j] * D[k];   /* Eq. 20 */
        double *Si = Sig + i * M * M;
        if (M > 0 && spd_inverse(M, Lb, Si, NULL)) return -1;
        for (int j = 0; j < M; ++j) rhs[j] = ELK[j] + Erho * D[j] * yt;
        for (int j = 0; j < M; ++j) {                                                       /* Eq. 21 */
            double t = 0.0;
            for (int k = 0; k < M; ++k) t += Si[j * M + k] * rhs[k];
            mu[i * M + j] = t;
        }
    }
    return 0;
}

/* The reductions over observations that Eq. 17, 24 and 25 need, from a stored
 * Q(beta):  sum_i {(y_i)^2 - 2 y_i D_i^T E[beta_i] + D_i^T E[beta_i beta_i^T] D_i}
 * (y_i = r_i - mu_i), sum_i E[beta_i], sum_i E[beta_i beta_i^T] (Eq. 26-27)
 * and sum_i ln|Sigma_i| for the entropy of Q(beta). */
int vbo_sums_from_beta(const vbo_prior *p, int64_t V, const float *r, const float *d,
                       const double *mu, const double *Sig, vbo_sums *s)
{
    int S = p->S, M = S - 1;
    memset(s, 0, sizeof(*s));
    s->V = (double)V;
    for (int64_t i = 0; i < V; ++i) {
        double D[VBO_MMAX], yt, Ebb[VBO_MMAX * VBO_MMAX];
        const double *mi = mu + i * M, *Si = Sig + i * M * M;
        observation(S, r, d, i, D, &yt);
        for (int j = 0; j < M; ++j)
            for (int k = 0; k < M; ++k) Ebb[j * M + k] = mi[j] * mi[k] + Si[j * M + k];   /* Eq. 27 */
        double Dmu = 0.0, DEbbD = 0.0;
        for (int j = 0; j < M; ++j) {
            Dmu += D[j] * mi[j];
            for (int k = 0; k < M; ++k) DEbbD += D[j] * Ebb[j * M + k] * D[k];
        }
        s->sum_S += yt * yt - 2.0 * yt * Dmu + DEbbD;                                     /* Eq. 17 */
        for (int j = 0; j < M; ++j) s->sum_mu[j] += mi[j];                               /* Eq. 24 */
        for (int j = 0; j < M * M; ++j) s->sum_Ebb[j] += Ebb[j];                          /* Eq. 25 */
        double ld = 0.0;
        if (M > 0 && spd_logdet(M, Si, &ld)) return -1;
        s->sum_logdet += ld;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Q(rho) and Q(K, Lambda).                                                  */
/* ------------------------------------------------------------------------ */

/* Eq. 16-18: a_rho = a0 + V/2, b_rho = b0 + (1/2) sum of Eq. 17's braces. */
void vbo_rho_update(const vbo_prior *p, const vbo_sums *s, vbo_glob *g)
{
    g->a_rho = p->a0 + 0.5 * s->V;
    g->b_rho = p->b0 + 0.5 * s->sum_S;
}

/* Eq. 22-25:
 *   lam   = q0 + V,  nu = n0 + V
 *   kappa = (sum_i E[beta_i] + q0 K0) / (V + q0)
 *   Winv  = Lambda_0^{-1} + sum_i E[beta_i beta_i^T] + q0 K0 K0^T - (q0 + V) kappa kappa^T */
void vbo_KLambda_update(const vbo_prior *p, const vbo_sums *s, vbo_glob *g)
{
    int M = p->S - 1;
    double V = s->V;
    g->lam = p->q0 + V;
    g->nu = p->n0 + V;
    for (int j = 0; j < M; ++j) g->kappa[j] = (s->sum_mu[j] + p->q0 * p->K0[j]) / (V + p->q0);
    for (int j = 0; j < M; ++j)
        for (int k = 0; k < M; ++k)
            g->Winv[j * M + k] = p->L0inv[j * M + k] + s->sum_Ebb[j * M + k]
                               + p->q0 * p->K0[j] * p->K0[k]
                               - (p->q0 + V) * g->kappa[j] * g->kappa[k];
}

/* ------------------------------------------------------------------------ */
/* ELBO, Eq. 11: E_Q[ln P(r, Z)] - E_Q[ln Q(Z)] for the factorisation of      */
/* Eq. 13, expanded term by term.                                             */
/* ------------------------------------------------------------------------ */
int vbo_elbo(const vbo_prior *p, const vbo_sums *s, const vbo_glob *g, double *elbo, int *const_dropped)
{
    int M = p->S - 1;
    double V = s->V;
    double EL[VBO_MMAX * VBO_MMAX], lndetWinv = 0.0, lndetL0inv = 0.0;
    if (M > 0) {
        if (spd_inverse(M, g->Winv, EL, &lndetWinv)) return -1;
        if (spd_logdet(M, p->L0inv, &lndetL0inv)) return -1;
    }
    for (int j = 0; j < M * M; ++j) EL[j] *= g->nu;                    /* E[Lambda], Eq. 28 */
    double lndetW = -lndetWinv;
    double Erho = g->a_rho / g->b_rho;                                  /* Eq. 29 */
    double Elnrho = vbo_digamma(g->a_rho) - log(g->b_rho);
    double ElnL = wishart_Elndet(M, lndetW, g->nu);

    /* C = sum_i E[(beta_i - K0K)(beta_i - K0K)^T] under Q(beta) with K0K = kappa */
    double C[VBO_MMAX * VBO_MMAX];
    for (int j = 0; j < M; ++j)
        for (int k = 0; k < M; ++k)
            C[j * M + k] = s->sum_Ebb[j * M + k] - g->kappa[j] * s->sum_mu[k]
                         - s->sum_mu[j] * g->kappa[k] + V * g->kappa[j] * g->kappa[k];
    double trELC = 0.0, trL0EL = 0.0, quadK = 0.0;
    for (int j = 0; j < M; ++j)
        for (int k = 0; k < M; ++k) {
            trELC += EL[j * M + k] * C[k * M + j];
            trL0EL += p->L0inv[j * M + k] * EL[k * M + j];
            quadK += (g->kappa[j] - p->K0[j]) * EL[j * M + k] * (g->kappa[k] - p->K0[k]);
        }

    /* E ln P(r | beta, rho), Eq. 3 */
    double t_lik = 0.5 * V * (Elnrho - VBO_LN2PI) - 0.5 * Erho * s->sum_S;
    /* E ln P(beta | K, Lambda), Eq. 4; E over K | Lambda adds tr(Lambda (lam Lambda)^{-1}) = M / lam */
    double t_beta = 0.5 * V * (ElnL - M * VBO_LN2PI) - 0.5 * trELC - 0.5 * V * M / g->lam;
    /* E ln P(K | Lambda), Eq. 6 */
    double t_K = 0.5 * M * (log(p->q0) - VBO_LN2PI) + 0.5 * ElnL - 0.5 * p->q0 * (quadK + M / g->lam);
    /* E ln P(Lambda), Eq. 7: Wishart with scale Lambda_0 (= inverse of L0inv) */
    double t_Lam = 0.5 * (p->n0 - M - 1.0) * ElnL - 0.5 * trL0EL;
    int dropped = 0;
    if (M > 0) {
        if (p->n0 > M - 1.0) t_Lam += wishart_lnB(M, -lndetL0inv, p->n0);
        else dropped = 1;
    }
    /* E ln P(rho), Eq. 5 */
    double t_rho = p->a0 * log(p->b0) - lgamma(p->a0) + (p->a0 - 1.0) * Elnrho - p->b0 * Erho;
    /* entropies of Q(beta) (Gaussians), Q(K | Lambda), Q(Lambda) (Wishart), Q(rho) (Gamma) */
    double h_beta = 0.5 * s->sum_logdet + 0.5 * V * M * (1.0 + VBO_LN2PI);
    double h_K = -0.5 * ElnL - 0.5 * M * (log(g->lam) - VBO_LN2PI) + 0.5 * M;
    double h_Lam = M > 0 ? (-wishart_lnB(M, lndetW, g->nu) - 0.5 * (g->nu - M - 1.0) * ElnL + 0.5 * g->nu * M) : 0.0;
    double h_rho = g->a_rho - log(g->b_rho) + lgamma(g->a_rho) + (1.0 - g->a_rho) * vbo_digamma(g->a_rho);

    *elbo = t_lik + t_beta + t_K + t_Lam + t_rho + h_beta + h_K + h_Lam + h_rho;
    if (const_dropped) *const_dropped = dropped;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The whole iteration (Section 3.5).                                        */
/* ------------------------------------------------------------------------ */

/* Runs sweep 0 (Q(rho), Q(K, Lambda) and the ELBO from the initial Q(beta))
 * and then sweeps t = 1 .. max_iter of Q(beta) -> Q(rho) -> Q(K, Lambda) ->
 * ELBO, stopping after sweep t >= 1 when |L_t - L_{t-1}| < tol |L_t|.
 * trace (optional) receives L_0 .. L_iters.  Returns 0, -1 on a matrix that is
 * not positive definite, -2 on allocation failure. */
int vbo_fit(const vbo_prior *p, int64_t V, const float *r, const float *d, double tol, int max_iter,
            vbo_glob *g, double *trace, int *iters, int *converged, double *elbo_out, int *const_dropped)
{
    int M = p->S - 1;
    size_t nm = (size_t)(V > 0 ? V : 1) * (size_t)(M > 0 ? M : 1);
    double *mu = (double *)malloc(nm * sizeof(double));
    double *Sig = (double *)malloc(nm * (size_t)(M > 0 ? M : 1) * sizeof(double));
    int rc = 0;
    vbo_sums s;
    double L = 0.0, Lprev;
    *iters = 0;
    *converged = 0;
    if (!mu || !Sig) { rc = -2; goto done; }
    memset(g, 0, sizeof(*g));
    vbo_beta_init(p, V, mu, Sig);
    if (vbo_sums_from_beta(p, V, r, d, mu, Sig, &s)) { rc = -1; goto done; }
    vbo_rho_update(p, &s, g);
    vbo_KLambda_update(p, &s, g);
    if (vbo_elbo(p, &s, g, &L, const_dropped)) { rc = -1; goto done; }
    if (trace) trace[0] = L;
    for (int t = 1; t <= max_iter; ++t) {
        Lprev = L;
        if (vbo_beta_update(p, V, r, d, g, mu, Sig)) { rc = -1; goto done; }
        if (vbo_sums_from_beta(p, V, r, d, mu, Sig, &s)) { rc = -1; goto done; }
        vbo_rho_update(p, &s, g);
        vbo_KLambda_update(p, &s, g);
        if (vbo_elbo(p, &s, g, &L, const_dropped)) { rc = -1; goto done; }
        if (trace) trace[t] = L;
        *iters = t;
        if (fabs(L - Lprev) < tol * fabs(L)) { *converged = 1; break; }
    }
done:
    if (elbo_out) *elbo_out = L;
    free(mu);
    free(Sig);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Profile-grouped form.  Observations that share the whole profile d_i      */
/* share Lambda_{beta_i} (Eq. 20), and mu_{beta_i} (Eq. 21) is affine in      */
/* y_i = r_i - mu_i: mu_{beta_i} = a + b y_i with a = Sigma E[Lambda K] and   */
/* b = E[rho] Sigma D.  Every sum of vbo_sums_from_beta is then a polynomial  */
/* of degree <= 2 in y_i, so the per-group counts n, sum y and sum y^2 give   */
/* the same sums exactly (up to rounding).  init != 0 uses the initial        */
/* Q(beta_i) = N(K0, Lambda_0^{-1}) instead of Eq. 20-21.                    */
/* ------------------------------------------------------------------------ */
int vbo_sums_grouped(const vbo_prior *p, int P, const double *dprof, const double *n,
                     const double *sy, const double *syy, const vbo_glob *g, int init, vbo_sums *s)
{
    int S = p->S, M = S - 1;
    double EL[VBO_MMAX * VBO_MMAX], ELK[VBO_MMAX], Erho = 0.0;
    memset(s, 0, sizeof(*s));
    if (!init) {
        if (M > 0 && spd_inverse(M, g->Winv, EL, NULL)) return -1;
        for (int j = 0; j < M * M; ++j) EL[j] *= g->nu;
        for (int j = 0; j < M; ++j) {
            double t = 0.0;
            for (int k = 0; k < M; ++k) t += EL[j * M + k] * g->kappa[k];
            ELK[j] = t;
        }
        Erho = g->a_rho / g->b_rho;
    }
    for (int q = 0; q < P; ++q) {
        double D[VBO_MMAX], Sg[VBO_MMAX * VBO_MMAX], a[VBO_MMAX], b[VBO_MMAX], Lb[VBO_MMAX * VBO_MMAX];
        double dS = dprof[q * S + M];
        for (int j = 0; j < M; ++j) D[j] = dprof[q * S + j] - dS;
        if (init) {
            for (int j = 0; j < M; ++j) { a[j] = p->K0[j]; b[j] = 0.0; }
            for (int j = 0; j < M * M; ++j) Sg[j] = p->L0inv[j];
        } else {
            for (int j = 0; j < M; ++j)
                for (int k = 0; k < M; ++k) Lb[j * M + k] = EL[j * M + k] + Erho * D[j] * D[k];
            if (M > 0 && spd_inverse(M, Lb, Sg, NULL)) return -1;
            for (int j = 0; j < M; ++j) {
                double ta = 0.0, tb = 0.0;
                for (int k = 0; k < M; ++k) {
                    ta += Sg[j * M + k] * ELK[k];
                    tb += Sg[j * M + k] * D[k];
                }
                a[j] = ta;
                b[j] = Erho * tb;
            }
        }
        double nq = n[q], y1 = sy[q], y2 = syy[q];
        double Ebb[VBO_MMAX * VBO_MMAX];   /* sum over the group of E[beta beta^T] */
        double mus[VBO_MMAX];              /* sum over the group of E[beta] */
        for (int j = 0; j < M; ++j) {
            mus[j] = nq * a[j] + b[j] * y1;
            for (int k = 0; k < M; ++k)
                Ebb[j * M + k] = nq * Sg[j * M + k] + nq * a[j] * a[k] + (a[j] * b[k] + b[j] * a[k]) * y1
                               + b[j] * b[k] * y2;
        }
        double Da = 0.0, Db = 0.0, DEbbD = 0.0;
        for (int j = 0; j < M; ++j) {
            Da += D[j] * a[j];
            Db += D[j] * b[j];
            for (int k = 0; k < M; ++k) DEbbD += D[j] * Ebb[j * M + k] * D[k];
        }
        s->V += nq;
        s->sum_S += y2 - 2.0 * (Da * y1 + Db * y2) + DEbbD;
        for (int j = 0; j < M; ++j) s->sum_mu[j] += mus[j];
        for (int j = 0; j < M * M; ++j) s->sum_Ebb[j] += Ebb[j];
        double ld = 0.0;
        if (M > 0 && spd_logdet(M, Sg, &ld)) return -1;
        s->sum_logdet += nq * ld;
    }
    return 0;
}

/* vbo_fit on profile-grouped data: the same schedule as vbo_fit. */
int vbo_fit_grouped(const vbo_prior *p, int P, const double *dprof, const double *n, const double *sy,
                    const double *syy, double tol, int max_iter, vbo_glob *g, double *trace, int *iters,
                    int *converged, double *elbo_out, int *const_dropped)
{
    vbo_sums s;
    double L = 0.0, Lprev;
    *iters = 0;
    *converged = 0;
    memset(g, 0, sizeof(*g));
    if (vbo_sums_grouped(p, P, dprof, n, sy, syy, g, 1, &s)) return -1;
    vbo_rho_update(p, &s, g);
    vbo_KLambda_update(p, &s, g);
    if (vbo_elbo(p, &s, g, &L, const_dropped)) return -1;
    if (trace) trace[0] = L;
    for (int t = 1; t <= max_iter; ++t) {
        Lprev = L;
        if (vbo_sums_grouped(p, P, dprof, n, sy, syy, g, 0, &s)) return -1;
        vbo_rho_update(p, &s, g);
        vbo_KLambda_update(p, &s, g);
        if (vbo_elbo(p, &s, g, &L, const_dropped)) return -1;
        if (trace) trace[t] = L;
        *iters = t;
        if (fabs(L - Lprev) < tol * fabs(L)) { *converged = 1; break; }
    }
    if (elbo_out) *elbo_out = L;
    return 0;
}

/* ELBO of given global factors with Q(beta) set by Eq. 20-21 from them: one
 * Q(beta) update, then Eq. 11 with Q(rho), Q(K, Lambda) unchanged. */
int vbo_elbo_at(const vbo_prior *p, int64_t V, const float *r, const float *d, const vbo_glob *g,
                double *elbo, int *const_dropped)
{
    int M = p->S - 1;
    size_t nm = (size_t)(V > 0 ? V : 1) * (size_t)(M > 0 ? M : 1);
    double *mu = (double *)malloc(nm * sizeof(double));
    double *Sig = (double *)malloc(nm * (size_t)(M > 0 ? M : 1) * sizeof(double));
    int rc = 0;
    vbo_sums s;
    if (!mu || !Sig) { rc = -2; goto done; }
    if (vbo_beta_update(p, V, r, d, g, mu, Sig)) { rc = -1; goto done; }
    if (vbo_sums_from_beta(p, V, r, d, mu, Sig, &s)) { rc = -1; goto done; }
    if (vbo_elbo(p, &s, g, elbo, const_dropped)) rc = -1;
done:
    free(mu);
    free(Sig);
    return rc;
}

/* ======================================================================== */
/* Expectation maximisation (Section 4.2, Eq. 42-47).                        */
/* ======================================================================== */
/*
 * Point estimates theta = (K, Lambda^{-1}, rho) of the same model (Eq. 3-4),
 * beta_i integrated out.  Readings taken here:
 *   - Eq. 45-47 carry no prior terms: the iteration maximises the marginal
 *     likelihood p(r | theta) (maximum-likelihood EM).
 *   - The paper gives no starting point; theta^(0) is passed in (the CUDA
 *     path's default is the prior's K0, Lambda_0^{-1} and a0 / b0).
 *   - Iteration n evaluates ln p(r | theta^(n)) and then forms theta^(n+1); it
 *     stops after iteration n >= 1 when |L_n - L_{n-1}| < tol |L_n|.
 */
typedef struct {
    double rho;                         /* noise precision */
    double K[VBO_MMAX];                 /* mean of beta_i */
    double Linv[VBO_MMAX * VBO_MMAX];   /* Lambda^{-1}, row-major M x M */
} vbo_em;

/* ln p(r | theta) = sum_i ln N(r_i; D_i^T K + mu_i, 1/rho + D_i^T Lambda^{-1} D_i)
 * (the marginal of Eq. 3 under Eq. 4), summed in observation order. */
int vbo_em_loglik(int S, int64_t V, const float *r, const float *d, const vbo_em *t, double *ll)
{
    const int M = S - 1;
    if (!(t->rho > 0.0)) return -1;
    double sum = 0.0;
    for (int64_t i = 0; i < V; ++i) {
        const float *di = d + (size_t)i * (size_t)S;
        const double dS = (double)di[M];
        double D[VBO_MMAX];
        for (int j = 0; j < M; ++j) D[j] = (double)di[j] - dS;
        double mean = dS, var = 1.0 / t->rho;
        for (int j = 0; j < M; ++j) {
            mean += D[j] * t->K[j];
            for (int k = 0; k < M; ++k) var += D[j] * t->Linv[j * M + k] * D[k];
        }
        const double e = (double)r[i] - mean;
        sum += -0.5 * (VBO_LN2PI + log(var) + e * e / var);
    }
    *ll = sum;
    return 0;
}

/* One EM iteration from theta_in: for every i, Sigma_i = [Lambda + rho D_i D_i^T]^{-1}
 * by an explicit inverse (Eq. 42), M_i (Eq. 43) and S_i (Eq. 44); then rho
 * (Eq. 45), K (Eq. 46) and Lambda^{-1} (Eq. 47). */
int vbo_em_step(int S, int64_t V, const float *r, const float *d, const vbo_em *in, vbo_em *out)
{
    const int M = S - 1;
    double Lam[VBO_MMAX * VBO_MMAX], LamK[VBO_MMAX];
    if (M > 0 && spd_inverse(M, in->Linv, Lam, NULL)) return -1;
    for (int j = 0; j < M; ++j) {
        double s = 0.0;
        for (int k = 0; k < M; ++k) s += Lam[j * M + k] * in->K[k];
        LamK[j] = s;
    }
    double sumS = 0.0, sumM[VBO_MMAX], sumMM[VBO_MMAX * VBO_MMAX];
    for (int j = 0; j < M; ++j) sumM[j] = 0.0;
    for (int j = 0; j < M * M; ++j) sumMM[j] = 0.0;
    for (int64_t i = 0; i < V; ++i) {
        const float *di = d + (size_t)i * (size_t)S;
        const double dS = (double)di[M];
        const double y = (double)r[i] - dS;                     /* r_i - mu_i */
        double D[VBO_MMAX], P[VBO_MMAX * VBO_MMAX], Sig[VBO_MMAX * VBO_MMAX], rhs[VBO_MMAX], Mi[VBO_MMAX];
        for (int j = 0; j < M; ++j) D[j] = (double)di[j] - dS;
        for (int j = 0; j < M; ++j)                              /* Lambda + rho D D^T */
            for (int k = 0; k < M; ++k) P[j * M + k] = Lam[j * M + k] + in->rho * D[j] * D[k];
        if (M > 0 && spd_inverse(M, P, Sig, NULL)) return -1;   /* Eq. 42 */
        for (int j = 0; j < M; ++j) rhs[j] = LamK[j] + in->rho * D[j] * y;
        for (int j = 0; j < M; ++j) {                            /* Eq. 43 */
            double s = 0.0;
            for (int k = 0; k < M; ++k) s += Sig[j * M + k] * rhs[k];
            Mi[j] = s;
        }
        double DM = 0.0, DQD = 0.0;                              /* Eq. 44 */
        for (int j = 0; j < M; ++j) {
            DM += D[j] * Mi[j];
            for (int k = 0; k < M; ++k) DQD += D[j] * (Mi[j] * Mi[k] + Sig[j * M + k]) * D[k];
        }
        sumS += y * y - 2.0 * y * DM + DQD;
        for (int j = 0; j < M; ++j) {
            sumM[j] += Mi[j];
            for (int k = 0; k < M; ++k) sumMM[j * M + k] += Mi[j] * Mi[k] + Sig[j * M + k];
        }
    }
    if (!(sumS > 0.0)) return -1;
    const double Vd = (double)V;
    out->rho = Vd / sumS;                                        /* Eq. 45 */
    for (int j = 0; j < M; ++j) out->K[j] = sumM[j] / Vd;        /* Eq. 46 */
    for (int j = 0; j < M; ++j)                                  /* Eq. 47 */
        for (int k = 0; k < M; ++k) out->Linv[j * M + k] = sumMM[j * M + k] / Vd - out->K[j] * out->K[k];
    for (int j = 0; j < M; ++j)
        for (int k = 0; k < j; ++k) {
            const double a = 0.5 * (out->Linv[j * M + k] + out->Linv[k * M + j]);
            out->Linv[j * M + k] = a;
            out->Linv[k * M + j] = a;
        }
    return 0;
}

/* EM from theta0: trace[n] = ln p(r | theta^(n)) for n = 0..*iters; *out =
 * theta^(*iters + 1). */
int vbo_em_fit(int S, int64_t V, const float *r, const float *d, const vbo_em *theta0, double tol, int max_iter,
               vbo_em *out, double *trace, int *iters, int *converged)
{
    vbo_em cur = *theta0, nxt;
    double L = 0.0, Lprev = 0.0;
    *iters = 0;
    *converged = 0;
    for (int n = 0; n <= max_iter; ++n) {
        if (vbo_em_loglik(S, V, r, d, &cur, &L)) return -1;
        if (trace) trace[n] = L;
        if (vbo_em_step(S, V, r, d, &cur, &nxt)) return -1;
        cur = nxt;
        *iters = n;
        if (n >= 1 && fabs(L - Lprev) < tol * fabs(L)) {
            *converged = 1;
            break;
        }
        Lprev = L;
    }
    *out = cur;
    return 0;
}
