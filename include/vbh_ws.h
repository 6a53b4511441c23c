/*
 * vbh_ws.h -- learned warm start for the CAVI fit: a set encoder that maps a
 * data set to a starting point of the iteration (the paper starts every fit
 * from the prior, Section 3.5; this entry replaces that start and the fit
 * falls back to it when no model is used).
 *
 * The encoder works for one number of subpopulations S (M = S - 1).  Per
 * observation the feature vector x_i = [D_i (M), y_i, y_i^2, y_i D_i (M)]
 * (D_i = d_{i,1:M} - d_{i,S}, y_i = r_i - d_{i,S}; F = 2M + 2 values) goes
 * through phi(x) = GELU(W2 GELU(W1 x + b1) + b2) (hidden width H); phi is
 * averaged over the observations; the head GELU(W3 p + b3) -> W4 (.) + b4 gives
 * P = M + 1 + M(M+1)/2 outputs, standardised by a per-output mean and
 * standard deviation: kappa (M), ln E[rho] (1) and the Cholesky factor L of
 * Sigma0 = E[Lambda]^{-1} packed row by row (L_jk for k <= j, the diagonal as
 * ln L_jj).  GELU(z) = z Phi(z).  Matrices are held in BF16 for the forward
 * and backward passes (FP32 accumulation) and in FP32 for the optimiser.
 *
 * Conventions as in vbh.h: 0 or a negative VBH_E* status; calls are
 * synchronous on the model's stream; device pointers are 16-byte aligned CUDA
 * allocations on the model's device; the caller owns every buffer it passes.
 * Parameters: one flat FP32 vector W1 (H x F), b1 (H), W2 (H x H), b2 (H),
 * W3 (H x H), b3 (H), W4 (P x H), b4 (P), matrices row-major.
 */
#ifndef VBH_WS_H
#define VBH_WS_H

#include <stddef.h>
#include <stdint.h>

#include "vbh.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vbh_ws vbh_ws;

/* New encoder for S subpopulations (2 <= S <= 11) and hidden width H (a
 * multiple of 64, <= 1024), weights drawn uniformly in +-sqrt(6 / (fan_in +
 * fan_out)) from a counter-based hash of `seed`, biases 0, standardisation
 * mean 0 and deviation 1. */
int vbh_ws_create(vbh_ws **m, int S, int hidden, uint64_t seed, int device, void *stream);
void vbh_ws_destroy(vbh_ws *m);

/* Feature width F, output width P and number of parameters. */
int vbh_ws_sizes(const vbh_ws *m, int *F, int *P, size_t *nparams);

/* Copy the FP32 parameters out or in (host arrays of nparams floats); setting
 * them refreshes the BF16 copies and resets the optimiser state. */
int vbh_ws_get_params(vbh_ws *m, float *host, size_t n);
int vbh_ws_set_params(vbh_ws *m, const float *host, size_t n);

/* Output standardisation (host arrays of P floats, std > 0): the model's raw
 * outputs are (target - mean) / std. */
int vbh_ws_set_norm(vbh_ws *m, const float *mean, const float *std);

/* Features of n (<= 2^20) evenly spaced observations of (r, d) (device pointers, V >= 1):
 * observation floor(j V / n) for j = 0..n-1 -> x (device, n x F floats). */
int vbh_ws_features(vbh_ws *m, const float *r, const float *d, int64_t V, int n, float *x);

/* Raw outputs of B sets of n observations each (B n <= 2^20): x (device,
 * B x n x F) -> out (device, B x P). */
int vbh_ws_forward(vbh_ws *m, int B, int n, const float *x, float *out);

/* Mean squared error of the raw outputs against target (device, B x P) and
 * its gradient in the parameters (host array of nparams floats, may be NULL). */
int vbh_ws_loss_grad(vbh_ws *m, int B, int n, const float *x, const float *target, double *loss, float *grad);

/* One Adam step (beta1 = 0.9, beta2 = 0.999, eps = 1e-8, learning rate lr) on
 * that loss; *loss receives the loss before the step. */
int vbh_ws_train_step(vbh_ws *m, int B, int n, const float *x, const float *target, float lr, double *loss);

/* Starting point of a CAVI fit of (r, d) (device pointers, V observations,
 * prior p) from the encoder applied to n evenly spaced observations, as a
 * vbh_result for vbh_opts.init = VBH_INIT_GIVEN: kappa, W_inv = nu Sigma0 with
 * nu = n0 + V, lambda = q0 + V, a_rho = a0 + V/2, b_rho = a_rho / E[rho]. */
int vbh_ws_predict(vbh_ws *m, const float *r, const float *d, int64_t V, const vbh_prior *p, int n,
                   vbh_result *init);

#ifdef __cplusplus
}
#endif

#endif /* VBH_WS_H */
