/*
 * vbh_ws.h -- learned warm start for the CAVI fit: a permutation-invariant set
 * encoder that maps a data set to a starting point of the iteration.  The
 * paper starts every fit from the prior (initialisation paragraph of Section
 * 3.5) and reports that restarts reach the same optimum (Section 4.3); this
 * entry replaces that start, and a fit without it falls back to it.  The
 * paper has no counterpart of the encoder itself.
 *
 * One encoder serves every S in 2..VBH_WS_SMAX (masked).  Per observation i of
 * a data set with S subpopulations (M = S - 1, D_i = d_{i,1:M} - d_{i,S},
 * y_i = r_i - d_{i,S}) the feature vector has VBH_WS_F = 64 slots:
 *   slots  0..8   D_ij (j < M; 0 beyond)
 *   slots  9..17  1 for j < M, 0 beyond (the mask: tells the encoder S)
 *   slot  18      y_i
 *   slot  19      y_i^2
 *   slots 20..28  y_i D_ij
 *   slots 29..37  y_i^2 D_ij
 *   slots 38..63  0
 * phi(x) = GELU(W2 GELU(W1 x + b1) + b2) (hidden width H = 256) is averaged
 * over the observations used; the head GELU(W3 p + b3) -> W4 (.) + b4 gives
 * VBH_WS_P = 64 output slots, standardised per S by a mean and deviation:
 *   slots  0..8   kappa_j (j < M)
 *   slot   9      ln E[rho]
 *   slots 10..54  the Cholesky factor L of Sigma0 = E[Lambda]^{-1}: entry
 *                 (j, k), k <= j < M, at slot 10 + j (j + 1) / 2 + k, the
 *                 diagonal as ln L_jj
 *   other slots   unused (loss weight 0).
 * GELU is the tanh form z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))) / 2.
 *
 * Arithmetic.  The per-observation layers run on the tensor cores (tcgen05
 * MMAs, BF16 operands, FP32 accumulation in tensor memory) with the bias,
 * GELU and the mean pool applied in the MMA epilogue; the features and the
 * hidden activations between the two layers are BF16; the backward pass
 * (layer 2 recomputed with its GELU derivative in the epilogue, the input
 * gradient of layer 2, the weight gradients over the observations) runs on
 * the same kernels.  The head (one row per data set) is FP32 on the CUDA
 * cores.  Weights are FP32 master copies (Adam) with BF16 copies for the
 * MMAs.  Sums over observations and data sets are taken in a fixed order:
 * every result is run-to-run identical.
 *
 * Conventions as in vbh.h: 0 or a negative VBH_E* status; calls are
 * synchronous on the model's stream; device pointers are 16-byte aligned CUDA
 * allocations on the model's device; the caller owns every buffer.
 * Parameters: one flat FP32 vector W1 (H x F), b1 (H), W2 (H x H), b2 (H),
 * W3 (H x H), b3 (H), W4 (P x H), b4 (P), matrices row-major.
 *
 * A batch of B data sets is given as host arrays of B entries: r[b], d[b]
 * (device pointers, V[b] floats and V[b] x S[b] floats row-major), V[b] >= 1,
 * S[b] in 2..VBH_WS_SMAX, and n[b], the number of observations the encoder
 * pools (n[b] = 0 or n[b] >= V[b]: all; else observations floor(j V[b] /
 * n[b]), j = 0..n[b]-1).  The pooled observations of one call must not
 * exceed 2^26 in total (VBH_EINVAL).
 */
#ifndef VBH_WS_H
#define VBH_WS_H

#include <stddef.h>
#include <stdint.h>

#include "vbh.h"

#ifdef __cplusplus
extern "C" {
#endif

#define VBH_WS_SMAX 10
#define VBH_WS_F 64
#define VBH_WS_P 64
#define VBH_WS_HIDDEN 256

typedef struct vbh_ws vbh_ws;

/* New encoder (H = VBH_WS_HIDDEN): weights drawn uniformly in +-sqrt(6 / (fan_in
 * + fan_out)) from a counter-based hash of `seed`, biases 0, standardisation
 * mean 0 and deviation 1. */
int vbh_ws_create(vbh_ws **m, uint64_t seed, int device, void *stream);
void vbh_ws_destroy(vbh_ws *m);

/* Number of parameters. */
size_t vbh_ws_num_params(const vbh_ws *m);

/* Copy the FP32 parameters out or in (host arrays of num_params floats);
 * setting them refreshes the BF16 copies and resets the optimiser state. */
int vbh_ws_get_params(vbh_ws *m, float *host, size_t n);
int vbh_ws_set_params(vbh_ws *m, const float *host, size_t n);

/* Output standardisation, host arrays of (VBH_WS_SMAX + 1) x VBH_WS_P floats
 * (row S; rows 0 and 1 unused; deviations > 0): raw output = (target - mean)
 * / std. */
int vbh_ws_set_norm(vbh_ws *m, const float *mean, const float *std);

/* Features of the pooled observations of one data set (device, n x VBH_WS_F
 * floats, row-major; n as for a batch entry) -- the encoder's input, for
 * checking. */
int vbh_ws_features(vbh_ws *m, const float *r, const float *d, int64_t V, int S, int64_t n, float *x);

/* Raw outputs (device, B x VBH_WS_P floats) of a batch. */
int vbh_ws_forward(vbh_ws *m, int B, const float *const *r, const float *const *d, const int64_t *V, const int *S,
                   const int64_t *n, float *out);

/* Loss sum_b sum_p w_bp (out_bp - t_bp)^2 / B against standardised targets t
 * and weights w (device, B x VBH_WS_P each) and its gradient in the
 * parameters (host array of num_params floats, may be NULL). */
int vbh_ws_loss_grad(vbh_ws *m, int B, const float *const *r, const float *const *d, const int64_t *V,
                     const int *S, const int64_t *n, const float *target, const float *weight, double *loss,
                     float *grad);

/* One Adam step (beta1 = 0.9, beta2 = 0.999, eps = 1e-8, learning rate lr) on
 * that loss; *loss receives the loss before the step. */
int vbh_ws_train_step(vbh_ws *m, int B, const float *const *r, const float *const *d, const int64_t *V,
                      const int *S, const int64_t *n, const float *target, const float *weight, float lr,
                      double *loss);

/* Starting points of CAVI fits of a batch (all observations pooled), as
 * vbh_results for vbh_opts.init = VBH_INIT_GIVEN: kappa, W_inv = nu Sigma0
 * with nu = n0 + V, lambda = q0 + V, a_rho = a0 + V/2, b_rho = a_rho / E[rho]
 * (p: B priors, or NULL for the default of each S).  A data set whose
 * prediction is not finite gets the status VBH_ENONFINITE in its result and
 * the call returns it. */
int vbh_ws_predict(vbh_ws *m, int B, const float *const *r, const float *const *d, const int64_t *V,
                   const int *S, const vbh_prior *p, vbh_result *init);

#ifdef __cplusplus
}
#endif

#endif /* VBH_WS_H */
