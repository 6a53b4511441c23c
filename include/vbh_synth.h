/*
 * vbh_synth.h -- C ABI of the seeded synthetic-input generator (device side).
 *
 * The paper has no counterpart of this library: it draws test and benchmark
 * inputs from the generative model of Eq. 3-4 (Section 4 experiments), so
 * that the CUDA path and the CPU oracle can be fed the same arrays.  It holds
 * none of the arithmetic of the variational method.  The recipe (Philox4x32-10
 * counters per observation, Box-Muller normals) is documented in
 * paper_2401_10068_gb300/synth/__init__.py, whose host implementation returns
 * the same values.
 */
#ifndef VBH_SYNTH_H
#define VBH_SYNTH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Write observations start .. start + V - 1 of the data set keyed by `seed`
 * into device buffers r (V floats) and d (V x S floats, row-major), on
 * `stream` (a cudaStream_t), and wait for completion.
 *   K_true: S - 1 doubles (host), the mean of beta_i (Eq. 4);
 *   L_beta: (S - 1) x (S - 1) doubles (host, row-major), lower Cholesky factor
 *           of the covariance of beta_i;
 *   rho:    noise precision (Eq. 3), > 0;
 *   p_const: probability of a constant profile (all zeros or all ones).
 * Returns 0, -1 for an invalid argument, -3 for a CUDA error. */
int vbh_synth_generate(float *r, float *d, int64_t V, int S, int64_t start, uint64_t seed, const double *K_true,
                       const double *L_beta, double rho, double p_const, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* VBH_SYNTH_H */
