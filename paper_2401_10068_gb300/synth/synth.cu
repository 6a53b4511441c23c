// synth.cu -- device implementation of the seeded synthetic-input recipe of
// paper_2401_10068_gb300/synth/__init__.py (library libvbh_synth.so, C ABI in
// include/vbh_synth.h).  It draws data from the generative model of Eq. 3-4
// only; no arithmetic of the variational method is here.
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): key (seed lo, seed hi),
// counter (i lo, i hi, block, 0).  Block 0 gives the profile bits and the
// constant-profile selector, blocks >= 1 give Box-Muller normals.  FP64
// arithmetic uses explicit round-to-nearest operations in the same order as
// the host implementation so that both produce the same values.
#include <cuda_runtime.h>
#include <stdint.h>

#include "vbh_synth.h"

namespace {

constexpr int SMAX = 32;

struct SynthParams {
    double K[SMAX];
    double L[SMAX * SMAX];      // Cholesky factor of Sigma_beta, row-major (M x M)
    double inv_sqrt_rho;
    double p_const;
};

__device__ __forceinline__ void philox(uint32_t c[4], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t p0 = uint64_t(0xD2511F53u) * c[0];
        const uint64_t p1 = uint64_t(0xCD9E8D57u) * c[2];
        const uint32_t n0 = uint32_t(p1 >> 32) ^ c[1] ^ k0;
        const uint32_t n1 = uint32_t(p1);
        const uint32_t n2 = uint32_t(p0 >> 32) ^ c[3] ^ k1;
        const uint32_t n3 = uint32_t(p0);
        c[0] = n0;
        c[1] = n1;
        c[2] = n2;
        c[3] = n3;
    }
}

__device__ __forceinline__ double unif(uint32_t x)
{
    return __dmul_rn(__dadd_rn(double(x), 0.5), 2.3283064365386963e-10);   // (x + 1/2) 2^-32
}

__global__ void synth_kernel(float *r, float *d, long long V, int S, long long start, uint32_t k0, uint32_t k1,
                             const SynthParams *__restrict__ P)
{
    const int M = S - 1;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < V;
         n += (long long)gridDim.x * blockDim.x) {
        const unsigned long long i = (unsigned long long)(start + n);
        uint32_t c[4] = {uint32_t(i), uint32_t(i >> 32), 0u, 0u};
        philox(c, k0, k1);
        double bits[SMAX];
        const bool cst = unif(c[1]) < P->p_const;
        const double cv = double(c[2] & 1u);
        for (int j = 0; j < S; ++j) bits[j] = cst ? cv : double((c[0] >> j) & 1u);
        double z[SMAX + 4];
        const int nblk = (S + 3) / 4;
        for (int b = 0; b < nblk; ++b) {
            uint32_t y[4] = {uint32_t(i), uint32_t(i >> 32), uint32_t(b + 1), 0u};
            philox(y, k0, k1);
            for (int h = 0; h < 2; ++h) {
                const double R = sqrt(__dmul_rn(-2.0, log(unif(y[2 * h]))));
                const double t = __dmul_rn(6.283185307179586, unif(y[2 * h + 1]));
                double sn, cs;
                sincos(t, &sn, &cs);
                z[4 * b + 2 * h] = __dmul_rn(R, cs);
                z[4 * b + 2 * h + 1] = __dmul_rn(R, sn);
            }
        }
        const double dS = bits[M];
        double acc = 0.0;
        for (int j = 0; j < M; ++j) {
            double bj = P->K[j];
            for (int k = 0; k <= j; ++k) bj = __dadd_rn(bj, __dmul_rn(P->L[j * M + k], z[k]));
            acc = __dadd_rn(acc, __dmul_rn(__dadd_rn(bits[j], -dS), bj));
        }
        const double rr = __dadd_rn(__dadd_rn(acc, dS), __dmul_rn(z[M], P->inv_sqrt_rho));
        r[n] = __double2float_rn(rr);
        for (int j = 0; j < S; ++j) d[n * S + j] = float(bits[j]);
    }
}

} // namespace

extern "C" int vbh_synth_generate(float *r, float *d, int64_t V, int S, int64_t start, uint64_t seed,
                                  const double *K_true, const double *L_beta, double rho, double p_const,
                                  void *stream)
{
    if (S < 1 || S > SMAX || V < 0 || start < 0 || !(rho > 0.0) || !(p_const >= 0.0)) return -1;
    if (V == 0) return 0;
    if (!r || !d || (S > 1 && (!K_true || !L_beta))) return -1;
    const int M = S - 1;
    SynthParams hp{};
    for (int j = 0; j < M; ++j) hp.K[j] = K_true[j];
    for (int j = 0; j < M * M; ++j) hp.L[j] = L_beta[j];
    hp.inv_sqrt_rho = 1.0 / __builtin_sqrt(rho);
    hp.p_const = p_const;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    SynthParams *dp = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void **>(&dp), sizeof(SynthParams), s) != cudaSuccess) return -3;
    int rc = 0;
    if (cudaMemcpyAsync(dp, &hp, sizeof(hp), cudaMemcpyHostToDevice, s) != cudaSuccess) rc = -3;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (!rc) {
        long long blocks = (V + 255) / 256;
        if (blocks > 16LL * nsm) blocks = 16LL * nsm;
        synth_kernel<<<int(blocks), 256, 0, s>>>(r, d, V, S, start, uint32_t(seed), uint32_t(seed >> 32), dp);
        if (cudaGetLastError() != cudaSuccess) rc = -3;
    }
    cudaFreeAsync(dp, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = -3;
    return rc;
}
