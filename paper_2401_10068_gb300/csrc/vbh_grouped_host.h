// vbh_grouped_host.h -- host interface of the profile-grouped sweep (binary
// profiles, S <= GROUPED_SMAX).
#pragma once

#include <cuda_runtime.h>

#include "vbh_internal.cuh"

namespace vbh {

constexpr int GROUPED_SMAX = 16;             // 2^16 profile codes at most
constexpr int GROUPED_THREADS = 256;

// Kernel arguments of the grouped sweep.
struct GroupArgs {
    SweepArgs sa;                            // V, st, partials, cond, use_cond, mode (r and d unused)
    const double *stats;                     // [P][3]: n, sum y, sum y^2 per profile code (y = r - d_S)
    int P;                                   // 2^S
};

// From this S on the sweep takes 32 codes per warp (lane = code).
constexpr int GROUPED_WIDE_S = 12;

// The grouped sweep kernel for S, its grid (8 warps per block; up to one block
// per SM, two for the wide form) and its dynamic shared memory (the same for
// every S).
const void *grouped_sweep_func(int S);
int grouped_grid(int S, int nsm);
size_t grouped_smem_bytes();

// stats (3 * 2^S doubles, device, zeroed by the caller) += per-code counts and
// FP64 sums of y and y^2, code = sum_j d_ij 2^j; *nonbinary_dev (device) gains
// the number of profile values other than 0 and 1.
int grouped_histogram(const float *r, const float *d, long long V, int S, double *stats,
                      unsigned long long *nonbinary_dev, cudaStream_t stream, int nsm);

} // namespace vbh
