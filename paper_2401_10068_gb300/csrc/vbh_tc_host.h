// vbh_tc_host.h -- host interface of the tensor-core sweep (12 <= S <= 32).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "vbh_internal.cuh"

namespace vbh {

// Bytes of one input tile of the tensor-core sweep: 128 observations, the
// BF16 slots of D = d_{1:M} - d_S (32 slots x 128 observations, in the kernel's
// shared-memory order) then y = r - d_S (128 x 4).
constexpr unsigned TC_TILE_BYTES = 128 * 64 + 128 * 4;

// Kernel arguments of the tensor-core sweep.
struct TcArgs {
    SweepArgs sa;                  // V, st, partials, cond, use_cond, mode (r and d unused)
    const unsigned char *tiles;    // the repacked inputs (tc_convert_inputs)
    int S;
    int binary;                    // 1: every D value is -1, 0 or 1
};

struct TcKernelInfo {
    const void *sweep;     // tc_sweep_kernel<NSPLIT>
    const void *setup;     // setup_kernel_rt
    size_t smem;
    int threads;
    int tile;
};

// Kernel of the tensor-core sweep with NSPLIT = 2 (BF16 form, 16-bit globals)
// or 3 (FP32-exact globals).
bool tc_kernel_info(int nsplit, TcKernelInfo *out);

// Tiles of the repacked inputs of V observations (an even number).
inline long long tc_tiles(long long V) { return ((V + 127) / 128 + 1) / 2 * 2; }

// Device bytes of the repacked inputs of V observations.
inline size_t tc_input_bytes(long long V) { return size_t(tc_tiles(V)) * TC_TILE_BYTES; }

// d (V x S FP32) and r (V FP32), device -> buf (tc_input_bytes(V) bytes,
// device), in tiles of 128 observations.  counts_dev[0] (device) gains the
// number of D = d_j - d_S values BF16 does not represent exactly, counts_dev[1]
// the number other than -1, 0 and 1.
int tc_convert_inputs(const float *d, const float *r, long long V, int S, void *buf, unsigned long long *counts_dev,
                      cudaStream_t stream, int nsm);

} // namespace vbh
