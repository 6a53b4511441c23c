// vbh_tc_host.h -- host interface of the tensor-core sweep (12 <= S <= 32).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "vbh_internal.cuh"

namespace vbh {

// Kernel arguments of the tensor-core sweep (the tensor maps are passed beside them).
struct TcArgs {
    SweepArgs sa;          // r = the padded r copy; V, st, partials, cond, use_cond, mode (d unused: tensor map)
    int S;
    int binary;            // 1: every profile value is 0 or 1
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

// Observations padded to whole tiles of 128.
inline long long tc_padded(long long V) { return (V + 127) / 128 * 128; }

// Device bytes of the converted inputs of V observations: BF16 profiles
// (tc_padded(V) x 64 bytes) followed by the padded r (tc_padded(V) floats).
inline size_t tc_input_bytes(long long V) { return size_t(tc_padded(V)) * 68; }

// d (V x S FP32) and r (V FP32), device -> buf (tc_input_bytes(V) bytes,
// device).  counts_dev[0] (device) gains the number of profile values BF16
// does not represent exactly, counts_dev[1] the number other than 0 and 1.
int tc_convert_inputs(const float *d, const float *r, long long V, int S, void *buf, unsigned long long *counts_dev,
                      cudaStream_t stream, int nsm);

// The padded r inside buf.
inline const float *tc_r_pad(const void *buf, long long V)
{
    return reinterpret_cast<const float *>(static_cast<const unsigned char *>(buf) + size_t(tc_padded(V)) * 64);
}

// Tensor map (CUtensorMap, 128 bytes) of the BF16 profiles in buf.
int tc_encode_tensor_map(const void *buf, long long V, void *tmap_d);


} // namespace vbh
