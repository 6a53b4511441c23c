// vbh_tc.cu -- instantiations and host helpers of the tensor-core sweep
// (12 <= S <= 32): the runtime-S set-up kernel and the repacking of the
// inputs into BF16 tiles.
#include <cuda_runtime.h>

#include "vbh.h"
#include "vbh_error.h"
#include "vbh_tc.cuh"
#include "vbh_tc_host.h"

namespace vbh {

// Set-up of one state of any M (runtime), one warp.
__global__ void setup_kernel_rt(DevState *st, int init)
{
    __shared__ double A[MMAX * MMAX], Lc[MMAX * MMAX];
    if (threadIdx.x >= 32) return;
    setup_state_rt(st->M, st, init, threadIdx.x, A, Lc);
}

bool tc_kernel_info(int nsplit, TcKernelInfo *out)
{
    switch (nsplit) {
    case 2:
        out->sweep = reinterpret_cast<const void *>(&tc_sweep_kernel<2>);
        out->smem = TcCfg<2>::SMEM_BYTES;
        out->threads = TcCfg<2>::THREADS;
        break;
    case 3:
        out->sweep = reinterpret_cast<const void *>(&tc_sweep_kernel<3>);
        out->smem = TcCfg<3>::SMEM_BYTES;
        out->threads = TcCfg<3>::THREADS;
        break;
    default:
        return false;
    }
    out->setup = reinterpret_cast<const void *>(&setup_kernel_rt);
    out->tile = 2 * TcCfg<2>::TILE;                 // a block takes pairs of tiles
    return true;
}

int tc_convert_inputs(const float *d, const float *r, long long V, int S, void *buf, unsigned long long *counts_dev,
                      cudaStream_t stream, int nsm)
{
    if (V == 0) return VBH_OK;
    const long long ntiles = tc_tiles(V);
    const long long work = ntiles * 16 * 32;
    long long blocks = (work + 255) / 256;
    if (blocks > 16LL * nsm) blocks = 16LL * nsm;
    tc_inputs_kernel<<<int(blocks), 256, 0, stream>>>(d, r, V, S, ntiles, static_cast<unsigned char *>(buf),
                                                      counts_dev);
    VBH_CHECK_CUDA(cudaGetLastError());
    return VBH_OK;
}

} // namespace vbh
