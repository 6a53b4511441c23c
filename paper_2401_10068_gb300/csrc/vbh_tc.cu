// vbh_tc.cu -- instantiations and host helpers of the tensor-core sweep
// (12 <= S <= 32): the runtime-S set-up kernel, the BF16 conversion of the
// profiles (with a padded copy of r) and the tensor map of the profiles.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdio>

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
    out->tile = TcCfg<2>::TILE;
    return true;
}

int tc_convert_inputs(const float *d, const float *r, long long V, int S, void *buf, unsigned long long *counts_dev,
                      cudaStream_t stream, int nsm)
{
    if (V == 0) return VBH_OK;
    const long long Vp = tc_padded(V);
    long long blocks = (Vp * 32 + 255) / 256;
    if (blocks > 16LL * nsm) blocks = 16LL * nsm;
    tc_inputs_kernel<<<int(blocks), 256, 0, stream>>>(d, r, V, Vp, S, static_cast<__nv_bfloat16 *>(buf),
                                                      const_cast<float *>(tc_r_pad(buf, V)), counts_dev);
    VBH_CHECK_CUDA(cudaGetLastError());
    return VBH_OK;
}

namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        const cudaError_t e =
            cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess) {
            char buf[96];
            std::snprintf(buf, sizeof(buf), "%s, query result %d", cudaGetErrorName(e), int(q));
            record_error("cudaGetDriverEntryPointByVersion(cuTensorMapEncodeTiled)", __FILE__, __LINE__, buf);
            (void)cudaGetLastError();
            return nullptr;
        }
        fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}
} // namespace

// Profiles: BF16 [Vp rows x 32 components], box 32 x 128 rows, 64-byte
// swizzle (the layout the kernel's MMAs read).
int tc_encode_tensor_map(const void *buf, long long V, void *tmap_d)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return VBH_ECUDA;
    if (V <= 0 || V >= (1LL << 31)) return VBH_EINVAL;
    const cuuint64_t dimd[2] = {32, cuuint64_t(tc_padded(V))};
    const cuuint64_t strd[1] = {64};
    const cuuint32_t boxd[2] = {32, 128};
    const cuuint32_t es[2] = {1, 1};
    const CUresult cr = fn(static_cast<CUtensorMap *>(tmap_d), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                           const_cast<void *>(buf), dimd, strd, boxd, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) {
        char msg[32];
        std::snprintf(msg, sizeof(msg), "CUresult %d", int(cr));
        record_error("cuTensorMapEncodeTiled(profiles)", __FILE__, __LINE__, msg);
        return VBH_ECUDA;
    }
    return VBH_OK;
}

} // namespace vbh
