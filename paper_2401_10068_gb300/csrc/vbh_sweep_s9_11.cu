// Instantiations of the fused sweep (single and batched forms) for S in {9, 10, 11}.
#include "vbh_batched.cuh"
#include "vbh_sweep.cuh"
#include "vbh_resident.cuh"
#include "vbh_dispatch.cuh"

namespace vbh {

bool kernel_info_s9_11(int S, KernelInfo *out)
{
    switch (S) {
        VBH_KERNEL_INFO_CASE(9)
        VBH_KERNEL_INFO_CASE(10)
        VBH_KERNEL_INFO_CASE(11)
    default:
        return false;
    }
}

bool batch_kernel_info_s9_11(int S, BatchKernelInfo *out)
{
    switch (S) {
        VBH_BATCH_KERNEL_INFO_CASE(9)
        VBH_BATCH_KERNEL_INFO_CASE(10)
        VBH_BATCH_KERNEL_INFO_CASE(11)
    default:
        return false;
    }
}

} // namespace vbh
