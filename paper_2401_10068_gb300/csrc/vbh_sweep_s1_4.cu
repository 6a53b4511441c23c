// Instantiations of the fused sweep (single and batched forms) for S in {1, 2, 3, 4}.
#include "vbh_batched.cuh"
#include "vbh_sweep.cuh"
#include "vbh_resident.cuh"
#include "vbh_dispatch.cuh"

namespace vbh {

bool kernel_info_s1_4(int S, KernelInfo *out)
{
    switch (S) {
        VBH_KERNEL_INFO_CASE(1)
        VBH_KERNEL_INFO_CASE(2)
        VBH_KERNEL_INFO_CASE(3)
        VBH_KERNEL_INFO_CASE(4)
    default:
        return false;
    }
}

bool batch_kernel_info_s1_4(int S, BatchKernelInfo *out)
{
    switch (S) {
        VBH_BATCH_KERNEL_INFO_CASE(1)
        VBH_BATCH_KERNEL_INFO_CASE(2)
        VBH_BATCH_KERNEL_INFO_CASE(3)
        VBH_BATCH_KERNEL_INFO_CASE(4)
    default:
        return false;
    }
}

} // namespace vbh
