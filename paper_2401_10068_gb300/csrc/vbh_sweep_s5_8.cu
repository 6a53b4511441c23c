// Instantiations of the fused sweep (single and batched forms) for S in {5, 6, 7, 8}.
#include "vbh_batched.cuh"
#include "vbh_sweep.cuh"
#include "vbh_resident.cuh"
#include "vbh_dispatch.cuh"

namespace vbh {

bool kernel_info_s5_8(int S, KernelInfo *out)
{
    switch (S) {
        VBH_KERNEL_INFO_CASE(5)
        VBH_KERNEL_INFO_CASE(6)
        VBH_KERNEL_INFO_CASE(7)
        VBH_KERNEL_INFO_CASE(8)
    default:
        return false;
    }
}

bool batch_kernel_info_s5_8(int S, BatchKernelInfo *out)
{
    switch (S) {
        VBH_BATCH_KERNEL_INFO_CASE(5)
        VBH_BATCH_KERNEL_INFO_CASE(6)
        VBH_BATCH_KERNEL_INFO_CASE(7)
        VBH_BATCH_KERNEL_INFO_CASE(8)
    default:
        return false;
    }
}

} // namespace vbh
