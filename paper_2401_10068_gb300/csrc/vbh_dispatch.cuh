// vbh_dispatch.cuh -- per-S kernel table of the fused sweep (host side).
#pragma once

#include <cstddef>

namespace vbh {

struct KernelInfo {
    const void *sweep;     // sweep_kernel<S>
    const void *setup;     // setup_kernel<S - 1>
    size_t smem;           // dynamic shared memory of the sweep
    int threads;           // block size of the sweep
    int tile;              // observations per tile
    int nstat;             // statistics per block partial
};

// Each translation unit that instantiates sweep kernels fills the entries of
// its S range and returns false for the others.
bool kernel_info_s1_4(int S, KernelInfo *out);
bool kernel_info_s5_8(int S, KernelInfo *out);
bool kernel_info_s9_11(int S, KernelInfo *out);

} // namespace vbh

#define VBH_KERNEL_INFO_CASE(SV)                                                                                       \
    case SV: {                                                                                                         \
        using C = ::vbh::SweepCfg<SV>;                                                                                 \
        static_assert(size_t(::vbh::gu_ws_doubles<SV - 1>()) * 8 <= C::RING_BYTES, "workspace exceeds the ring");    \
        out->sweep = reinterpret_cast<const void *>(&::vbh::sweep_kernel<SV>);                                         \
        out->setup = reinterpret_cast<const void *>(&::vbh::setup_kernel<SV - 1>);                                     \
        out->smem = C::SMEM_BYTES;                                                                                     \
        out->threads = C::THREADS;                                                                                     \
        out->tile = C::T;                                                                                              \
        out->nstat = C::NSTAT;                                                                                         \
        return true;                                                                                                   \
    }
