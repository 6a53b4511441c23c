// vbh_dispatch.cuh -- per-S kernel table of the fused sweep (host side).
#pragma once

#include <cstddef>

namespace vbh {

struct KernelInfo {
    const void *sweep;     // sweep_kernel<S, false>
    const void *sweep_comp;// sweep_kernel<S, true>: with the compensated statistics (one more column)
    const void *setup;     // setup_kernel<S - 1>
    size_t smem;           // dynamic shared memory of the sweep
    size_t smem_comp;      // and of its compensated form
    int threads;           // block size of the sweep
    int tile;              // observations per tile
    int nstat;             // statistics per block partial (plain form; the compensated form has nstat + 1)
    const void *resident;      // resident_kernel<S, false>: every sweep of a step in one cooperative launch
    const void *resident_comp; // resident_kernel<S, true>
    size_t res_fixed;          // its dynamic shared memory before the slice of observations
    size_t res_fixed_comp;
    size_t res_obs_bytes;      // shared memory per resident observation
    int res_threads;
    int res_max_blocks;        // blocks whose partial rows a block's buffer holds
    int res_max_blocks_comp;
};

// One form (plain or compensated statistics) of the batched data pass.
struct BatchPassInfo {
    const void *pass;      // batched_pass_kernel<S, COMP>
    size_t fixed;          // shared memory without the ring
    size_t stage_bytes;    // shared memory of one pipeline stage
    int max_stages;
    int threads;
    int tile;              // observations per tile
    int rows_per_chunk;    // partial rows per chunk (compute warps)
};

// Kernels of the batched form for one S class.
struct BatchKernelInfo {
    BatchPassInfo plain, comp;
    const void *update;    // batched_update_kernel<S - 1>
    const void *setup;     // batched_setup_kernel<S - 1>
    size_t update_smem;
    int nstat;             // statistics per partial row (plain form; the compensated form has nstat + 1)
};

// Each translation unit that instantiates sweep kernels fills the entries of
// its S range and returns false for the others.
bool kernel_info_s1_4(int S, KernelInfo *out);
bool kernel_info_s5_8(int S, KernelInfo *out);
bool kernel_info_s9_11(int S, KernelInfo *out);
bool batch_kernel_info_s1_4(int S, BatchKernelInfo *out);
bool batch_kernel_info_s5_8(int S, BatchKernelInfo *out);
bool batch_kernel_info_s9_11(int S, BatchKernelInfo *out);

} // namespace vbh

#define VBH_KERNEL_INFO_CASE(SV)                                                                                       \
    case SV: {                                                                                                         \
        using C = ::vbh::SweepCfg<SV>;                                                                                 \
        out->sweep = reinterpret_cast<const void *>(&::vbh::sweep_kernel<SV, false>);                                  \
        out->sweep_comp = reinterpret_cast<const void *>(&::vbh::sweep_kernel<SV, true>);                              \
        out->setup = reinterpret_cast<const void *>(&::vbh::setup_kernel<SV - 1>);                                     \
        out->smem = C::SMEM_BYTES;                                                                                     \
        out->smem_comp = C::SMEM_BYTES_C;                                                                              \
        out->threads = C::THREADS;                                                                                     \
        out->tile = C::T;                                                                                              \
        out->nstat = C::NSTAT;                                                                                         \
        out->resident = reinterpret_cast<const void *>(&::vbh::resident_kernel<SV, false>);                            \
        out->resident_comp = reinterpret_cast<const void *>(&::vbh::resident_kernel<SV, true>);                        \
        out->res_fixed = ::vbh::ResidentCfg<SV, false>::OFF_SLICE;                                                     \
        out->res_fixed_comp = ::vbh::ResidentCfg<SV, true>::OFF_SLICE;                                                 \
        out->res_obs_bytes = ::vbh::ResidentCfg<SV, false>::OBS_BYTES;                                                 \
        out->res_threads = ::vbh::ResidentCfg<SV, false>::THREADS;                                                     \
        out->res_max_blocks = ::vbh::ResidentCfg<SV, false>::RB_ROWS;                                                  \
        out->res_max_blocks_comp = ::vbh::ResidentCfg<SV, true>::RB_ROWS;                                              \
        return true;                                                                                                   \
    }

#define VBH_BATCH_PASS_INFO(DST, SV, CMP)                                                                             \
    do {                                                                                                               \
        using BC = ::vbh::BatchCfg<SV, CMP>;                                                                           \
        (DST).pass = reinterpret_cast<const void *>(&::vbh::batched_pass_kernel<SV, CMP>);                             \
        (DST).fixed = CMP ? BC::FIXED_C : BC::FIXED;                                                                   \
        (DST).stage_bytes = BC::STAGE_BYTES;                                                                           \
        (DST).max_stages = BC::MAX_STAGES;                                                                             \
        (DST).threads = BC::THREADS;                                                                                   \
        (DST).tile = BC::T;                                                                                            \
        (DST).rows_per_chunk = BC::CW;                                                                                 \
    } while (0)

#define VBH_BATCH_KERNEL_INFO_CASE(SV)                                                                                 \
    case SV: {                                                                                                         \
        VBH_BATCH_PASS_INFO(out->plain, SV, false);                                                                    \
        VBH_BATCH_PASS_INFO(out->comp, SV, true);                                                                      \
        out->update = reinterpret_cast<const void *>(&::vbh::batched_update_kernel<SV - 1>);                           \
        out->setup = reinterpret_cast<const void *>(&::vbh::batched_setup_kernel<SV - 1>);                             \
        out->update_smem = size_t(::vbh::gu_ws_doubles<SV - 1>()) * 8;                                                 \
        out->nstat = ::vbh::SweepCfg<SV>::NSTAT;                                                                       \
        return true;                                                                                                   \
    }
