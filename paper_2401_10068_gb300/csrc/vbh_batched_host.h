// vbh_batched_host.h -- host-side state of the batched form kept in a handle.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <vector>

#include "vbh.h"

namespace vbh {

struct BatchedHost {
    void *arena = nullptr;           // device memory: states, traces, work lists, partials, staging
    size_t arena_cap = 0;
    void *host_states = nullptr;     // pinned host copies of the states
    size_t host_states_cap = 0;
    std::vector<vbh_batch_plan> plan; // per class: the pass shape of the last call (the autotuner's choice)
};

int fit_batched_impl(BatchedHost &hb, cudaStream_t stream, int nsm, int B, const int64_t *V, const int *S,
                     const float *const *r, const float *const *d, const vbh_prior *p, const vbh_opts *o,
                     vbh_result *out, bool direct);

} // namespace vbh
