// vbh_error.h -- per-thread detail of the last CUDA failure behind a VBH_ECUDA
// or VBH_ENOMEM status (vbh_last_error_detail).
#pragma once

namespace vbh {

// Record "<what> at <file>:<line>: <detail>" for the calling host thread.
void record_error(const char *what, const char *file, int line, const char *detail);

// The calling thread's last record ("" if none).
const char *last_error_buf();

} // namespace vbh

// Evaluate a cudaError_t expression; on failure record it and return the
// matching status from the enclosing function.
#define VBH_CHECK_CUDA(call)                                                                                           \
    do {                                                                                                               \
        cudaError_t e_ = (call);                                                                                       \
        if (e_ != cudaSuccess) {                                                                                       \
            vbh::record_error(#call, __FILE__, __LINE__, cudaGetErrorName(e_));                                        \
            (void)cudaGetLastError();                                                                                  \
            return e_ == cudaErrorMemoryAllocation ? VBH_ENOMEM : VBH_ECUDA;                                           \
        }                                                                                                              \
    } while (0)
