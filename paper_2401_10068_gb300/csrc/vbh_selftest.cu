// vbh_selftest.cu -- diagnostics: the bounded device waits (vbh_selftest_wait)
// and the short-latency FP64 functions of the global updates
// (vbh_selftest_math).
//
// Every kernel of the library waits on mbarriers (bulk copies landing, MMAs
// completing) through mbar_wait_bounded / mbar_wait_backoff, which give up
// after a wall-time budget and let the kernel record VBH_ETIMEOUT instead of
// hanging.  In the sweeps those waits always complete, so the give-up path is
// exercised here on a barrier phase that nothing completes: one block, no
// fault, no trap, nothing left in flight when it returns.
#include <cuda_runtime.h>

#include <cstdint>

#include "vbh.h"
#include "vbh_error.h"
#include "vbh_internal.cuh"

namespace vbh {
namespace {

constexpr int COPY_BYTES = 1024;

// out[0]: bounded polling wait on a phase nobody completes (expect ETIMEOUT);
// out[1]: the same with a sleep between polls (expect ETIMEOUT); out[2]: a
// wait on a phase a bulk copy completes (expect OK); out[3]: the copied bytes
// (expect OK); *waited: nanoseconds the first wait took.
__global__ void selftest_wait_kernel(const unsigned char *src, unsigned long long budget_ns, int *out,
                                     unsigned long long *waited)
{
    __shared__ __align__(128) unsigned char buf[COPY_BYTES];
    __shared__ __align__(8) uint64_t bar[3];
    if (threadIdx.x != 0) return;
    for (int i = 0; i < 3; ++i) mbar_init(&bar[i], 1);
    fence_mbar_init();
    const uint64_t t0 = global_ns();
    const bool a = mbar_wait_bounded(&bar[0], 0u, budget_ns);
    *waited = global_ns() - t0;
    const bool b = mbar_wait_backoff(&bar[1], 0u, budget_ns);
    mbar_arrive_expect_tx(&bar[2], COPY_BYTES);
    bulk_load(buf, src, COPY_BYTES, &bar[2]);
    const bool c = mbar_wait_bounded(&bar[2], 0u, 1000000000ull);
    int bad = 0;
    if (c)
        for (int i = 0; i < COPY_BYTES; ++i) bad |= (buf[i] != static_cast<unsigned char>(i * 7 + 3));
    out[0] = a ? VBH_OK : VBH_ETIMEOUT;
    out[1] = b ? VBH_OK : VBH_ETIMEOUT;
    out[2] = c ? VBH_OK : VBH_ETIMEOUT;
    out[3] = (c && !bad) ? VBH_OK : VBH_ENONFINITE;
}

// out[i] = f(x[i]): fn 0 log_tang (its table built by the block as the
// resident loop builds it), fn 1 rsqrt_fast.
__global__ void selftest_math_kernel(int fn, const double *x, double *out, int n)
{
    __shared__ double tab[256];
    log_tang_table(tab, threadIdx.x, blockDim.x);
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = (fn == 0) ? log_tang(x[i], tab) : rsqrt_fast(x[i]);
}

} // namespace
} // namespace vbh

extern "C" int vbh_selftest_math(int device, void *stream, int fn, const double *x, double *out, int n)
{
    if (!x || !out || n < 1 || n > (1 << 24) || fn < 0 || fn > 1) return VBH_EINVAL;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (cudaSetDevice(device) != cudaSuccess) return VBH_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double *mem = nullptr;
    int rc = VBH_OK;
    const size_t bytes = sizeof(double) * size_t(n);
    if (cudaMalloc(&mem, 2 * bytes) != cudaSuccess) {
        vbh::record_error("cudaMalloc", __FILE__, __LINE__, cudaGetErrorName(cudaGetLastError()));
        rc = VBH_ENOMEM;
    }
    if (!rc) {
        auto run = [&]() -> int {
            VBH_CHECK_CUDA(cudaMemcpyAsync(mem, x, bytes, cudaMemcpyHostToDevice, s));
            const int blocks = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
            vbh::selftest_math_kernel<<<blocks, 256, 0, s>>>(fn, mem, mem + n, n);
            VBH_CHECK_CUDA(cudaGetLastError());
            VBH_CHECK_CUDA(cudaMemcpyAsync(out, mem + n, bytes, cudaMemcpyDeviceToHost, s));
            VBH_CHECK_CUDA(cudaStreamSynchronize(s));
            return VBH_OK;
        };
        rc = run();
    }
    if (mem) cudaFree(mem);
    if (prev >= 0) cudaSetDevice(prev);
    return rc;
}

extern "C" int vbh_selftest_wait(int device, void *stream, uint64_t budget_ns, int *status, uint64_t *waited_ns)
{
    if (!status || !waited_ns || budget_ns == 0 || budget_ns > 1000000000ull) return VBH_EINVAL;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (cudaSetDevice(device) != cudaSuccess) return VBH_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char host_src[vbh::COPY_BYTES];
    for (int i = 0; i < vbh::COPY_BYTES; ++i) host_src[i] = static_cast<unsigned char>(i * 7 + 3);
    unsigned char *mem = nullptr;
    int rc = VBH_OK;
    int out[4] = {0, 0, 0, 0};
    unsigned long long waited = 0;
    const size_t bytes = vbh::COPY_BYTES + 64;
    if (cudaMalloc(&mem, bytes) != cudaSuccess) {
        vbh::record_error("cudaMalloc", __FILE__, __LINE__, cudaGetErrorName(cudaGetLastError()));
        rc = VBH_ENOMEM;
    }
    int *dout = reinterpret_cast<int *>(mem + vbh::COPY_BYTES);
    unsigned long long *dwait = reinterpret_cast<unsigned long long *>(mem + vbh::COPY_BYTES + 32);
    if (!rc) {
        auto run = [&]() -> int {
            VBH_CHECK_CUDA(cudaMemcpyAsync(mem, host_src, vbh::COPY_BYTES, cudaMemcpyHostToDevice, s));
            vbh::selftest_wait_kernel<<<1, 32, 0, s>>>(mem, (unsigned long long)budget_ns, dout, dwait);
            VBH_CHECK_CUDA(cudaGetLastError());
            VBH_CHECK_CUDA(cudaMemcpyAsync(out, dout, sizeof(out), cudaMemcpyDeviceToHost, s));
            VBH_CHECK_CUDA(cudaMemcpyAsync(&waited, dwait, sizeof(waited), cudaMemcpyDeviceToHost, s));
            VBH_CHECK_CUDA(cudaStreamSynchronize(s));
            return VBH_OK;
        };
        rc = run();
    }
    if (mem) cudaFree(mem);
    if (prev >= 0) cudaSetDevice(prev);
    if (rc) return rc;
    for (int i = 0; i < 4; ++i) status[i] = out[i];
    *waited_ns = waited;
    return VBH_OK;
}
