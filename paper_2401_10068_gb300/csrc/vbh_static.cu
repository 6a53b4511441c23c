// vbh_static.cu -- vbh_fit_static: a fit that allocates nothing.
//
// Every other entry point works through a vbh_handle, which allocates its
// device state, per-block partial sums and staging buffers with cudaMalloc
// and builds a CUDA graph.  Some callers cannot do that: a cudaMalloc or
// cudaFree synchronises the whole device and stalls other streams of
// latency-sensitive work sharing the GPU; host frameworks that hand out all
// device memory from their own pool (a caching allocator that has reserved
// most of the GPU) can make a foreign cudaMalloc fail for lack of memory;
// plug-in hosts and fixed-budget deployments forbid allocations outside the
// budget set when the library is loaded.  vbh_fit_static serves them: its
// scratch (the fit state, the per-block partials and the ELBO trace) lives in
// one file-scope __device__ array below, which every GPU that loads the
// library holds from load until exit, and the call performs no allocation of
// its own.
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstring>
#include <mutex>

#include "vbh.h"
#include "vbh_dispatch.cuh"
#include "vbh_error.h"
#include "vbh_internal.cuh"

namespace {

using vbh::DevState;

constexpr size_t TRACE_OFF = (sizeof(DevState) + 255) / 256 * 256;
constexpr size_t PART_OFF = TRACE_OFF + size_t(VBH_STATIC_TRACE_MAX) * sizeof(double);
static_assert(PART_OFF < VBH_STATIC_SCRATCH_BYTES, "scratch too small for the state and trace");
constexpr size_t PART_DOUBLES = (VBH_STATIC_SCRATCH_BYTES - PART_OFF) / sizeof(double);

// The scratch shared by every vbh_fit_static call on a device.  In host code
// this name is only a stand-in; its device address comes from
// cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char vbh_static_scratch[VBH_STATIC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char *g_addr[MAX_DEVICES] = {};

bool kernel_info_any(int S, vbh::KernelInfo *ki)
{
    return vbh::kernel_info_s1_4(S, ki) || vbh::kernel_info_s5_8(S, ki) || vbh::kernel_info_s9_11(S, ki);
}

// Device address of the scratch on the current device, looked up once per
// device with that device current.  The same first call loads every kernel
// this entry point can launch (the sweeps, plain and compensated, and the
// set-up kernels of S = 1..11): with CUDA's lazy module loading a module is
// loaded, which allocates device memory, at the first use of one of its
// symbols, so without this a later call at a new S would allocate.  After
// the first call per device no call loads code or allocates.
int scratch_address(int device, unsigned char **out)
{
    if (device < 0 || device >= MAX_DEVICES) return VBH_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[device]) {
        void *p = nullptr;
        VBH_CHECK_CUDA(cudaGetSymbolAddress(&p, vbh_static_scratch));
        if (!p) {
            vbh::record_error("cudaGetSymbolAddress(vbh_static_scratch)", __FILE__, __LINE__, "null address");
            return VBH_ECUDA;
        }
        for (int S = 1; S <= vbh::S_FP32_MAX; ++S) {
            vbh::KernelInfo ki;
            if (!kernel_info_any(S, &ki)) return VBH_EUNSUPPORTED;
            cudaFuncAttributes fa;
            VBH_CHECK_CUDA(cudaFuncGetAttributes(&fa, ki.sweep));
            VBH_CHECK_CUDA(cudaFuncGetAttributes(&fa, ki.sweep_comp));
            VBH_CHECK_CUDA(cudaFuncGetAttributes(&fa, ki.setup));
            VBH_CHECK_CUDA(cudaFuncSetAttribute(ki.sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, int(ki.smem)));
            VBH_CHECK_CUDA(
                cudaFuncSetAttribute(ki.sweep_comp, cudaFuncAttributeMaxDynamicSharedMemorySize, int(ki.smem_comp)));
        }
        g_addr[device] = static_cast<unsigned char *>(p);
    }
    *out = g_addr[device];
    return VBH_OK;
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

bool spd(int M, const double *A)
{
    double L[vbh::MMAX * vbh::MMAX];
    for (int j = 0; j < M; ++j) {
        for (int i = 0; i < M; ++i) {
            if (!std::isfinite(A[i * M + j])) return false;
            if (std::fabs(A[i * M + j] - A[j * M + i]) > 1e-10 * std::sqrt(std::fabs(A[i * M + i] * A[j * M + j])))
                return false;
        }
        double s = A[j * M + j];
        for (int k = 0; k < j; ++k) s -= L[j * M + k] * L[j * M + k];
        if (!(s > 0.0)) return false;
        L[j * M + j] = std::sqrt(s);
        for (int i = j + 1; i < M; ++i) {
            double t = A[i * M + j];
            for (int k = 0; k < j; ++k) t -= L[i * M + k] * L[j * M + k];
            L[i * M + j] = t / L[j * M + j];
        }
    }
    return true;
}

bool device_ptr_on(const void *p, int device)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return false;
    if (at.type == cudaMemoryTypeDevice && at.device != device) return false;
    return reinterpret_cast<uintptr_t>(p) % 16 == 0;
}

struct DeviceSwitch {
    int prev = -1;
    bool ok = false;
    explicit DeviceSwitch(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceSwitch()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

#define VBH_S_CK(call) VBH_CHECK_CUDA(call)

} // namespace

extern "C" int vbh_fit_static(const float *r, const float *d, int64_t V, int S, const vbh_prior *p,
                              const vbh_opts *o, vbh_result *out, int device, void *stream)
{
    // ---- arguments (host only) ----
    if (!p || !o || !out || S < 1 || S > VBH_SMAX || V < 0 || V > (int64_t(1) << 40) || p->S != S)
        return VBH_EINVAL;
    if (S > vbh::S_FP32_MAX) return VBH_EUNSUPPORTED;
    if (!finite_pos(p->q0) || !finite_pos(p->n0) || !finite_pos(p->a0) || !finite_pos(p->b0)) return VBH_EINVAL;
    const int M = S - 1;
    if (p->K0)
        for (int j = 0; j < M; ++j)
            if (!std::isfinite(p->K0[j])) return VBH_EINVAL;
    if (p->Lambda0_inv && !spd(M, p->Lambda0_inv)) return VBH_EINVAL;
    if (o->max_iter < 0 || !(o->tol >= 0.0) || !std::isfinite(o->tol) || o->precision != VBH_FP32) return VBH_EINVAL;
    if (o->init != VBH_INIT_PAPER && o->init != VBH_INIT_GIVEN) return VBH_EINVAL;
    if (o->method != VBH_CAVI) return VBH_EUNSUPPORTED;           // this entry point runs CAVI only
    if (o->grouped != 0) return VBH_EUNSUPPORTED;                 // and the per-observation sweep only
    if (o->stats != VBH_STATS_AUTO && o->stats != VBH_STATS_COMPENSATED && o->stats != VBH_STATS_PLAIN)
        return VBH_EINVAL;
    const bool comp = o->stats == VBH_STATS_COMPENSATED || (o->stats == VBH_STATS_AUTO && o->tol > 0.0);
    if (o->elbo_trace && o->max_iter + 1 > VBH_STATIC_TRACE_MAX) return VBH_EINVAL;   // trace beyond the scratch
    const vbh_result *q = o->init_state;
    if (o->init == VBH_INIT_GIVEN) {
        if (!q || q->S != S || !finite_pos(q->a_rho) || !finite_pos(q->b_rho) || !(q->nu > M - 1.0) ||
            !finite_pos(q->lambda) || !spd(M, q->W_inv))
            return VBH_EINVAL;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        (void)cudaGetLastError();
        return VBH_ECUDA;
    }
    if (device < 0 || device >= ndev) return VBH_EINVAL;
    DeviceSwitch ds(device);
    if (!ds.ok) return VBH_ECUDA;
    if (V > 0 && (!r || !d || !device_ptr_on(r, device) || !device_ptr_on(d, device))) return VBH_EINVAL;

    vbh::KernelInfo ki;
    if (!kernel_info_any(S, &ki)) return VBH_EUNSUPPORTED;
    const void *sweep = comp ? ki.sweep_comp : ki.sweep;
    const size_t smem = comp ? ki.smem_comp : ki.smem;
    const int nstat = ki.nstat + (comp ? 1 : 0);
    unsigned char *base = nullptr;
    int rc = scratch_address(device, &base);
    if (rc) return rc;
    DevState *st = reinterpret_cast<DevState *>(base);
    double *trace = reinterpret_cast<double *>(base + TRACE_OFF);
    double *partials = reinterpret_cast<double *>(base + PART_OFF);

    // ---- launch shape: the persistent grid, capped by the partials that fit
    //      (the shared-memory attribute was set by the first call) ----
    int nsm = 0, per_sm = 0;
    VBH_S_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device));
    VBH_S_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep, ki.threads, smem));
    if (per_sm < 1) {
        vbh::record_error("occupancy of the sweep kernel", __FILE__, __LINE__, "no block fits on an SM");
        return VBH_ECUDA;
    }
    long long grid = (long long)nsm * per_sm;
    const long long tiles = (V + ki.tile - 1) / ki.tile;
    if (tiles < grid) grid = tiles;
    if (grid > vbh::GRID_MAX) grid = vbh::GRID_MAX;
    while (grid > 1 && size_t(vbh::partial_rows(grid)) * size_t(nstat) > PART_DOUBLES) --grid;
    if (grid < 1) grid = 1;

    // ---- the whole state is written by each call: nothing of an earlier call
    //      (ticket counter, status, trace) carries over ----
    DevState hs;
    std::memset(&hs, 0, sizeof(hs));
    hs.S = S;
    hs.M = M;
    hs.V = double(V);
    hs.q0 = p->q0;
    hs.n0 = p->n0;
    hs.a0 = p->a0;
    hs.b0 = p->b0;
    for (int j = 0; j < M; ++j) hs.K0[j] = p->K0 ? p->K0[j] : 1.0 / S;
    for (int a = 0; a < M; ++a)
        for (int b = 0; b < M; ++b)
            hs.L0inv[a * M + b] = p->Lambda0_inv ? 0.5 * (p->Lambda0_inv[a * M + b] + p->Lambda0_inv[b * M + a])
                                                 : 0.005 + (a == b ? (a % 2 == 0 ? 0.005 : 0.003) : 0.0);
    hs.tol = o->tol;
    hs.max_iter = o->max_iter;
    hs.target = o->max_iter;
    hs.trace = o->elbo_trace ? trace : nullptr;
    hs.comp = comp ? 1 : 0;
    if (o->init == VBH_INIT_GIVEN) {
        hs.a_rho = q->a_rho;
        hs.b_rho = q->b_rho;
        hs.nu = q->nu;
        hs.lam = q->lambda;
        for (int j = 0; j < M; ++j) hs.kappa[j] = q->kappa[j];
        for (int a = 0; a < M; ++a)
            for (int b = 0; b < M; ++b) hs.Winv[a * M + b] = 0.5 * (q->W_inv[a * M + b] + q->W_inv[b * M + a]);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    VBH_S_CK(cudaMemcpyAsync(st, &hs, sizeof(hs), cudaMemcpyHostToDevice, s));

    // ---- set-up, sweep 0, then one launch per sweep, issued in batches of
    //      SWEEP_BATCH: between batches the control fields are read back and
    //      no further launch is issued once the fit has stopped (converged,
    //      failed or at max_iter; a launch after that returns at once) ----
    const int init = (o->init == VBH_INIT_GIVEN) ? 0 : 1;
    {
        void *args[] = {&st, const_cast<int *>(&init)};
        VBH_S_CK(cudaLaunchKernel(ki.setup, dim3(1), dim3(32), args, 0, s));
    }
    vbh::SweepArgs a{};
    a.r = r;
    a.d = d;
    a.V = V;
    a.st = st;
    a.partials = partials;
    a.use_cond = 0;
    a.mode = init ? vbh::MODE_INIT : vbh::MODE_ELBO;
    void *args[] = {&a};
    VBH_S_CK(cudaLaunchKernel(sweep, dim3(unsigned(grid)), dim3(ki.threads), args, smem, s));
    a.mode = vbh::MODE_ITER;
    constexpr int SWEEP_BATCH = 64;
    struct Ctl {
        int iter, target, max_iter, converged, status;
    } ctl{};
    static_assert(offsetof(DevState, status) - offsetof(DevState, iter) == 4 * sizeof(int), "control field layout");
    for (int t = 0; t < o->max_iter;) {
        const int n = (o->max_iter - t < SWEEP_BATCH) ? o->max_iter - t : SWEEP_BATCH;
        for (int i = 0; i < n; ++i)
            VBH_S_CK(cudaLaunchKernel(sweep, dim3(unsigned(grid)), dim3(ki.threads), args, smem, s));
        t += n;
        if (t >= o->max_iter) break;
        VBH_S_CK(cudaMemcpyAsync(&ctl, &st->iter, sizeof(ctl), cudaMemcpyDeviceToHost, s));
        VBH_S_CK(cudaStreamSynchronize(s));
        if (ctl.converged || ctl.status != VBH_OK || ctl.iter >= o->max_iter) break;
    }

    // ---- results ----
    VBH_S_CK(cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s));
    VBH_S_CK(cudaStreamSynchronize(s));
    if (o->elbo_trace) {
        const int n = hs.iter + 1;
        VBH_S_CK(cudaMemcpyAsync(o->elbo_trace, trace, sizeof(double) * size_t(n), cudaMemcpyDeviceToHost, s));
        VBH_S_CK(cudaStreamSynchronize(s));
    }
    std::memset(out, 0, sizeof(*out));
    out->S = S;
    out->iters = hs.iter;
    out->converged = hs.converged;
    out->status = hs.status;
    out->elbo_const_dropped = hs.const_dropped;
    double sum = 0.0;
    for (int j = 0; j < M; ++j) {
        out->kappa[j] = hs.kappa[j];
        out->weights[j] = hs.kappa[j];
        sum += hs.kappa[j];
    }
    out->weights[M] = 1.0 - sum;
    std::memcpy(out->W_inv, hs.Winv, sizeof(double) * size_t(M) * size_t(M));
    out->nu = hs.nu;
    out->lambda = hs.lam;
    out->a_rho = hs.a_rho;
    out->b_rho = hs.b_rho;
    out->rho_mean = hs.a_rho / hs.b_rho;
    out->rho_mode = (hs.a_rho - 1.0) / hs.b_rho;
    out->elbo = hs.elbo;
    return hs.status;
}
