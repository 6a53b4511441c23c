// vbh_api.cu -- the C ABI declared in include/vbh.h: handle, argument
// checks, input staging, the CUDA-graph sweep loop and result read-back.
// All arithmetic of the method runs in the kernels of vbh_sweep.cuh.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "vbh.h"
#include "vbh_batched_host.h"
#include "vbh_dispatch.cuh"
#include "vbh_internal.cuh"
#include "vbh_error.h"
#include "vbh_grouped_host.h"
#include "vbh_tc_host.h"

using vbh::DevState;
using vbh::KernelInfo;

// How the sweeps of a fit are launched: the CUDA-core kernel (S <= 11) or the
// tensor-core kernel (12 <= S <= 32, which reads BF16 profiles through
// tensor maps).
struct Launch {
    bool grp = false;                       // profile-grouped sweep
    int P = 0;                              // profile codes (2^S)
    const double *gstats = nullptr;         // their (n, sum y, sum y^2)
    bool tc = false;
    bool comp = false;                      // compensated statistics (CUDA-core sweep only)
    int S = 0;
    int grid = 0;
    int nsplit = 3;
    int binary = 1;
    KernelInfo ki{};
    vbh::TcKernelInfo tki{};
    const unsigned char *tiles = nullptr;   // repacked inputs of the tensor-core sweep
    const void *func() const
    {
        return grp ? vbh::grouped_sweep_func(S) : tc ? tki.sweep : comp ? ki.sweep_comp : ki.sweep;
    }
    const void *setup() const { return (tc || grp) ? tki.setup : ki.setup; }
    int threads() const { return grp ? vbh::GROUPED_THREADS : tc ? tki.threads : ki.threads; }
    size_t smem() const { return grp ? vbh::grouped_smem_bytes() : tc ? tki.smem : comp ? ki.smem_comp : ki.smem; }
    int tile() const { return tc ? tki.tile : ki.tile; }
    // the resident sweep loop (S <= 11, CUDA-core sweep): one cooperative launch per step
    bool res = false;
    int res_grid = 0;
    int res_per_block = 0;
    int res_ns = 0;                         // columns of its partial rows
    size_t res_smem = 0;
    const void *res_func() const { return comp ? ki.resident_comp : ki.resident; }
};

struct vbh_handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    int nsm = 0;
    DevState *st = nullptr;            // device state of the step-wise fit
    DevState *st_aux = nullptr;        // device state used by vbh_elbo
    DevState *mirror = nullptr;        // pinned host copy of a DevState
    double *partials = nullptr;
    size_t partials_cap = 0;           // bytes
    double *trace = nullptr;
    int trace_cap = 0;
    float *stage_r = nullptr, *stage_d = nullptr;
    size_t stage_cap_r = 0, stage_cap_d = 0;   // bytes
    // copy streams for host inputs: large copies are split over them so that several
    // copy engines move the data; events join them with the handle's stream
    static constexpr int NCOPY = 4;
    cudaStream_t copy_stream[NCOPY] = {};
    cudaEvent_t copy_event[NCOPY + 1] = {};
    // current fit
    bool begun = false;
    int S = 0;
    long long V = 0;
    const float *r = nullptr, *d = nullptr;    // device pointers used by the kernels
    int max_iter = 0;
    double *user_trace = nullptr;
    Launch L;
    bool bf16_phase = false;       // VBH_BF16 fit still in its 16-bit sweeps
    int bf16_limit = 0;            // last sweep index of the 16-bit sweeps
    int refine = 0;                // FP32 sweeps after them
    // repacked inputs of the tensor-core path
    void *tc_tiles = nullptr;
    size_t tc_cap = 0;
    unsigned long long *counts = nullptr;       // [inexact, non-binary] profile values (device)
    double *gstats = nullptr;                    // profile histogram of the grouped sweep
    size_t gstats_cap = 0;
    const void *g_tiles = nullptr;
    const void *g_gstats = nullptr;
    // cached graph of the sweep loop
    cudaGraphExec_t gexec = nullptr;
    int g_S = -1, g_grid = -1;
    long long g_V = -1;
    const float *g_r = nullptr, *g_d = nullptr;
    const double *g_partials = nullptr;
    const void *g_func = nullptr;
    bool attr_set[vbh::SMAX + 1] = {};
    bool direct = false;               // VBH_LAUNCH=direct: one stream launch per sweep, no graph
    // the resident sweep loop
    bool coop = false;                 // the device supports cooperative launches
    int smem_optin = 0;                // dynamic shared memory a block may opt in to
    int res_obs = 2;                   // observations per thread and sweep the block count aims at
    size_t res_attr[vbh::S_FP32_MAX + 1][2] = {};   // shared memory the resident kernels were opted in to
    DevState *res_priv = nullptr;      // private state copies of blocks 1 ..
    size_t res_priv_cap = 0;           // bytes
    vbh::BatchedHost batched;          // buffers of vbh_fit_batched
};

namespace vbh {

// Sweep budget of one vbh_fit_step call: the graph loop runs while iter < target.
__global__ void set_target_kernel(DevState *st, int nsweeps)
{
    if (threadIdx.x == 0) {
        long long t = (long long)st->iter + nsweeps;
        st->target = t > st->max_iter ? st->max_iter : int(t);
    }
}

namespace {
thread_local char g_error_detail[512] = "";
} // namespace

void record_error(const char *what, const char *file, int line, const char *detail)
{
    const char *base = std::strrchr(file, '/');
    std::snprintf(g_error_detail, sizeof(g_error_detail), "%s at %s:%d: %s", what, base ? base + 1 : file, line,
                  detail ? detail : "");
}

const char *last_error_buf() { return g_error_detail; }

} // namespace vbh

namespace {

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

#define VBH_CK(call) VBH_CHECK_CUDA(call)

bool kernel_info(int S, KernelInfo *ki)
{
    return vbh::kernel_info_s1_4(S, ki) || vbh::kernel_info_s5_8(S, ki) || vbh::kernel_info_s9_11(S, ki);
}

// The default Lambda_0^{-1}: 0.005 * 1 1^T + diag(0.005, 0.003, 0.005, ...).
void default_L0inv(int M, double *out)
{
    for (int r = 0; r < M; ++r)
        for (int c = 0; c < M; ++c) out[r * M + c] = 0.005 + (r == c ? (r % 2 == 0 ? 0.005 : 0.003) : 0.0);
}

// Symmetric (to 1e-10 relative; callers' matrices may differ from their
// transpose in the last bits) and positive definite.
bool host_spd(int M, const double *A)
{
    double L[vbh::MMAX * vbh::MMAX];
    for (int j = 0; j < M; ++j) {
        for (int i = 0; i < M; ++i) {
            if (!std::isfinite(A[i * M + j])) return false;
            const double scale = std::sqrt(std::fabs(A[i * M + i] * A[j * M + j]));
            if (std::fabs(A[i * M + j] - A[j * M + i]) > 1e-10 * scale) return false;
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

bool pos_finite(double x) { return std::isfinite(x) && x > 0.0; }

// dst = (A + A^T) / 2
void symmetrize(int M, const double *A, double *dst)
{
    for (int r = 0; r < M; ++r)
        for (int c = 0; c < M; ++c) dst[r * M + c] = 0.5 * (A[r * M + c] + A[c * M + r]);
}

int check_prior(const vbh_prior *p, int S)
{
    if (!p || p->S != S) return VBH_EINVAL;
    if (!pos_finite(p->q0) || !pos_finite(p->n0) || !pos_finite(p->a0) || !pos_finite(p->b0)) return VBH_EINVAL;
    const int M = S - 1;
    if (p->K0)
        for (int j = 0; j < M; ++j)
            if (!std::isfinite(p->K0[j])) return VBH_EINVAL;
    if (p->Lambda0_inv && !host_spd(M, p->Lambda0_inv)) return VBH_EINVAL;
    return VBH_OK;
}

// Device pointer usable as-is (16-byte aligned, on this device), host pointer
// to stage, or invalid.
enum PtrKind { PTR_DEVICE, PTR_HOST, PTR_BAD };

PtrKind classify(const void *p, int device)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return PTR_HOST;
    }
    switch (at.type) {
    case cudaMemoryTypeDevice:
        if (at.device != device) return PTR_BAD;
        return (reinterpret_cast<uintptr_t>(p) % 16 == 0) ? PTR_DEVICE : PTR_BAD;
    case cudaMemoryTypeManaged:
        return (reinterpret_cast<uintptr_t>(p) % 16 == 0) ? PTR_DEVICE : PTR_HOST;
    default:
        return PTR_HOST;
    }
}

int ensure(void **buf, size_t *cap, size_t bytes)
{
    if (*cap >= bytes && *buf) return VBH_OK;
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    if (bytes == 0) return VBH_OK;
    if (cudaMalloc(buf, bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        return VBH_ENOMEM;
    }
    *cap = bytes;
    return VBH_OK;
}

// Host -> device copy ordered on the handle's stream.  Copies of 256 MiB or
// more are split into chunks issued round robin on the handle's copy streams
// (after the work queued so far on the handle's stream), whose completion the
// handle's stream then waits for.
int copy_h2d(vbh_handle *h, void *dst, const void *src, size_t bytes)
{
    constexpr size_t SPLIT_MIN = size_t(256) << 20;
    if (bytes < SPLIT_MIN || !h->copy_stream[0]) {
        VBH_CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, h->stream));
        return VBH_OK;
    }
    constexpr int NC = vbh_handle::NCOPY;
    VBH_CK(cudaEventRecord(h->copy_event[NC], h->stream));
    for (int i = 0; i < NC; ++i) VBH_CK(cudaStreamWaitEvent(h->copy_stream[i], h->copy_event[NC], 0));
    const size_t nchunk = 4 * NC;
    const size_t chunk = ((bytes + nchunk - 1) / nchunk + 4095) & ~size_t(4095);
    size_t off = 0;
    for (size_t c = 0; off < bytes; ++c) {
        const size_t len = (bytes - off < chunk) ? bytes - off : chunk;
        VBH_CK(cudaMemcpyAsync(static_cast<char *>(dst) + off, static_cast<const char *>(src) + off, len,
                               cudaMemcpyHostToDevice, h->copy_stream[c % NC]));
        off += len;
    }
    for (int i = 0; i < NC; ++i) {
        VBH_CK(cudaEventRecord(h->copy_event[i], h->copy_stream[i]));
        VBH_CK(cudaStreamWaitEvent(h->stream, h->copy_event[i], 0));
    }
    return VBH_OK;
}

// Resolve (r, d) to device pointers, copying host inputs into the handle's
// staging buffers, ordered on the handle's stream.
int stage_inputs(vbh_handle *h, const float *r, const float *d, long long V, int S, const float **rd,
                 const float **dd)
{
    if (V == 0) {
        *rd = nullptr;
        *dd = nullptr;
        return VBH_OK;
    }
    const PtrKind kr = classify(r, h->device), kd = classify(d, h->device);
    if (kr == PTR_BAD || kd == PTR_BAD) return VBH_EINVAL;
    const size_t br = size_t(V) * 4, bd = size_t(V) * size_t(S) * 4;
    if (kr == PTR_HOST) {
        int rc = ensure(reinterpret_cast<void **>(&h->stage_r), &h->stage_cap_r, br);
        if (rc) return rc;
        if ((rc = copy_h2d(h, h->stage_r, r, br))) return rc;
        *rd = h->stage_r;
    } else {
        *rd = r;
    }
    if (kd == PTR_HOST) {
        int rc = ensure(reinterpret_cast<void **>(&h->stage_d), &h->stage_cap_d, bd);
        if (rc) return rc;
        if ((rc = copy_h2d(h, h->stage_d, d, bd))) return rc;
        *dd = h->stage_d;
    } else {
        *dd = d;
    }
    return VBH_OK;
}

void fill_prior(DevState *s, const vbh_prior *p, int S, long long V)
{
    const int M = S - 1;
    s->S = S;
    s->M = M;
    s->V = double(V);
    s->q0 = p->q0;
    s->n0 = p->n0;
    s->a0 = p->a0;
    s->b0 = p->b0;
    for (int j = 0; j < M; ++j) s->K0[j] = p->K0 ? p->K0[j] : 1.0 / S;
    if (p->Lambda0_inv)
        symmetrize(M, p->Lambda0_inv, s->L0inv);
    else
        default_L0inv(M, s->L0inv);
}

// Kernel choice, launch shape and partials buffer of a fit of (V, S).  For the
// tensor-core path the BF16 profiles and the tensor maps are prepared too.
// Shape of the resident sweep loop for (V, S): blocks of at most
// res_obs x threads observations, fewer and larger ones when the SMs would not
// suffice, none (false) when the data set does not fit in the shared memory of
// h->nsm blocks.
bool resident_shape(const vbh_handle *h, const KernelInfo &ki, bool comp, long long V, int *grid, int *per_block,
                    int *ns, size_t *smem)
{
    if (V <= 0 || !h->coop) return false;
    const size_t fixed = comp ? ki.res_fixed_comp : ki.res_fixed;
    const size_t budget = size_t(h->smem_optin) - 1024;        // room for the kernel's static shared memory
    if (budget <= fixed + 64 * ki.res_obs_bytes) return false;
    const long long cap = (static_cast<long long>(budget - fixed) / static_cast<long long>(ki.res_obs_bytes)) & ~3LL;
    const long long want = (long long)ki.res_threads * h->res_obs;
    const int rows = comp ? ki.res_max_blocks_comp : ki.res_max_blocks;   // rows the block's buffer holds
    const long long nb_max = h->nsm < rows ? h->nsm : rows;
    long long nb = (V + want - 1) / want;
    if (nb > nb_max) nb = nb_max;
    long long per = (((V + nb - 1) / nb) + 3) & ~3LL;
    if (per > cap) per = cap;
    nb = (V + per - 1) / per;
    if (nb > nb_max) return false;
    *grid = int(nb);
    *per_block = int(per);
    *ns = comp ? ki.nstat + 1 : ki.nstat;
    *smem = fixed + size_t(per) * ki.res_obs_bytes;
    return true;
}

int prepare_launch(vbh_handle *h, int S, long long V, int precision, const float *rd, const float *dd, Launch *L,
                   bool grouped = false, bool comp = false, int loop = VBH_LOOP_STREAM)
{
    L->S = S;
    const int M = S - 1;
    const size_t nstat = size_t(M * (M + 1) / 2 + M + 4);   // room for the compensated form's extra column
    if (grouped) {
        // one histogram pass, then sweeps over the 2^S profile codes
        if (S > vbh::GROUPED_SMAX || loop == VBH_LOOP_RESIDENT) return VBH_EUNSUPPORTED;
        L->grp = true;
        L->P = 1 << S;
        if (!vbh::tc_kernel_info(3, &L->tki)) return VBH_EUNSUPPORTED;          // the runtime-M set-up kernel
        int rc = ensure(reinterpret_cast<void **>(&h->gstats), &h->gstats_cap, size_t(3) * L->P * sizeof(double));
        if (rc) return rc;
        if (!h->counts) {
            size_t cap = 0;
            if ((rc = ensure(reinterpret_cast<void **>(&h->counts), &cap, 2 * sizeof(unsigned long long)))) return rc;
        }
        VBH_CK(cudaMemsetAsync(h->gstats, 0, size_t(3) * L->P * sizeof(double), h->stream));
        VBH_CK(cudaMemsetAsync(h->counts, 0, 2 * sizeof(unsigned long long), h->stream));
        if ((rc = vbh::grouped_histogram(rd, dd, V, S, h->gstats, h->counts + 1, h->stream, h->nsm))) return rc;
        unsigned long long nonbin = 0;
        VBH_CK(cudaMemcpyAsync(&nonbin, h->counts + 1, sizeof(nonbin), cudaMemcpyDeviceToHost, h->stream));
        VBH_CK(cudaStreamSynchronize(h->stream));
        if (nonbin != 0) return VBH_EINVAL;                                      // the grouped form needs binary d
        L->gstats = h->gstats;
        long long g = vbh::grouped_grid(S, h->nsm);
        if (g > vbh::GRID_MAX) g = vbh::GRID_MAX;
        L->grid = int(g);
        return ensure(reinterpret_cast<void **>(&h->partials), &h->partials_cap,
                      size_t(vbh::partial_rows(g)) * nstat * sizeof(double));
    }
    if (S <= vbh::S_FP32_MAX) {
        L->tc = false;
        L->comp = comp;
        if (!kernel_info(S, &L->ki)) return VBH_EUNSUPPORTED;
        if (!h->attr_set[S]) {
            VBH_CK(cudaFuncSetAttribute(L->ki.sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, int(L->ki.smem)));
            VBH_CK(cudaFuncSetAttribute(L->ki.sweep_comp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        int(L->ki.smem_comp)));
            h->attr_set[S] = true;
        }
    } else {
        if (V >= (1LL << 31)) return VBH_EUNSUPPORTED;
        L->tc = true;
        L->nsplit = (precision == VBH_BF16) ? 2 : 3;
        if (!vbh::tc_kernel_info(L->nsplit, &L->tki)) return VBH_EUNSUPPORTED;
        VBH_CK(cudaFuncSetAttribute(L->tki.sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, int(L->tki.smem)));
    }
    int per_sm = 0;
    VBH_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, L->func(), L->threads(), L->smem()));
    if (per_sm < 1) {
        vbh::record_error("occupancy of the sweep kernel", __FILE__, __LINE__, "no block fits on an SM");
        return VBH_ECUDA;
    }
    if (L->tc) per_sm = 1;                                   // one CTA per SM owns all 512 TMEM columns
    long long tiles = (V + L->tile() - 1) / L->tile();
    long long g = (long long)h->nsm * per_sm;
    if (tiles < g) g = tiles;
    if (g > vbh::GRID_MAX) g = vbh::GRID_MAX;
    if (g < 1) g = 1;
    L->grid = int(g);
    long long rows = vbh::partial_rows(g);
    if (!L->tc && loop != VBH_LOOP_STREAM) {
        // the resident kernels are opted in to the whole shared-memory budget once, so
        // that the shape below can take any block size within it
        const size_t budget = size_t(h->smem_optin) - 1024;
        size_t &set = h->res_attr[S][L->comp ? 1 : 0];
        if (set < budget) {
            VBH_CK(cudaFuncSetAttribute(L->res_func(), cudaFuncAttributeMaxDynamicSharedMemorySize, int(budget)));
            set = budget;
        }
        L->res = resident_shape(h, L->ki, L->comp, V, &L->res_grid, &L->res_per_block, &L->res_ns, &L->res_smem);
        if (!L->res && loop == VBH_LOOP_RESIDENT) return VBH_EUNSUPPORTED;
        if (L->res) {
            int per = 0;
            VBH_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, L->res_func(), L->ki.res_threads, L->res_smem));
            if (per < 1 || (long long)per * h->nsm < L->res_grid) {
                L->res = false;
                if (loop == VBH_LOOP_RESIDENT) return VBH_EUNSUPPORTED;
            }
        }
        if (L->res) {
            if (2LL * L->res_grid > rows) rows = 2LL * L->res_grid;
            int rc = ensure(reinterpret_cast<void **>(&h->res_priv), &h->res_priv_cap,
                            sizeof(DevState) * size_t(L->res_grid > 1 ? L->res_grid - 1 : 1));
            if (rc) return rc;
        }
    } else if (loop == VBH_LOOP_RESIDENT) {
        return VBH_EUNSUPPORTED;
    }
    int rc = ensure(reinterpret_cast<void **>(&h->partials), &h->partials_cap, size_t(rows) * nstat * sizeof(double));
    if (rc) return rc;
    if (L->tc && V > 0) {
        if ((rc = ensure(&h->tc_tiles, &h->tc_cap, vbh::tc_input_bytes(V)))) return rc;
        if (!h->counts) {
            size_t cap = 0;
            if ((rc = ensure(reinterpret_cast<void **>(&h->counts), &cap, 2 * sizeof(unsigned long long)))) return rc;
        }
        VBH_CK(cudaMemsetAsync(h->counts, 0, 2 * sizeof(unsigned long long), h->stream));
        if ((rc = vbh::tc_convert_inputs(dd, rd, V, S, h->tc_tiles, h->counts, h->stream, h->nsm))) return rc;
        unsigned long long cnt[2] = {0, 0};
        VBH_CK(cudaMemcpyAsync(cnt, h->counts, sizeof(cnt), cudaMemcpyDeviceToHost, h->stream));
        VBH_CK(cudaStreamSynchronize(h->stream));
        // the FP32 form needs differences d_j - d_S that BF16 holds exactly (binary profiles give -1, 0, 1)
        if (cnt[0] != 0 && precision != VBH_BF16) return VBH_EUNSUPPORTED;
        L->binary = cnt[1] == 0 ? 1 : 0;
        L->tiles = static_cast<const unsigned char *>(h->tc_tiles);
    }
    return VBH_OK;
}

// Switch of a VBH_BF16 fit to its FP32 sweeps: clear the convergence flag of
// the 16-bit sweeps and cap the FP32 ones.
__global__ void refine_phase_kernel(DevState *st, int max_iter)
{
    if (threadIdx.x == 0) {
        st->converged = 0;
        st->max_iter = max_iter;
    }
}

int launch_sweep(vbh_handle *h, DevState *st, int mode, Launch &L, const float *r, const float *d, long long V)
{
    vbh::SweepArgs a{};
    a.r = r;
    a.d = d;
    a.V = V;
    a.st = st;
    a.partials = h->partials;
    a.use_cond = 0;
    a.mode = mode;
    if (L.grp) {
        vbh::GroupArgs ga{a, L.gstats, L.P};
        void *args[] = {&ga};
        VBH_CK(cudaLaunchKernel(L.func(), dim3(L.grid), dim3(L.threads()), args, L.smem(), h->stream));
    } else if (L.tc) {
        vbh::TcArgs ta{a, L.tiles, L.S, L.binary};
        void *args[] = {&ta};
        VBH_CK(cudaLaunchKernel(L.tki.sweep, dim3(L.grid), dim3(L.tki.threads), args, L.tki.smem, h->stream));
    } else {
        void *args[] = {&a};
        VBH_CK(cudaLaunchKernel(L.func(), dim3(L.grid), dim3(L.ki.threads), args, L.smem(), h->stream));
    }
    return VBH_OK;
}

// Every sweep of a step in one cooperative launch of the resident kernel.
int launch_resident(vbh_handle *h)
{
    Launch &L = h->L;
    vbh::ResidentArgs ra{};
    ra.r = h->r;
    ra.d = h->d;
    ra.V = h->V;
    ra.st = h->st;
    ra.priv = h->res_priv;
    ra.partials = h->partials;
    ra.per_block = L.res_per_block;
    VBH_CK(cudaMemsetAsync(h->partials, 0, sizeof(double) * 2 * size_t(L.res_grid) * L.res_ns, h->stream));
    void *args[] = {&ra};
    VBH_CK(cudaLaunchCooperativeKernel(L.res_func(), dim3(L.res_grid), dim3(L.ki.res_threads), args, L.res_smem,
                                       h->stream));
    return VBH_OK;
}

int launch_setup(vbh_handle *h, DevState *st, const Launch &L, int init)
{
    void *args[] = {&st, &init};
    VBH_CK(cudaLaunchKernel(L.setup(), dim3(1), dim3(32), args, 0, h->stream));
    return VBH_OK;
}

int build_graph(vbh_handle *h)
{
    Launch &L = h->L;
    if (h->gexec && h->g_S == h->S && h->g_grid == L.grid && h->g_V == h->V && h->g_r == h->r && h->g_d == h->d &&
        h->g_partials == h->partials && h->g_func == L.func() && h->g_tiles == (L.tc ? h->tc_tiles : nullptr) &&
        h->g_gstats == (L.grp ? L.gstats : nullptr))
        return VBH_OK;
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    cudaGraph_t g = nullptr;
    VBH_CK(cudaGraphCreate(&g, 0));
    int rc = VBH_OK;
    cudaGraphConditionalHandle cond;
    cudaGraphNodeParams cp{};
    cudaGraphNode_t wnode, knode, knode2;
    cudaGraphNodeParams kp{};
    vbh::SweepArgs a{};
    vbh::TcArgs ta{};
    vbh::GroupArgs ga{};
    void *args[] = {&a};
    void *targs[] = {&ta};
    void *gargs[] = {&ga};
    if (cudaGraphConditionalHandleCreate(&cond, g, 1u, cudaGraphCondAssignDefault) != cudaSuccess) {
        vbh::record_error("cudaGraphConditionalHandleCreate", __FILE__, __LINE__, cudaGetErrorName(cudaGetLastError()));
        rc = VBH_ECUDA;
        goto out;
    }
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if (cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &cp) != cudaSuccess) {
        vbh::record_error("cudaGraphAddNode(while)", __FILE__, __LINE__, cudaGetErrorName(cudaGetLastError()));
        rc = VBH_ECUDA;
        goto out;
    }
    a.r = h->r;
    a.d = h->d;
    a.V = h->V;
    a.st = h->st;
    a.partials = h->partials;
    a.cond = cond;
    a.use_cond = 1;
    a.mode = vbh::MODE_ITER;
    ga.sa = a;
    ga.stats = L.gstats;
    ga.P = L.P;
    ta.sa = a;
    ta.tiles = L.tiles;
    ta.S = L.S;
    ta.binary = L.binary;
    kp.type = cudaGraphNodeTypeKernel;
    kp.kernel.func = const_cast<void *>(L.func());
    kp.kernel.gridDim = dim3(L.grid);
    kp.kernel.blockDim = dim3(L.threads());
    kp.kernel.sharedMemBytes = (unsigned)L.smem();
    kp.kernel.kernelParams = L.grp ? gargs : L.tc ? targs : args;
    // two sweeps per iteration of the while node: the second launch does no pass when the
    // first converged or used up the sweep budget (the kernel checks the state first), and
    // the conditional is evaluated half as often
    if (cudaGraphAddNode(&knode, cp.conditional.phGraph_out[0], nullptr, nullptr, 0, &kp) != cudaSuccess ||
        cudaGraphAddNode(&knode2, cp.conditional.phGraph_out[0], &knode, nullptr, 1, &kp) != cudaSuccess) {
        vbh::record_error("cudaGraphAddNode(sweep)", __FILE__, __LINE__, cudaGetErrorName(cudaGetLastError()));
        rc = VBH_ECUDA;
        goto out;
    }
    if (cudaGraphInstantiate(&h->gexec, g, 0) != cudaSuccess) {
        vbh::record_error("cudaGraphInstantiate", __FILE__, __LINE__, cudaGetErrorName(cudaGetLastError()));
        h->gexec = nullptr;
        rc = VBH_ECUDA;
        goto out;
    }
    h->g_S = h->S;
    h->g_grid = L.grid;
    h->g_V = h->V;
    h->g_r = h->r;
    h->g_d = h->d;
    h->g_partials = h->partials;
    h->g_func = L.func();
    h->g_tiles = L.tc ? h->tc_tiles : nullptr;
    h->g_gstats = L.grp ? L.gstats : nullptr;
out:
    if (rc) (void)cudaGetLastError();
    cudaGraphDestroy(g);
    return rc;
}

int read_state(vbh_handle *h, DevState *st)
{
    VBH_CK(cudaMemcpyAsync(h->mirror, st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
    VBH_CK(cudaStreamSynchronize(h->stream));
    return VBH_OK;
}

void to_result(const DevState &s, vbh_result *out)
{
    std::memset(out, 0, sizeof(*out));
    const int M = s.M;
    out->S = s.S;
    out->iters = s.iter;
    out->converged = s.converged;
    out->status = s.status;
    out->elbo_const_dropped = s.const_dropped;
    double sum = 0.0;
    for (int j = 0; j < M; ++j) {
        out->kappa[j] = s.kappa[j];
        out->weights[j] = s.kappa[j];
        sum += s.kappa[j];
    }
    out->weights[M] = 1.0 - sum;
    std::memcpy(out->W_inv, s.Winv, sizeof(double) * M * M);
    out->nu = s.nu;
    out->lambda = s.lam;
    out->a_rho = s.a_rho;
    out->b_rho = s.b_rho;
    out->rho_mean = s.a_rho / s.b_rho;
    out->rho_mode = s.em ? out->rho_mean : (s.a_rho - 1.0) / s.b_rho;   // EM: the point estimate
    out->elbo = s.elbo;
}

int check_common(vbh_handle *h, const float *r, const float *d, int64_t V, int S)
{
    if (!h) return VBH_EINVAL;
    if (S < 1 || S > VBH_SMAX) return VBH_EINVAL;
    if (V < 0 || V > (int64_t(1) << 40)) return VBH_EINVAL;
    if (V > 0 && (!r || !d)) return VBH_EINVAL;
    return VBH_OK;
}

} // namespace

extern "C" {

void vbh_prior_default(int S, vbh_prior *p)
{
    if (!p) return;
    p->S = S;
    p->K0 = nullptr;
    p->q0 = 1e-3;
    p->n0 = 1.0;
    p->a0 = 0.5;
    p->b0 = 0.5;
    p->Lambda0_inv = nullptr;
}

void vbh_opts_default(vbh_opts *o)
{
    if (!o) return;
    o->tol = 1e-8;
    o->max_iter = 200;
    o->precision = VBH_FP32;
    o->refine_iters = 10;
    o->method = VBH_CAVI;
    o->grouped = 0;
    o->stats = VBH_STATS_AUTO;
    o->loop = VBH_LOOP_AUTO;
    o->init = VBH_INIT_PAPER;
    o->init_state = nullptr;
    o->elbo_trace = nullptr;
}

const char *vbh_strerror(int status)
{
    switch (status) {
    case VBH_OK: return "ok";
    case VBH_EINVAL: return "invalid argument";
    case VBH_ENOMEM: return "out of memory";
    case VBH_ECUDA: return "CUDA runtime error";
    case VBH_ENONFINITE: return "non-finite global update or ELBO";
    case VBH_ETIMEOUT: return "bounded device wait ran out";
    case VBH_ESTATE: return "call out of order";
    case VBH_EUNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
    }
}

size_t vbh_state_bytes(void) { return sizeof(DevState); }

const char *vbh_last_error_detail(void) { return vbh::last_error_buf(); }

int vbh_create(vbh_handle **hp, int device, void *stream)
{
    if (!hp) return VBH_EINVAL;
    *hp = nullptr;
    // a failing CUDA call is recorded for vbh_last_error_detail and mapped to a status
    auto failed = [](cudaError_t e, const char *what, int line, int status) -> int {
        if (e == cudaSuccess) return VBH_OK;
        vbh::record_error(what, __FILE__, line, cudaGetErrorName(e));
        (void)cudaGetLastError();
        return status;
    };
    int ndev = 0;
    if (int rc0 = failed(cudaGetDeviceCount(&ndev), "cudaGetDeviceCount(&ndev)", __LINE__, VBH_ECUDA)) return rc0;
    if (device < 0 || device >= ndev) return VBH_EINVAL;
    DeviceGuard g(device);
    if (!g.ok) {
        const cudaError_t e = cudaGetLastError();
        return failed(e != cudaSuccess ? e : cudaErrorInvalidDevice, "cudaSetDevice(device)", __LINE__, VBH_ECUDA);
    }
    vbh_handle *h = new (std::nothrow) vbh_handle();
    if (!h) return VBH_ENOMEM;
    h->device = device;
    h->stream = static_cast<cudaStream_t>(stream);
    const char *launch = std::getenv("VBH_LAUNCH");
    h->direct = launch && std::strcmp(launch, "direct") == 0;
    if (const char *ro = std::getenv("VBH_RESIDENT_OBS")) {
        const int v = std::atoi(ro);
        if (v >= 1 && v <= 4096) h->res_obs = v;
    }
    int coop = 0;
    int rc = failed(cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, device),
                    "cudaDeviceGetAttribute(MultiProcessorCount)", __LINE__, VBH_ECUDA);
    if (!rc) rc = failed(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device),
                         "cudaDeviceGetAttribute(CooperativeLaunch)", __LINE__, VBH_ECUDA);
    if (!rc) rc = failed(cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device),
                         "cudaDeviceGetAttribute(MaxSharedMemoryPerBlockOptin)", __LINE__, VBH_ECUDA);
    h->coop = coop != 0;
    if (!rc) rc = failed(cudaMalloc(&h->st, sizeof(DevState)), "cudaMalloc(state)", __LINE__, VBH_ENOMEM);
    if (!rc) rc = failed(cudaMalloc(&h->st_aux, sizeof(DevState)), "cudaMalloc(state)", __LINE__, VBH_ENOMEM);
    if (!rc) rc = failed(cudaMallocHost(&h->mirror, sizeof(DevState)), "cudaMallocHost(mirror)", __LINE__, VBH_ENOMEM);
    for (int i = 0; !rc && i < vbh_handle::NCOPY; ++i)
        rc = failed(cudaStreamCreateWithFlags(&h->copy_stream[i], cudaStreamNonBlocking), "cudaStreamCreateWithFlags",
                    __LINE__, VBH_ECUDA);
    for (int i = 0; !rc && i <= vbh_handle::NCOPY; ++i)
        rc = failed(cudaEventCreateWithFlags(&h->copy_event[i], cudaEventDisableTiming), "cudaEventCreateWithFlags",
                    __LINE__, VBH_ECUDA);
    if (rc) {
        (void)cudaGetLastError();
        vbh_destroy(h);
        return rc;
    }
    *hp = h;
    return VBH_OK;
}

void vbh_destroy(vbh_handle *h)
{
    if (!h) return;
    DeviceGuard g(h->device);
    cudaStreamSynchronize(h->stream);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    cudaFree(h->st);
    cudaFree(h->st_aux);
    cudaFree(h->partials);
    cudaFree(h->trace);
    cudaFree(h->stage_r);
    cudaFree(h->stage_d);
    cudaFree(h->tc_tiles);
    cudaFree(h->gstats);
    cudaFree(h->counts);
    cudaFree(h->res_priv);
    if (h->mirror) cudaFreeHost(h->mirror);
    for (int i = 0; i < vbh_handle::NCOPY; ++i)
        if (h->copy_stream[i]) {
            cudaStreamSynchronize(h->copy_stream[i]);
            cudaStreamDestroy(h->copy_stream[i]);
        }
    for (int i = 0; i <= vbh_handle::NCOPY; ++i)
        if (h->copy_event[i]) cudaEventDestroy(h->copy_event[i]);
    cudaFree(h->batched.arena);
    if (h->batched.host_states) cudaFreeHost(h->batched.host_states);
    (void)cudaGetLastError();
    delete h;
}

int vbh_fit_begin(vbh_handle *h, const float *r, const float *d, int64_t V, int S, const vbh_prior *p,
                  const vbh_opts *o)
{
    int rc = check_common(h, r, d, V, S);
    if (rc) return rc;
    if ((rc = check_prior(p, S))) return rc;
    if (!o || o->max_iter < 0 || !(o->tol >= 0.0) || !std::isfinite(o->tol) ||
        (o->precision != VBH_FP32 && o->precision != VBH_BF16))
        return VBH_EINVAL;
    if (o->precision == VBH_BF16 && o->refine_iters < 0) return VBH_EINVAL;
    if (o->method != VBH_CAVI && o->method != VBH_EM) return VBH_EINVAL;
    const bool em = o->method == VBH_EM;
    if (o->init != VBH_INIT_PAPER && o->init != VBH_INIT_GIVEN) return VBH_EINVAL;
    if (o->init == VBH_INIT_GIVEN && (!o->init_state || o->init_state->S != S)) return VBH_EINVAL;
    DeviceGuard g(h->device);
    if (!g.ok) return VBH_ECUDA;
    h->begun = false;
    const float *rd = nullptr, *dd = nullptr;
    if ((rc = stage_inputs(h, r, d, V, S, &rd, &dd))) return rc;
    if (o->grouped != 0 && o->grouped != 1) return VBH_EINVAL;
    if (o->stats != VBH_STATS_AUTO && o->stats != VBH_STATS_COMPENSATED && o->stats != VBH_STATS_PLAIN)
        return VBH_EINVAL;
    if (o->loop != VBH_LOOP_AUTO && o->loop != VBH_LOOP_STREAM && o->loop != VBH_LOOP_RESIDENT) return VBH_EINVAL;
    const bool comp = o->stats == VBH_STATS_COMPENSATED || (o->stats == VBH_STATS_AUTO && o->tol > 0.0);
    Launch L;
    if ((rc = prepare_launch(h, S, V, o->precision, rd, dd, &L, o->grouped == 1, comp, o->loop))) return rc;
    if (o->max_iter + 1 > h->trace_cap) {
        size_t cap = 0;
        cudaFree(h->trace);
        h->trace = nullptr;
        h->trace_cap = 0;
        if ((rc = ensure(reinterpret_cast<void **>(&h->trace), &cap, sizeof(double) * size_t(o->max_iter + 1))))
            return rc;
        h->trace_cap = o->max_iter + 1;
    }
    DevState *s = h->mirror;
    VBH_CK(cudaStreamSynchronize(h->stream));     // the mirror may still be a copy target
    std::memset(s, 0, sizeof(DevState));
    fill_prior(s, p, S, V);
    s->tol = o->tol;
    s->max_iter = o->max_iter;
    s->target = 0;
    s->trace = h->trace;
    s->em = em ? 1 : 0;
    s->comp = L.comp ? 1 : 0;
    const int M = S - 1;
    if (em && o->init == VBH_INIT_PAPER) {
        // theta^(0) from the prior: K0, Lambda_0^{-1}, rho = a0 / b0 (as (a_rho, b_rho) = (rho, 1), nu = 1)
        for (int j = 0; j < M; ++j) s->kappa[j] = s->K0[j];
        for (int j = 0; j < M * M; ++j) s->Winv[j] = s->L0inv[j];
        s->a_rho = p->a0 / p->b0;
        s->b_rho = 1.0;
        s->nu = 1.0;
        s->lam = double(V);
    } else if (o->init == VBH_INIT_GIVEN) {
        const vbh_result *q = o->init_state;
        if (!pos_finite(q->a_rho) || !pos_finite(q->b_rho)) return VBH_EINVAL;
        if (!em && (!(q->nu > M - 1.0) || !pos_finite(q->lambda))) return VBH_EINVAL;
        if (!host_spd(M, q->W_inv)) return VBH_EINVAL;
        s->a_rho = em ? q->a_rho / q->b_rho : q->a_rho;
        s->b_rho = em ? 1.0 : q->b_rho;
        s->nu = em ? 1.0 : q->nu;
        s->lam = em ? double(V) : q->lambda;
        for (int j = 0; j < M; ++j) s->kappa[j] = q->kappa[j];
        symmetrize(M, q->W_inv, s->Winv);
    }
    // the 16-bit sweeps of a VBH_BF16 fit, then its FP32 ones
    const bool bf16 = L.tc && !L.grp && L.nsplit == 2;
    const int refine = bf16 ? (o->refine_iters < o->max_iter ? o->refine_iters : o->max_iter) : 0;
    if (bf16) s->max_iter = o->max_iter - refine;
    VBH_CK(cudaMemcpyAsync(h->st, s, sizeof(DevState), cudaMemcpyHostToDevice, h->stream));
    if (em) {
        // EM iteration 0 from theta^(0): ln p(r | theta^(0)), then theta^(1)
        if ((rc = launch_setup(h, h->st, L, 0))) return rc;
        if ((rc = launch_sweep(h, h->st, vbh::MODE_INIT, L, rd, dd, V))) return rc;
    } else if (o->init == VBH_INIT_GIVEN) {
        // sweep 0 = the ELBO of the given factors (Q(beta) from them); the
        // sweeps that follow update all factors
        if ((rc = launch_setup(h, h->st, L, 0))) return rc;
        if ((rc = launch_sweep(h, h->st, vbh::MODE_ELBO, L, rd, dd, V))) return rc;
    } else {
        if ((rc = launch_setup(h, h->st, L, 1))) return rc;
        if ((rc = launch_sweep(h, h->st, vbh::MODE_INIT, L, rd, dd, V))) return rc;
    }
    if ((rc = read_state(h, h->st))) return rc;
    if (h->mirror->status) return h->mirror->status;
    h->begun = true;
    h->S = S;
    h->V = V;
    h->r = rd;
    h->d = dd;
    h->L = L;
    h->bf16_phase = bf16;
    h->bf16_limit = o->max_iter - refine;
    h->refine = refine;
    h->max_iter = o->max_iter;
    h->user_trace = o->elbo_trace;
    return VBH_OK;
}

namespace {
// Up to n sweeps of the current kernel (fewer on convergence or at the caps).
int run_sweeps(vbh_handle *h, int n)
{
    int rc = VBH_OK;
    vbh::set_target_kernel<<<1, 32, 0, h->stream>>>(h->st, n);
    VBH_CK(cudaGetLastError());
    if (h->L.res) {
        if ((rc = launch_resident(h))) return rc;
    } else if (h->direct) {
        // each launch checks the control fields first and does nothing once the
        // fit has converged or reached its target
        const int m = n < h->max_iter ? n : h->max_iter;
        for (int i = 0; i < m; ++i)
            if ((rc = launch_sweep(h, h->st, vbh::MODE_ITER, h->L, h->r, h->d, h->V))) return rc;
    } else {
        if ((rc = build_graph(h))) return rc;
        VBH_CK(cudaGraphLaunch(h->gexec, h->stream));
    }
    return read_state(h, h->st);
}
} // namespace

int vbh_fit_step(vbh_handle *h, int nsweeps, int *converged)
{
    if (!h || nsweeps < 0) return VBH_EINVAL;
    if (!h->begun) return VBH_ESTATE;
    DeviceGuard g(h->device);
    if (!g.ok) return VBH_ECUDA;
    int rc = VBH_OK;
    int left = nsweeps;
    if (h->bf16_phase) {
        const int it0 = h->mirror->iter;
        if (left > 0 && (rc = run_sweeps(h, left))) return rc;
        left -= h->mirror->iter - it0;
        if (h->mirror->status) return h->mirror->status;
        if (h->mirror->converged || h->mirror->iter >= h->bf16_limit) {
            // switch to the FP32 sweeps: same BF16 profiles and tensor maps, three-part operands
            Launch &L = h->L;
            L.nsplit = 3;
            if (!vbh::tc_kernel_info(3, &L.tki)) return VBH_EUNSUPPORTED;
            VBH_CK(cudaFuncSetAttribute(L.tki.sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, int(L.tki.smem)));
            const int cap = h->mirror->iter + h->refine < h->max_iter ? h->mirror->iter + h->refine : h->max_iter;
            refine_phase_kernel<<<1, 32, 0, h->stream>>>(h->st, cap);
            VBH_CK(cudaGetLastError());
            h->bf16_phase = false;
            if ((rc = read_state(h, h->st))) return rc;
        }
    }
    if (!h->bf16_phase && left > 0 && (rc = run_sweeps(h, left))) return rc;
    if (converged) *converged = h->mirror->converged;
    return h->mirror->status;
}

int vbh_fit_result(vbh_handle *h, vbh_result *out)
{
    if (!h || !out) return VBH_EINVAL;
    if (!h->begun) return VBH_ESTATE;
    DeviceGuard g(h->device);
    if (!g.ok) return VBH_ECUDA;
    int rc = read_state(h, h->st);
    if (rc) return rc;
    to_result(*h->mirror, out);
    if (h->user_trace) {
        const int n = h->mirror->iter + 1;
        VBH_CK(cudaMemcpyAsync(h->user_trace, h->trace, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
        VBH_CK(cudaStreamSynchronize(h->stream));
    }
    return out->status;
}

int vbh_fit(vbh_handle *h, const float *r, const float *d, int64_t V, int S, const vbh_prior *p,
            const vbh_opts *o, vbh_result *out)
{
    if (!out) return VBH_EINVAL;
    int rc = vbh_fit_begin(h, r, d, V, S, p, o);
    if (rc) return rc;
    int conv = 0;
    if (o->max_iter > 0) {
        rc = vbh_fit_step(h, o->max_iter, &conv);
        if (rc) {
            vbh_fit_result(h, out);
            return rc;
        }
    }
    return vbh_fit_result(h, out);
}

int vbh_fit_batched(vbh_handle *h, int B, const int64_t *V, const int *S, const float *const *r,
                    const float *const *d, const vbh_prior *p, const vbh_opts *o, vbh_result *out)
{
    if (!h) return VBH_EINVAL;
    DeviceGuard g(h->device);
    if (!g.ok) return VBH_ECUDA;
    h->begun = false;                  // the step-wise fit's staging buffers are not touched, but keep it simple
    return vbh::fit_batched_impl(h->batched, h->stream, h->nsm, B, V, S, r, d, p, o, out, h->direct);
}

int vbh_batched_plan(vbh_handle *h, vbh_batch_plan *out, int cap, int *n)
{
    if (!h || !n || cap < 0 || (cap > 0 && !out)) return VBH_EINVAL;
    const auto &plan = h->batched.plan;
    *n = int(plan.size());
    for (int i = 0; i < cap && i < int(plan.size()); ++i) out[i] = plan[size_t(i)];
    return VBH_OK;
}

int vbh_elbo(vbh_handle *h, const float *r, const float *d, int64_t V, int S, const vbh_prior *p,
             const vbh_result *q, double *elbo)
{
    int rc = check_common(h, r, d, V, S);
    if (rc) return rc;
    if ((rc = check_prior(p, S))) return rc;
    if (!q || !elbo || q->S != S) return VBH_EINVAL;
    const int M = S - 1;
    if (!pos_finite(q->a_rho) || !pos_finite(q->b_rho) || !(q->nu > M - 1.0) || !pos_finite(q->lambda))
        return VBH_EINVAL;
    if (!host_spd(M, q->W_inv)) return VBH_EINVAL;
    DeviceGuard g(h->device);
    if (!g.ok) return VBH_ECUDA;
    const float *rd = nullptr, *dd = nullptr;
    if ((rc = stage_inputs(h, r, d, V, S, &rd, &dd))) return rc;
    // a fit in progress loses its inputs when the staging buffers, the BF16
    // profiles or the partials buffer are reused here
    if (h->begun && (rd != h->r || dd != h->d || S > vbh::S_FP32_MAX || h->L.tc)) h->begun = false;
    Launch L;
    if ((rc = prepare_launch(h, S, V, VBH_FP32, rd, dd, &L, false, true))) return rc;
    DevState *s = h->mirror;
    VBH_CK(cudaStreamSynchronize(h->stream));
    std::memset(s, 0, sizeof(DevState));
    fill_prior(s, p, S, V);
    s->comp = L.comp ? 1 : 0;
    s->a_rho = q->a_rho;
    s->b_rho = q->b_rho;
    s->nu = q->nu;
    s->lam = q->lambda;
    for (int j = 0; j < M; ++j) s->kappa[j] = q->kappa[j];
    symmetrize(M, q->W_inv, s->Winv);
    VBH_CK(cudaMemcpyAsync(h->st_aux, s, sizeof(DevState), cudaMemcpyHostToDevice, h->stream));
    if ((rc = launch_setup(h, h->st_aux, L, 0))) return rc;
    if ((rc = launch_sweep(h, h->st_aux, vbh::MODE_ELBO, L, rd, dd, V))) return rc;
    if ((rc = read_state(h, h->st_aux))) return rc;
    *elbo = h->mirror->elbo;
    return h->mirror->status;
}

} // extern "C"
