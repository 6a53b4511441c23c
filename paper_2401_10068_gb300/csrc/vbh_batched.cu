// vbh_batched.cu -- vbh_fit_batched: many independent fits in one device loop.
//
// Host side of the batched form (kernels in vbh_batched.cuh): argument checks,
// input staging, the per-class work lists (chunks of contiguous observations,
// largest first), the chunk-size autotuner, and the CUDA graph whose while
// loop runs one batched sweep per iteration: for every S class in parallel a
// data pass and the per-data-set updates, then the control kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include "vbh.h"
#include "vbh_batched.cuh"
#include "vbh_batched_host.h"
#include "vbh_dispatch.cuh"

namespace vbh {

// After all classes' updates: continue while a data set is running.
__global__ void batched_control_kernel(BatchControl *ctl, cudaGraphConditionalHandle cond, int use_cond)
{
    if (threadIdx.x != 0) return;
    ctl->sweep += 1;
    const unsigned int keep = (ctl->active > 0 && ctl->sweep < ctl->max_sweeps) ? 1u : 0u;
    ctl->active = 0;
    for (unsigned int c = 0; c < ctl->nclasses; ++c) *ctl->class_next[c] = 0u;
    if (use_cond) cudaGraphSetConditional(cond, keep);
}


namespace {

#define VBH_B_CK(call)                                                                                                 \
    do {                                                                                                               \
        cudaError_t e_ = (call);                                                                                       \
        if (e_ != cudaSuccess) {                                                                                       \
            (void)cudaGetLastError();                                                                                  \
            return e_ == cudaErrorMemoryAllocation ? VBH_ENOMEM : VBH_ECUDA;                                           \
        }                                                                                                              \
    } while (0)

bool batch_info(int S, BatchKernelInfo *bi)
{
    return batch_kernel_info_s1_4(S, bi) || batch_kernel_info_s5_8(S, bi) || batch_kernel_info_s9_11(S, bi);
}

bool spd_sym(int M, const double *A)
{
    double L[MMAX * MMAX];
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

bool fpos(double x) { return std::isfinite(x) && x > 0.0; }

// Bump allocator over one device buffer owned by the handle.
struct Arena {
    unsigned char *base = nullptr;
    size_t cap = 0, used = 0;
    void *take(size_t bytes)
    {
        used = (used + 255) / 256 * 256;
        void *p = base + used;
        used += bytes;
        return p;
    }
};

struct ClassPlan {
    int S = 0;
    BatchKernelInfo bi{};
    BatchPassInfo pi{};                     // the pass of the chosen form (plain or compensated)
    std::vector<int> ds;                    // data sets of the class
    std::vector<int> chunk_ds;
    std::vector<long long> lo, hi;
    std::vector<int> order;
    int max_stages = 0;                     // most stages whose ring fits one block
    int stages = 0;                         // the pass's stages (autotuned)
    int chunk_tiles = 0;                    // tiles per chunk (autotuned)
    int grid = 0;                           // persistent blocks of the pass at `stages`
    int per_sm = 0;
    float pass_ms = 0.f;                    // the autotuner's time of the chosen pass (0: not timed)
    size_t smem() const { return pi.fixed + size_t(stages) * pi.stage_bytes; }
};

void build_chunks(ClassPlan &cp, const int64_t *V, int chunk_tiles, std::vector<int> &first, std::vector<int> &nch)
{
    cp.chunk_ds.clear();
    cp.lo.clear();
    cp.hi.clear();
    const long long T = cp.pi.tile;
    for (int b : cp.ds) {
        const long long ntiles = V[b] / T;
        const long long per = chunk_tiles;
        const long long n = std::max<long long>(1, (ntiles + per - 1) / per);
        first[b] = int(cp.chunk_ds.size());
        nch[b] = int(n);
        for (long long j = 0; j < n; ++j) {
            cp.chunk_ds.push_back(b);
            cp.lo.push_back(j * per * T);
            cp.hi.push_back(j == n - 1 ? V[b] : (j + 1) * per * T);
        }
    }
    cp.order.resize(cp.chunk_ds.size());
    std::iota(cp.order.begin(), cp.order.end(), 0);
    std::stable_sort(cp.order.begin(), cp.order.end(), [&](int a, int b) {
        return (cp.hi[a] - cp.lo[a]) > (cp.hi[b] - cp.lo[b]);
    });
}

} // namespace

int fit_batched_impl(BatchedHost &hb, cudaStream_t stream, int nsm, int B, const int64_t *V, const int *S,
                     const float *const *r, const float *const *d, const vbh_prior *p, const vbh_opts *o,
                     vbh_result *out, bool direct)
{
    hb.plan.clear();
    // ---------------- arguments ----------------
    if (B < 0 || (B > 0 && (!V || !S || !r || !d || !out)) || !o) return VBH_EINVAL;
    if (B == 0) return VBH_OK;
    if (o->max_iter < 0 || !(o->tol >= 0.0) || !std::isfinite(o->tol) || o->precision != VBH_FP32) return VBH_EINVAL;
    if (o->init != VBH_INIT_PAPER && o->init != VBH_INIT_GIVEN) return VBH_EINVAL;
    if (o->method != VBH_CAVI) return VBH_EUNSUPPORTED;           // this entry point runs CAVI only
    if (o->init == VBH_INIT_GIVEN && !o->init_state) return VBH_EINVAL;
    if (o->stats != VBH_STATS_AUTO && o->stats != VBH_STATS_COMPENSATED && o->stats != VBH_STATS_PLAIN)
        return VBH_EINVAL;
    // the compensated statistics of the stopping test (one more partial column)
    const bool comp = o->stats == VBH_STATS_COMPENSATED || (o->stats == VBH_STATS_AUTO && o->tol > 0.0);
    for (int b = 0; b < B; ++b) {
        if (S[b] < 1 || S[b] > VBH_SMAX || V[b] < 0 || V[b] > (int64_t(1) << 40)) return VBH_EINVAL;
        if (S[b] > S_FP32_MAX) return VBH_EUNSUPPORTED;
        if (V[b] > 0 && (!r[b] || !d[b])) return VBH_EINVAL;
        const int M = S[b] - 1;
        if (p) {
            const vbh_prior &q = p[b];
            if (q.S != S[b] || !fpos(q.q0) || !fpos(q.n0) || !fpos(q.a0) || !fpos(q.b0)) return VBH_EINVAL;
            if (q.K0)
                for (int j = 0; j < M; ++j)
                    if (!std::isfinite(q.K0[j])) return VBH_EINVAL;
            if (q.Lambda0_inv && !spd_sym(M, q.Lambda0_inv)) return VBH_EINVAL;
        }
        if (o->init == VBH_INIT_GIVEN) {
            const vbh_result &g = o->init_state[b];
            if (g.S != S[b] || !fpos(g.a_rho) || !fpos(g.b_rho) || !(g.nu > M - 1.0) || !fpos(g.lambda) ||
                !spd_sym(M, g.W_inv))
                return VBH_EINVAL;
        }
    }
    int device = 0;
    VBH_B_CK(cudaGetDevice(&device));

    // ---------------- inputs: device pointers as given, host inputs staged ----------------
    std::vector<const float *> rdev(B), ddev(B);
    size_t stage_bytes = 0;
    std::vector<int> host_in(B, 0);
    for (int b = 0; b < B; ++b) {
        if (V[b] == 0) continue;
        cudaPointerAttributes ar, ad;
        const bool okr = cudaPointerGetAttributes(&ar, r[b]) == cudaSuccess;
        const bool okd = cudaPointerGetAttributes(&ad, d[b]) == cudaSuccess;
        (void)cudaGetLastError();
        const bool devr = okr && (ar.type == cudaMemoryTypeDevice || ar.type == cudaMemoryTypeManaged);
        const bool devd = okd && (ad.type == cudaMemoryTypeDevice || ad.type == cudaMemoryTypeManaged);
        if (devr != devd) return VBH_EINVAL;                  // both on the device or both on the host
        if (devr) {
            if ((ar.type == cudaMemoryTypeDevice && ar.device != device) ||
                (ad.type == cudaMemoryTypeDevice && ad.device != device))
                return VBH_EINVAL;
            if (reinterpret_cast<uintptr_t>(r[b]) % 16 || reinterpret_cast<uintptr_t>(d[b]) % 16) return VBH_EINVAL;
            rdev[b] = r[b];
            ddev[b] = d[b];
        } else {
            host_in[b] = 1;
            stage_bytes += (size_t(V[b]) * 4 + 255) / 256 * 256 + (size_t(V[b]) * S[b] * 4 + 255) / 256 * 256;
        }
    }

    // ---------------- classes and work lists ----------------
    int smem_optin = 0, rc = VBH_OK;
    VBH_B_CK(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    static const int kCandidates[] = {8, 32, 128};            // tiles per chunk
    static const int kStageCandidates[] = {2, 3, 4, 6, 8};
    constexpr int kDefaultStages = 3;
    // the pass's stages and, from its occupancy at that ring, its persistent grid
    auto set_stages = [&](ClassPlan &cp, int st) -> int {
        cp.stages = st;
        int per_sm = 0;
        VBH_B_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cp.pi.pass, cp.pi.threads, cp.smem()));
        cp.per_sm = per_sm;
        cp.grid = nsm * std::max(per_sm, 1);
        return per_sm >= 1 ? VBH_OK : VBH_EUNSUPPORTED;
    };
    std::vector<ClassPlan> classes;
    for (int s = 1; s <= S_FP32_MAX; ++s) {
        ClassPlan cp;
        cp.S = s;
        for (int b = 0; b < B; ++b)
            if (S[b] == s) cp.ds.push_back(b);
        if (cp.ds.empty()) continue;
        if (!batch_info(s, &cp.bi)) return VBH_EUNSUPPORTED;
        cp.pi = comp ? cp.bi.comp : cp.bi.plain;
        if (comp) cp.bi.nstat += 1;
        cp.max_stages = 0;
        for (int st = 1; st <= cp.pi.max_stages; ++st)
            if (cp.pi.fixed + size_t(st) * cp.pi.stage_bytes + 1024 <= size_t(smem_optin)) cp.max_stages = st;
        if (cp.max_stages < 2) return VBH_EUNSUPPORTED;
        VBH_B_CK(cudaFuncSetAttribute(cp.pi.pass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      int(cp.pi.fixed + size_t(cp.max_stages) * cp.pi.stage_bytes)));
        VBH_B_CK(cudaFuncSetAttribute(cp.bi.update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      int(cp.bi.update_smem)));
        if ((rc = set_stages(cp, std::min(kDefaultStages, cp.max_stages)))) return rc;
        cp.chunk_tiles = kCandidates[1];
        classes.push_back(std::move(cp));
    }
    const int nclass = int(classes.size());
    std::vector<int> first(B, 0), nch(B, 0);

    // upper bound of chunks: smallest candidate chunk size
    size_t max_chunks = 0;
    for (auto &cp : classes) {
        build_chunks(cp, V, kCandidates[0], first, nch);
        max_chunks = std::max(max_chunks, cp.chunk_ds.size());
    }

    // ---------------- device memory (one arena, grown when too small) ----------------
    const int ntrace = o->max_iter + 1;
    size_t need = 0;
    auto add = [&](size_t bytes) { need = (need + 255) / 256 * 256 + bytes; };
    add(sizeof(DevState) * B);
    add(sizeof(double) * size_t(B) * ntrace);
    add(sizeof(float *) * B * 2);
    add(sizeof(long long) * B);
    add(sizeof(int) * B * 2);
    add(sizeof(BatchControl));
    add(sizeof(unsigned int) * (SMAX + 1));
    for (auto &cp : classes) {
        add(sizeof(int) * cp.ds.size());
        add(sizeof(int) * max_chunks * 2);
        add(sizeof(long long) * max_chunks * 2);
        add(sizeof(double) * max_chunks * cp.pi.rows_per_chunk * cp.bi.nstat);
    }
    add(stage_bytes);
    need += 4096;
    if (hb.arena_cap < need) {
        cudaFree(hb.arena);
        hb.arena = nullptr;
        hb.arena_cap = 0;
        VBH_B_CK(cudaMalloc(&hb.arena, need));
        hb.arena_cap = need;
    }
    Arena ar{static_cast<unsigned char *>(hb.arena), hb.arena_cap, 0};
    DevState *states = static_cast<DevState *>(ar.take(sizeof(DevState) * B));
    double *traces = static_cast<double *>(ar.take(sizeof(double) * size_t(B) * ntrace));
    const float **r_ptrs = static_cast<const float **>(ar.take(sizeof(float *) * B));
    const float **d_ptrs = static_cast<const float **>(ar.take(sizeof(float *) * B));
    long long *ds_V = static_cast<long long *>(ar.take(sizeof(long long) * B));
    int *ds_first = static_cast<int *>(ar.take(sizeof(int) * B));
    int *ds_nch = static_cast<int *>(ar.take(sizeof(int) * B));
    BatchControl *ctl = static_cast<BatchControl *>(ar.take(sizeof(BatchControl)));
    unsigned int *counters = static_cast<unsigned int *>(ar.take(sizeof(unsigned int) * (SMAX + 1)));
    struct ClassDev {
        int *ds_list, *chunk_ds, *order;
        long long *lo, *hi;
        double *partials;
    };
    std::vector<ClassDev> cdev(nclass);
    for (int c = 0; c < nclass; ++c) {
        cdev[c].ds_list = static_cast<int *>(ar.take(sizeof(int) * classes[c].ds.size()));
        cdev[c].chunk_ds = static_cast<int *>(ar.take(sizeof(int) * max_chunks));
        cdev[c].order = static_cast<int *>(ar.take(sizeof(int) * max_chunks));
        cdev[c].lo = static_cast<long long *>(ar.take(sizeof(long long) * max_chunks));
        cdev[c].hi = static_cast<long long *>(ar.take(sizeof(long long) * max_chunks));
        cdev[c].partials = static_cast<double *>(
            ar.take(sizeof(double) * max_chunks * classes[c].pi.rows_per_chunk * classes[c].bi.nstat));
    }
    unsigned char *stage = static_cast<unsigned char *>(ar.take(stage_bytes));
    for (int b = 0; b < B; ++b) {
        if (!host_in[b]) continue;
        const size_t br = size_t(V[b]) * 4, bd = size_t(V[b]) * S[b] * 4;
        float *rs = reinterpret_cast<float *>(stage);
        stage += (br + 255) / 256 * 256;
        float *dsg = reinterpret_cast<float *>(stage);
        stage += (bd + 255) / 256 * 256;
        VBH_B_CK(cudaMemcpyAsync(rs, r[b], br, cudaMemcpyHostToDevice, stream));
        VBH_B_CK(cudaMemcpyAsync(dsg, d[b], bd, cudaMemcpyHostToDevice, stream));
        rdev[b] = rs;
        ddev[b] = dsg;
    }

    // ---------------- host-built initial states ----------------
    if (hb.host_states_cap < size_t(B)) {
        if (hb.host_states) cudaFreeHost(hb.host_states);
        hb.host_states = nullptr;
        hb.host_states_cap = 0;
        VBH_B_CK(cudaMallocHost(&hb.host_states, sizeof(DevState) * B));
        hb.host_states_cap = B;
    }
    VBH_B_CK(cudaStreamSynchronize(stream));
    DevState *hs = static_cast<DevState *>(hb.host_states);
    std::memset(hs, 0, sizeof(DevState) * B);
    for (int b = 0; b < B; ++b) {
        DevState &s = hs[b];
        const int Sb = S[b], M = Sb - 1;
        vbh_prior pd;
        vbh_prior_default(Sb, &pd);
        const vbh_prior &q = p ? p[b] : pd;
        s.S = Sb;
        s.M = M;
        s.V = double(V[b]);
        s.q0 = q.q0;
        s.n0 = q.n0;
        s.a0 = q.a0;
        s.b0 = q.b0;
        for (int j = 0; j < M; ++j) s.K0[j] = q.K0 ? q.K0[j] : 1.0 / Sb;
        for (int a = 0; a < M; ++a)
            for (int c = 0; c < M; ++c)
                s.L0inv[a * M + c] = q.Lambda0_inv ? 0.5 * (q.Lambda0_inv[a * M + c] + q.Lambda0_inv[c * M + a])
                                                   : 0.005 + (a == c ? (a % 2 == 0 ? 0.005 : 0.003) : 0.0);
        s.tol = o->tol;
        s.max_iter = o->max_iter;
        s.target = o->max_iter;
        s.trace = traces + size_t(b) * ntrace;
        s.comp = comp ? 1 : 0;
        if (o->init == VBH_INIT_GIVEN) {
            const vbh_result &g = o->init_state[b];
            s.a_rho = g.a_rho;
            s.b_rho = g.b_rho;
            s.nu = g.nu;
            s.lam = g.lambda;
            for (int j = 0; j < M; ++j) s.kappa[j] = g.kappa[j];
            for (int a = 0; a < M; ++a)
                for (int c = 0; c < M; ++c) s.Winv[a * M + c] = 0.5 * (g.W_inv[a * M + c] + g.W_inv[c * M + a]);
        }
    }
    VBH_B_CK(cudaMemcpyAsync(states, hs, sizeof(DevState) * B, cudaMemcpyHostToDevice, stream));
    std::vector<long long> hV(V, V + B);
    VBH_B_CK(cudaMemcpyAsync(r_ptrs, rdev.data(), sizeof(float *) * B, cudaMemcpyHostToDevice, stream));
    VBH_B_CK(cudaMemcpyAsync(d_ptrs, ddev.data(), sizeof(float *) * B, cudaMemcpyHostToDevice, stream));
    VBH_B_CK(cudaMemcpyAsync(ds_V, hV.data(), sizeof(long long) * B, cudaMemcpyHostToDevice, stream));
    BatchControl hctl{};
    hctl.max_sweeps = unsigned(o->max_iter);
    hctl.nclasses = unsigned(nclass);
    for (int c = 0; c < nclass; ++c) hctl.class_next[c] = counters + c;
    VBH_B_CK(cudaMemcpyAsync(ctl, &hctl, sizeof(hctl), cudaMemcpyHostToDevice, stream));
    VBH_B_CK(cudaMemsetAsync(counters, 0, sizeof(unsigned int) * (SMAX + 1), stream));
    VBH_B_CK(cudaStreamSynchronize(stream));                  // host vectors above go out of scope later

    // Upload the work lists of every class (chunk size `chunk_tiles`, or each
    // class's own when it is 0) and fill the class arguments.
    std::vector<BatchClass> bcs(nclass);
    auto upload = [&](int chunk_tiles, int mode) -> int {
        for (int c = 0; c < nclass; ++c) {
            ClassPlan &cp = classes[c];
            build_chunks(cp, V, chunk_tiles > 0 ? chunk_tiles : cp.chunk_tiles, first, nch);
            const size_t n = cp.chunk_ds.size();
            VBH_B_CK(cudaMemcpyAsync(cdev[c].ds_list, cp.ds.data(), sizeof(int) * cp.ds.size(), cudaMemcpyHostToDevice,
                                     stream));
            VBH_B_CK(cudaMemcpyAsync(cdev[c].chunk_ds, cp.chunk_ds.data(), sizeof(int) * n, cudaMemcpyHostToDevice,
                                     stream));
            VBH_B_CK(cudaMemcpyAsync(cdev[c].order, cp.order.data(), sizeof(int) * n, cudaMemcpyHostToDevice, stream));
            VBH_B_CK(cudaMemcpyAsync(cdev[c].lo, cp.lo.data(), sizeof(long long) * n, cudaMemcpyHostToDevice, stream));
            VBH_B_CK(cudaMemcpyAsync(cdev[c].hi, cp.hi.data(), sizeof(long long) * n, cudaMemcpyHostToDevice, stream));
            BatchClass &bc = bcs[c];
            bc.r = r_ptrs;
            bc.d = d_ptrs;
            bc.states = states;
            bc.chunk_ds = cdev[c].chunk_ds;
            bc.chunk_lo = cdev[c].lo;
            bc.chunk_hi = cdev[c].hi;
            bc.ds_V = ds_V;
            bc.order = cdev[c].order;
            bc.nchunks = int(n);
            bc.partials = cdev[c].partials;
            bc.nstat = cp.bi.nstat;
            bc.rows_per_chunk = cp.pi.rows_per_chunk;
            bc.stages = cp.stages;
            bc.next = counters + c;
            bc.ds_list = cdev[c].ds_list;
            bc.ds_first_chunk = ds_first;
            bc.ds_nchunks = ds_nch;
            bc.nds = int(cp.ds.size());
            bc.mode = mode;
            bc.ctl = ctl;
        }
        VBH_B_CK(cudaMemcpyAsync(ds_first, first.data(), sizeof(int) * B, cudaMemcpyHostToDevice, stream));
        VBH_B_CK(cudaMemcpyAsync(ds_nch, nch.data(), sizeof(int) * B, cudaMemcpyHostToDevice, stream));
        VBH_B_CK(cudaStreamSynchronize(stream));
        return VBH_OK;
    };
    auto pass_grid = [&](int c) {
        return std::max(1, std::min(classes[c].grid, bcs[c].nchunks));
    };
    auto launch_pass = [&](int c) -> int {
        void *args[] = {&bcs[c]};
        VBH_B_CK(cudaLaunchKernel(classes[c].pi.pass, dim3(pass_grid(c)), dim3(classes[c].pi.threads), args,
                                  classes[c].smem(), stream));
        return VBH_OK;
    };
    auto launch_update = [&](int c) -> int {
        void *args[] = {&bcs[c], &ctl};
        VBH_B_CK(cudaLaunchKernel(classes[c].bi.update, dim3(bcs[c].nds), dim3(256), args, classes[c].bi.update_smem,
                                  stream));
        return VBH_OK;
    };

    // ---------------- set-up of every state ----------------
    const int init = (o->init == VBH_INIT_GIVEN) ? 0 : 1;
    if ((rc = upload(kCandidates[1], MODE_INIT))) return rc;
    for (int c = 0; c < nclass; ++c) {
        int iv = init;
        void *args[] = {&bcs[c], &iv};
        VBH_B_CK(cudaLaunchKernel(classes[c].bi.setup, dim3(bcs[c].nds), dim3(32), args, 0, stream));
    }

    // ---------------- autotuner: per class, tiles per chunk x pipeline stages ----------------
    // Each candidate is timed on one data pass of its class alone (CUDA events);
    // the fastest is kept.  Small batches (< 2^26 observations) keep the defaults.
    long long total_obs = 0;
    for (int b = 0; b < B; ++b) total_obs += V[b];
    if (total_obs >= (1LL << 26)) {
        cudaEvent_t e0, e1;
        VBH_B_CK(cudaEventCreate(&e0));
        VBH_B_CK(cudaEventCreate(&e1));
        std::vector<float> best_ms(nclass, 1e30f);
        std::vector<int> best_chunk(nclass, kCandidates[1]), best_st(nclass, 0);
        for (int cand : kCandidates) {
            if ((rc = upload(cand, MODE_INIT))) break;
            for (int c = 0; c < nclass && !rc; ++c) {
                ClassPlan &cp = classes[c];
                for (int st : kStageCandidates) {
                    if (st > cp.max_stages) continue;
                    if (set_stages(cp, st) != VBH_OK) continue;
                    bcs[c].stages = st;
                    VBH_B_CK(cudaMemsetAsync(counters + c, 0, sizeof(unsigned int), stream));
                    VBH_B_CK(cudaEventRecord(e0, stream));
                    if ((rc = launch_pass(c))) break;
                    VBH_B_CK(cudaEventRecord(e1, stream));
                    VBH_B_CK(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    VBH_B_CK(cudaEventElapsedTime(&ms, e0, e1));
                    if (ms < best_ms[c]) {
                        best_ms[c] = ms;
                        best_chunk[c] = cand;
                        best_st[c] = st;
                    }
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc) return rc;
        for (int c = 0; c < nclass; ++c) {
            ClassPlan &cp = classes[c];
            cp.chunk_tiles = best_chunk[c];
            if (best_st[c] > 0) {
                if ((rc = set_stages(cp, best_st[c]))) return rc;
                cp.pass_ms = best_ms[c];
            } else if ((rc = set_stages(cp, std::min(kDefaultStages, cp.max_stages)))) {
                return rc;
            }
        }
        VBH_B_CK(cudaMemsetAsync(counters, 0, sizeof(unsigned int) * (SMAX + 1), stream));
    }
    hb.plan.clear();
    for (const ClassPlan &cp : classes)
        hb.plan.push_back({cp.S, cp.pi.tile, cp.chunk_tiles, cp.stages, cp.per_sm, cp.pass_ms});

    // ---------------- sweep 0 ----------------
    if ((rc = upload(0, init ? MODE_INIT : MODE_ELBO))) return rc;
    for (int c = 0; c < nclass; ++c)
        if ((rc = launch_pass(c))) return rc;
    for (int c = 0; c < nclass; ++c)
        if ((rc = launch_update(c))) return rc;
    VBH_B_CK(cudaMemsetAsync(counters, 0, sizeof(unsigned int) * (SMAX + 1), stream));
    VBH_B_CK(cudaMemsetAsync(&ctl->active, 0, sizeof(unsigned int), stream));

    // ---------------- sweeps 1 .. max_iter ----------------
    for (int c = 0; c < nclass; ++c) bcs[c].mode = MODE_ITER;
    if (o->max_iter > 0) {
        if (direct) {
            for (int t = 0; t < o->max_iter; ++t) {
                for (int c = 0; c < nclass; ++c)
                    if ((rc = launch_pass(c))) return rc;
                for (int c = 0; c < nclass; ++c)
                    if ((rc = launch_update(c))) return rc;
                batched_control_kernel<<<1, 32, 0, stream>>>(ctl, cudaGraphConditionalHandle{}, 0);
                VBH_B_CK(cudaGetLastError());
            }
        } else {
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ge = nullptr;
            VBH_B_CK(cudaGraphCreate(&g, 0));
            rc = VBH_OK;
            do {
                cudaGraphConditionalHandle cond;
                if (cudaGraphConditionalHandleCreate(&cond, g, 1u, cudaGraphCondAssignDefault) != cudaSuccess) {
                    rc = VBH_ECUDA;
                    break;
                }
                cudaGraphNodeParams cp{};
                cp.type = cudaGraphNodeTypeConditional;
                cp.conditional.handle = cond;
                cp.conditional.type = cudaGraphCondTypeWhile;
                cp.conditional.size = 1;
                cudaGraphNode_t wnode;
                if (cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &cp) != cudaSuccess) {
                    rc = VBH_ECUDA;
                    break;
                }
                cudaGraph_t body = cp.conditional.phGraph_out[0];
                std::vector<cudaGraphNode_t> ups;
                for (int c = 0; c < nclass && !rc; ++c) {
                    cudaGraphNodeParams kp{};
                    kp.type = cudaGraphNodeTypeKernel;
                    void *pargs[] = {&bcs[c]};
                    kp.kernel.func = const_cast<void *>(classes[c].pi.pass);
                    kp.kernel.gridDim = dim3(pass_grid(c));
                    kp.kernel.blockDim = dim3(classes[c].pi.threads);
                    kp.kernel.sharedMemBytes = unsigned(classes[c].smem());
                    kp.kernel.kernelParams = pargs;
                    cudaGraphNode_t pn, un;
                    if (cudaGraphAddNode(&pn, body, nullptr, nullptr, 0, &kp) != cudaSuccess) {
                        rc = VBH_ECUDA;
                        break;
                    }
                    cudaGraphNodeParams up{};
                    up.type = cudaGraphNodeTypeKernel;
                    void *uargs[] = {&bcs[c], &ctl};
                    up.kernel.func = const_cast<void *>(classes[c].bi.update);
                    up.kernel.gridDim = dim3(bcs[c].nds);
                    up.kernel.blockDim = dim3(256);
                    up.kernel.sharedMemBytes = unsigned(classes[c].bi.update_smem);
                    up.kernel.kernelParams = uargs;
                    if (cudaGraphAddNode(&un, body, &pn, nullptr, 1, &up) != cudaSuccess) {
                        rc = VBH_ECUDA;
                        break;
                    }
                    ups.push_back(un);
                }
                if (rc) break;
                cudaGraphNodeParams ck{};
                ck.type = cudaGraphNodeTypeKernel;
                int one = 1;
                void *cargs[] = {&ctl, &cond, &one};
                ck.kernel.func = reinterpret_cast<void *>(&batched_control_kernel);
                ck.kernel.gridDim = dim3(1);
                ck.kernel.blockDim = dim3(32);
                ck.kernel.kernelParams = cargs;
                cudaGraphNode_t cn;
                if (cudaGraphAddNode(&cn, body, ups.data(), nullptr, ups.size(), &ck) != cudaSuccess) {
                    rc = VBH_ECUDA;
                    break;
                }
                if (cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) {
                    ge = nullptr;
                    rc = VBH_ECUDA;
                    break;
                }
                if (cudaGraphLaunch(ge, stream) != cudaSuccess) rc = VBH_ECUDA;
            } while (0);
            if (rc) (void)cudaGetLastError();
            VBH_B_CK(cudaStreamSynchronize(stream));
            if (ge) cudaGraphExecDestroy(ge);
            cudaGraphDestroy(g);
            if (rc) return rc;
        }
    }

    // ---------------- results ----------------
    VBH_B_CK(cudaMemcpyAsync(hs, states, sizeof(DevState) * B, cudaMemcpyDeviceToHost, stream));
    BatchControl hc{};
    VBH_B_CK(cudaMemcpyAsync(&hc, ctl, sizeof(hc), cudaMemcpyDeviceToHost, stream));
    VBH_B_CK(cudaStreamSynchronize(stream));
    int status = hc.status;
    for (int b = 0; b < B; ++b) {
        const DevState &s = hs[b];
        vbh_result &res = out[b];
        std::memset(&res, 0, sizeof(res));
        const int M = s.M;
        res.S = s.S;
        res.iters = s.iter;
        res.converged = s.converged;
        res.status = s.status;
        res.elbo_const_dropped = s.const_dropped;
        double sum = 0.0;
        for (int j = 0; j < M; ++j) {
            res.kappa[j] = s.kappa[j];
            res.weights[j] = s.kappa[j];
            sum += s.kappa[j];
        }
        res.weights[M] = 1.0 - sum;
        std::memcpy(res.W_inv, s.Winv, sizeof(double) * size_t(M) * size_t(M));
        res.nu = s.nu;
        res.lambda = s.lam;
        res.a_rho = s.a_rho;
        res.b_rho = s.b_rho;
        res.rho_mean = s.a_rho / s.b_rho;
        res.rho_mode = (s.a_rho - 1.0) / s.b_rho;
        res.elbo = s.elbo;
        if (s.status && !status) status = s.status;
        if (o->elbo_trace)
            VBH_B_CK(cudaMemcpyAsync(o->elbo_trace + size_t(b) * ntrace, traces + size_t(b) * ntrace,
                                     sizeof(double) * size_t(s.iter + 1), cudaMemcpyDeviceToHost, stream));
    }
    if (o->elbo_trace) VBH_B_CK(cudaStreamSynchronize(stream));
    return status;
}

} // namespace vbh
