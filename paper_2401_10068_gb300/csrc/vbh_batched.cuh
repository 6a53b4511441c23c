// vbh_batched.cuh -- CAVI sweeps of many independent data sets at once.
//
// Every data set b (V_b observations, S_b subpopulations) has its own device
// state (DevState) and follows exactly the schedule of a single fit.  One
// batched sweep is, for each class of data sets with the same S:
//   data pass  (batched_pass_kernel<S>): persistent blocks take chunks --
//              contiguous observation ranges of one data set -- from an
//              atomic work queue (largest chunks first), stream them through
//              the same shared-memory ring and per-observation algebra as the
//              single-data-set kernel, and write one FP64 partial per chunk;
//   update     (batched_update_kernel<M>): one block per data set adds its
//              chunks' partials in chunk order and runs the FP64 global
//              update, ELBO and convergence test of that data set;
// then batched_control_kernel counts the data sets still running and sets
// the while condition of the CUDA graph that repeats the sweep.  Data sets
// that have converged (or reached their sweep limit) drop out: their chunks
// are skipped and their states are left as they are.
#pragma once

#include "vbh_sweep.cuh"

namespace vbh {

// Per-class work description (device memory, built by the host).
struct BatchClass {
    const float *const *r;          // [B] device pointers (all data sets)
    const float *const *d;          // [B]
    DevState *states;               // [B]
    const int *chunk_ds;            // [nchunks] data set of each chunk
    const long long *chunk_lo;      // [nchunks] first observation
    const long long *chunk_hi;      // [nchunks] one past the last observation
    const long long *ds_V;          // [B] observations per data set
    const int *order;               // [nchunks] scheduling order (chunk ids)
    int nchunks;
    double *partials;               // [nchunks][nstat]
    int nstat;                      // columns of a chunk partial: NSTAT, or NSTAT + 1 for the compensated form
    unsigned int *next;             // work-queue counter of this class
    const int *ds_list;             // [nds] data sets of this class
    const int *ds_first_chunk;      // [B] first chunk id of each data set (within its class)
    const int *ds_nchunks;          // [B]
    int nds;
    int mode;
    struct BatchControl *ctl;
};

struct BatchControl {
    int status;                     // ST_ETIMEOUT if a bounded wait of a data pass ran out
    unsigned int active;            // data sets still running after this sweep's updates
    unsigned int sweep;             // batched sweeps done
    unsigned int max_sweeps;
    unsigned int nclasses;
    unsigned int *class_next[SMAX + 1];
};

__device__ __forceinline__ bool ds_running(const DevState *st)
{
    return st->status == ST_OK && !st->converged && st->iter < st->target && st->iter < st->max_iter;
}

// Stage metadata written by the producer thread when it fills a stage.
struct StageMeta {
    int chunk;                      // -1: end of work
    int ds;
    long long obs0;                 // first observation of the unit
    int flags;                      // UNIT_TAIL | UNIT_LAST
    int pad;
};
enum : int { UNIT_TAIL = 1, UNIT_LAST = 2 };

template <int S>
struct BatchCfg {
    using C = SweepCfg<S>;
    static constexpr int THREADS = 256;
    // observations per thread per tile: 4 (1,024 per tile) except at S = 8,
    // where two blocks per SM need the 768-observation ring
    static constexpr int OPT = (S == 8) ? 3 : 4;
    static constexpr int T = THREADS * OPT;
    static constexpr int STAGES = 3;
    static constexpr uint32_t R_BYTES = T * 4u;
    static constexpr uint32_t D_BYTES = T * S * 4u;
    static constexpr uint32_t STAGE_BYTES = R_BYTES + D_BYTES;
    static constexpr size_t RING_BYTES = size_t(STAGES) * STAGE_BYTES;
    static constexpr size_t SMEM_BYTES = RING_BYTES + 64;
    // compensated form: the ring, the table of profile terms, the split pass globals
    static constexpr size_t OFF_TAB = RING_BYTES, OFF_SPLIT = OFF_TAB + C::TAB_BYTES;
    static constexpr size_t SMEM_BYTES_C = OFF_SPLIT + C::SPLIT_BYTES + 64;
};

// Producer state (thread 0 of a block): the chunk being issued and the next unit.
struct Cursor {
    int chunk;                      // current chunk (-1: none)
    int ds;
    long long next_obs;             // first observation of the next unit to issue
    long long hi;                   // end of the chunk
    long long full_hi;              // end of the chunk's full tiles
    int tail_done;
    int done;                       // no more work
};

template <int S>
__device__ __forceinline__ bool cursor_advance(Cursor &cu, const BatchClass &bc, int mode)
{
    using B = BatchCfg<S>;
    while (true) {
        if (cu.chunk >= 0 && (cu.next_obs < cu.full_hi || !cu.tail_done)) return true;
        const unsigned int q = atomicAdd(bc.next, 1u);
        if (q >= unsigned(bc.nchunks)) {
            cu.done = 1;
            return false;
        }
        const int c = bc.order[q];
        const int ds = bc.chunk_ds[c];
        if (mode == MODE_ITER && !ds_running(bc.states + ds)) continue;      // retired data set
        cu.chunk = c;
        cu.ds = ds;
        cu.next_obs = bc.chunk_lo[c];
        cu.hi = bc.chunk_hi[c];
        // full tiles are those whose observations all lie in the chunk; chunk
        // boundaries are multiples of the tile except at the data set's end.
        // A chunk without observations still yields one (empty) tail unit, so
        // that its partial is written.
        const long long ntiles = (cu.hi - cu.next_obs) / B::T;
        cu.full_hi = cu.next_obs + ntiles * B::T;
        cu.tail_done = (cu.full_hi == cu.hi && cu.hi > cu.next_obs) ? 1 : 0;
        return true;
    }
}

// Fill stage s with the next unit (a full tile by bulk copy, or the ragged
// tail of a chunk, read later with plain loads), or with the end mark.
template <int S>
__device__ __forceinline__ void issue_unit(Cursor &cu, const BatchClass &bc, int mode, unsigned char *stage,
                                           uint64_t *bar, StageMeta *meta)
{
    using B = BatchCfg<S>;
    if (cu.done || !cursor_advance<S>(cu, bc, mode)) {
        meta->chunk = -1;
        mbar_arrive_expect_tx(bar, 0u);
        return;
    }
    meta->chunk = cu.chunk;
    meta->ds = cu.ds;
    meta->obs0 = cu.next_obs;
    if (cu.next_obs < cu.full_hi) {
        const long long o = cu.next_obs;
        cu.next_obs += B::T;
        const bool last = (cu.next_obs == cu.full_hi) && cu.tail_done;
        meta->flags = last ? UNIT_LAST : 0;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar, B::STAGE_BYTES);
        bulk_load(stage, bc.r[cu.ds] + o, B::R_BYTES, bar);
        bulk_load(stage + B::R_BYTES, bc.d[cu.ds] + o * S, B::D_BYTES, bar);
    } else {
        meta->flags = UNIT_TAIL | UNIT_LAST;
        cu.tail_done = 1;
        cu.next_obs = cu.hi;
        mbar_arrive_expect_tx(bar, 0u);
    }
}

// One block barrier per unit: every thread waits for the stage, consumes it,
// and meets the others at the end of the unit, after which thread 0 refills
// the stage.  A chunk's FP64 partial is staged in one of two reduction buffers
// before that barrier and summed after it, so the next chunk's partial (into
// the other buffer) cannot overwrite it while it is read.
template <int S, bool COMP>
__global__ void __launch_bounds__(BatchCfg<S>::THREADS, COMP ? SweepCfg<S>::MINB_BC : SweepCfg<S>::MINB)
    batched_pass_kernel(BatchClass bc)
{
    using C = SweepCfg<S>;
    using B = BatchCfg<S>;
    constexpr int M = C::M, NG = C::NG, NSTAT = C::NSTAT;
    constexpr int NS = COMP ? C::NSTATC : C::NSTAT;        // columns of a chunk partial
    constexpr int NGRP = COMP ? C::NGRPC : C::NGRP;
    constexpr int THREADS = B::THREADS, T = B::T, STAGES = B::STAGES;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (COMP ? B::SMEM_BYTES_C - 64 : B::RING_BYTES));
    float4 *tab = reinterpret_cast<float4 *>(smem + B::OFF_TAB);     // compensated form only
    float *split = reinterpret_cast<float *>(smem + B::OFF_SPLIT);
    __shared__ StageMeta meta[STAGES];
    __shared__ double s_red[2][THREADS / 32][NGRP * 32];
    __shared__ int s_bad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int mode = bc.mode;

    if (tid == 0) {
        s_bad = 0;
        for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    Cursor cu{-1, 0, 0, 0, 0, 1, 0};
    if (tid == 0)
        for (int s = 0; s < STAGES; ++s)
            issue_unit<S>(cu, bc, mode, smem + size_t(s) * B::STAGE_BYTES, &full[s], &meta[s]);

    float acc[NSTAT];
    double acc64[NGRP];
    float prod = 1.0f, pl = 0.0f, uh = 0.0f, ul = 0.0f;
    int ex = 0;
#pragma unroll
    for (int i = 0; i < NSTAT; ++i) acc[i] = 0.0f;
#pragma unroll
    for (int g = 0; g < NGRP; ++g) acc64[g] = 0.0;
    // plain form: L~ (L) and kappa~ (kap) in registers; compensated form: the
    // split globals of the current data set and its table of profile terms in
    // shared memory, switched by the whole block between units
    float L[COMP ? 1 : C::NGA], kap[COMP ? 1 : C::MA], erho = 0.0f;
    L[0] = 0.0f;
    kap[0] = 0.0f;
    int cur_ds = -1;
    // (compensated form) make data set ds current: split globals, E[rho], table.
    // Called by every thread with the same ds, between units.
    auto switch_to = [&](int ds) {
        const DevState *st = bc.states + ds;
        for (int i = tid; i < C::SPLIT_FLOATS; i += THREADS) {
            float v;
            if (i < NG) v = st->sw.Sh[i];
            else if (i < 2 * NG) v = st->sw.Sl[i - NG];
            else if (i < 2 * NG + M) v = st->sw.kh[i - 2 * NG];
            else v = st->sw.kl[i - 2 * NG - M];
            split[i] = v;
        }
        erho = (mode == MODE_INIT) ? 0.0f : st->sw.erho;
        __syncthreads();
        build_profile_table<S>(tab, split, erho, tid, THREADS);
        __syncthreads();
        cur_ds = ds;
    };
    if constexpr (COMP) {
        __syncthreads();                                    // the first unit's metadata
        if (meta[0].chunk >= 0) switch_to(meta[0].ds);
    }
    int ftile = 0;
    int rbuf = 0;                                           // reduction buffer of the next chunk partial

    long long kbreak = 0;
    for (long long k = 0;; ++k) {
        const int s = int(k % STAGES);
        const bool ok = mbar_wait_bounded(&full[s], uint32_t((k / STAGES) & 1), 2000000000ull);
        StageMeta m;
        m.chunk = -1;
        m.flags = 0;
        if (ok) m = meta[s];                                // the same for every thread once the stage is full
        const bool work = ok && m.chunk >= 0;
        if (work) {
            if constexpr (!COMP) {
                if (m.ds != cur_ds) {                       // a new data set: its FP32 globals (cached reads)
                    const DevState *st = bc.states + m.ds;
#pragma unroll
                    for (int i = 0; i < NG; ++i) L[i] = st->sw.L[i];
#pragma unroll
                    for (int i = 0; i < M; ++i) kap[i] = st->sw.kappa[i];
                    erho = (mode == MODE_INIT) ? 0.0f : st->sw.erho;
                    cur_ds = m.ds;
                }
            }
            if (!(m.flags & UNIT_TAIL)) {
                const float *rt = reinterpret_cast<const float *>(smem + size_t(s) * B::STAGE_BYTES);
                const float *dt = rt + T;
#pragma unroll
                for (int u = 0; u < B::OPT; ++u) {
                    const int j = tid + u * THREADS;
                    float x[S];
                    load_row<S>(dt, j, x);
                    if constexpr (COMP) {
                        observe_comp<S>(x, rt[j], tab, split, erho, acc, prod, pl, uh, ul);
                        peel_exponent2(prod, pl, ex);
                    } else {
                        observe<S>(x, rt[j], L, kap, erho, acc, prod);
                        peel_exponent(prod, ex);
                    }
                }
                if (++ftile == 16) {
                    if constexpr (COMP)
                        flush_warp_comp<S>(acc, acc64, prod, pl, ex, uh, ul, lane);
                    else
                        flush_warp<S>(acc, acc64, prod, ex, lane);
                    ftile = 0;
                }
            } else {
                const float *rg = bc.r[m.ds];
                const float *dg = bc.d[m.ds];
                const long long hi = bc.chunk_hi[m.chunk];
                for (long long i = m.obs0 + tid; i < hi; i += THREADS) {
                    float x[S];
#pragma unroll
                    for (int q = 0; q < S; ++q) x[q] = __ldg(dg + i * S + q);
                    if constexpr (COMP) {
                        observe_comp<S>(x, __ldg(rg + i), tab, split, erho, acc, prod, pl, uh, ul);
                        peel_exponent2(prod, pl, ex);
                    } else {
                        observe<S>(x, __ldg(rg + i), L, kap, erho, acc, prod);
                        peel_exponent(prod, ex);
                    }
                }
            }
            if (m.flags & UNIT_LAST) {                      // chunk done: stage its FP64 partial
                if constexpr (COMP)
                    flush_warp_comp<S>(acc, acc64, prod, pl, ex, uh, ul, lane);
                else
                    flush_warp<S>(acc, acc64, prod, ex, lane);
                ftile = 0;
#pragma unroll
                for (int g = 0; g < NGRP; ++g) {
                    s_red[rbuf][warp][g * 32 + lane] = acc64[g];
                    acc64[g] = 0.0;
                }
            }
        }
        if (__syncthreads_or(!ok)) {                        // stage s is free again; s_red[rbuf] is complete
            if (tid == 0) s_bad = 1;
            kbreak = k;
            break;
        }
        if (!work) break;                                   // the end mark (every thread read it)
        if (m.flags & UNIT_LAST) {
            for (int j = tid; j < NS; j += THREADS) {
                double t = 0.0;
#pragma unroll
                for (int w = 0; w < THREADS / 32; ++w) t += s_red[rbuf][w][j];
                bc.partials[size_t(m.chunk) * NS + j] = t;
            }
            rbuf ^= 1;
        }
        if constexpr (COMP) {
            // the next unit's metadata was written before this unit's barrier (it was issued
            // STAGES - 1 units ago, or in the prologue); a new data set switches here, block-wide
            const StageMeta nx = meta[(k + 1) % STAGES];
            if (nx.chunk >= 0 && nx.ds != cur_ds) switch_to(nx.ds);
        }
        if (tid == 0) issue_unit<S>(cu, bc, mode, smem + size_t(s) * B::STAGE_BYTES, &full[s], &meta[s]);
    }
    if (s_bad && tid == 0) {
        // a wait ran out: record it, then let the copies this block issued and
        // did not consume land before the block exits (bounded)
        atomicCAS(&bc.ctl->status, ST_OK, ST_ETIMEOUT);
        for (long long kk = kbreak; kk < kbreak + STAGES; ++kk)
            (void)mbar_wait_bounded(&full[kk % STAGES], uint32_t((kk / STAGES) & 1), 100000000ull);
    }
}

template <int M>
__global__ void __launch_bounds__(256) batched_update_kernel(BatchClass bc, BatchControl *ctl)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int b = bc.ds_list[blockIdx.x];
    DevState *st = bc.states + b;
    const int mode = bc.mode;
    if (mode == MODE_ITER && !ds_running(st)) return;      // retired: chunks were skipped too
    SweepArgs a{};
    a.mode = mode;
    a.use_cond = 0;
    global_update<M>(st, bc.partials + size_t(bc.ds_first_chunk[b]) * bc.nstat, bc.ds_nchunks[b], a,
                     reinterpret_cast<double *>(smem));
    __syncthreads();                                       // the control fields were written by another warp
    if (threadIdx.x == 0 && ds_running(st)) atomicAdd(&ctl->active, 1u);
}

// Set-up of every data set of a class (one warp per data set).
template <int M>
__global__ void batched_setup_kernel(BatchClass bc, int init)
{
    constexpr int MM = M > 0 ? M * M : 1;
    __shared__ double A[MM], Lc[MM];
    if (threadIdx.x >= 32) return;
    setup_state<M>(bc.states + bc.ds_list[blockIdx.x], init, threadIdx.x, A, Lc);
}

} // namespace vbh
