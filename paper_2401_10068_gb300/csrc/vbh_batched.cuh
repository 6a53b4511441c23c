// vbh_batched.cuh -- CAVI sweeps of many independent data sets at once.
//
// Every data set b (V_b observations, S_b subpopulations) has its own device
// state (DevState) and follows exactly the schedule of a single fit.  One
// batched sweep is, for each class of data sets with the same S:
//   data pass  (batched_pass_kernel<S>): persistent blocks take chunks --
//              contiguous observation ranges of one data set -- from an
//              atomic work queue (largest chunks first), stream them through
//              a shared-memory ring filled by a producer warp, with the same
//              per-observation algebra as the single-data-set kernel, and
//              write one FP64 partial row per chunk and compute warp;
//   update     (batched_update_kernel<M>): one block per data set adds its
//              chunks' partial rows in order and runs the FP64 global
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
    double *partials;               // [nchunks][rows_per_chunk][nstat]
    int nstat;                      // columns of a partial row: NSTAT, or NSTAT + 1 for the compensated form
    int rows_per_chunk;             // partial rows per chunk (the pass's compute warps)
    int stages;                     // pipeline stages of the pass (2 .. BatchCfg<S, COMP>::MAX_STAGES)
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
// Stage metadata written by the producer when it fills a stage.
struct StageMeta {
    int chunk;                      // -1: end of work
    int ds;
    long long obs0;                 // first observation of the unit
    int flags;                      // UNIT_TAIL | UNIT_LAST
    int pad;
};
enum : int { UNIT_TAIL = 1, UNIT_LAST = 2 };

// Shape of the batched pass.  Warps 0 .. CW-1 compute, warp CW is the
// producer: its lane 0 owns the work-queue cursor and refills a stage once
// the compute warps have released it (per-stage empty mbarriers), so the
// compute warps never meet at a block barrier.  Seven compute warps where
// two or more blocks share an SM (registers for 128 per thread), eleven where
// one block holds it (the larger S: up to 168 registers per thread), so that
// an SM keeps at least 14 compute warps or 11 wider ones.  The number of
// stages is chosen at run time (the autotuner, up to MAX_STAGES); shared
// memory holds the barriers and metadata, then (compensated form) the table
// of profile terms and two copies of the split pass globals, then the ring.
template <int S, bool COMP>
struct BatchCfg {
    using C = SweepCfg<S>;
    static constexpr int MINB = COMP ? C::MINB_BC : C::MINB;       // resident blocks per SM the registers allow
    static constexpr int CW = (MINB >= 2) ? 7 : 11;                // compute warps
    static constexpr int THREADS = 32 * (CW + 1);
    static constexpr int CT = 32 * CW;                             // compute threads
    static constexpr int PRODUCER_WARP = CW;
    static constexpr int OPT = 4;                                  // observations per compute thread per tile
    static constexpr int T = CT * OPT;                             // observations per tile (896 or 1,408)
    static constexpr int MAX_STAGES = 8;
    static constexpr uint32_t R_BYTES = T * 4u;
    static constexpr uint32_t D_BYTES = T * S * 4u;
    static constexpr uint32_t STAGE_BYTES = R_BYTES + D_BYTES;
    static_assert(R_BYTES % 16 == 0 && D_BYTES % 16 == 0, "bulk copies need 16-byte sizes and offsets");
    // mbarriers: full[MAX_STAGES], empty[MAX_STAGES], the compute warps' rendezvous
    static constexpr size_t OFF_BAR = 0;
    static constexpr size_t OFF_META = 256;
    static_assert(size_t(2 * MAX_STAGES + 1) * 8 <= OFF_META, "barriers overlap the metadata");
    static_assert(OFF_META + MAX_STAGES * sizeof(StageMeta) <= 512, "metadata overlaps the ring");
    static constexpr size_t FIXED = 512;                           // plain form: the ring starts here
    static constexpr size_t TAB_AL = (C::TAB_BYTES + 127) / 128 * 128;
    static constexpr size_t SPLIT_AL = (C::SPLIT_BYTES + 127) / 128 * 128;
    static constexpr size_t OFF_TAB = FIXED, OFF_SPLIT = OFF_TAB + TAB_AL;
    static constexpr size_t FIXED_C = OFF_SPLIT + 2 * SPLIT_AL;    // compensated form: the ring starts here
    static constexpr size_t smem(bool comp, int stages) { return (comp ? FIXED_C : FIXED) + size_t(stages) * STAGE_BYTES; }
};

// Producer state (lane 0 of the producer warp): the chunk being issued and the next unit.
struct Cursor {
    int chunk;                      // current chunk (-1: none)
    int ds;
    long long next_obs;             // first observation of the next unit to issue
    long long hi;                   // end of the chunk
    long long full_hi;              // end of the chunk's full tiles
    int tail_done;
    int done;                       // no more work
    const float *rp, *dp;           // the data set's inputs
};

template <int S, bool COMP>
__device__ __forceinline__ bool cursor_advance(Cursor &cu, const BatchClass &bc, int mode)
{
    using B = BatchCfg<S, COMP>;
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
        cu.rp = bc.r[ds];
        cu.dp = bc.d[ds];
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

// Fill a stage with the next unit (a full tile by bulk copy, or the ragged
// tail of a chunk, read later with plain loads), or with the end mark.
// Returns false after writing the end mark.
template <int S, bool COMP>
__device__ __forceinline__ bool issue_unit(Cursor &cu, const BatchClass &bc, int mode, unsigned char *stage,
                                           uint64_t *bar, StageMeta *meta)
{
    using B = BatchCfg<S, COMP>;
    if (cu.done || !cursor_advance<S, COMP>(cu, bc, mode)) {
        meta->chunk = -1;
        mbar_arrive_expect_tx(bar, 0u);
        return false;
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
        bulk_load(stage, cu.rp + o, B::R_BYTES, bar);
        bulk_load(stage + B::R_BYTES, cu.dp + o * S, B::D_BYTES, bar);
    } else {
        meta->flags = UNIT_TAIL | UNIT_LAST;
        cu.tail_done = 1;
        cu.next_obs = cu.hi;
        mbar_arrive_expect_tx(bar, 0u);
    }
    return true;
}

constexpr uint64_t BATCH_WAIT_NS = 2000000000ull;    // bound of every wait of the pass

// Record a timed-out wait of the pass (any thread).
__device__ __forceinline__ void batch_abort(const BatchClass &bc, volatile int *s_abort)
{
    *s_abort = 1;
    atomicCAS(&bc.ctl->status, ST_OK, ST_ETIMEOUT);
}

// The data pass of one class.  Units flow through a ring of bc.stages stages:
// the producer fills stage k % stages with unit k after the compute warps
// released unit k - stages (empty[s]); every compute warp takes every unit
// (thread t its observations t + CT u), releases the stage, and at the last
// unit of a chunk writes its own FP64 row of the chunk partial
// (partials[chunk][warp][NS]; the update adds the rows in order).  The
// compensated form switches the table of profile terms when the data set
// changes: the compute warps write the new split globals into the spare copy,
// meet (every warp is then done with the old table), build the table and meet
// again, both times at a bounded mbarrier rendezvous.
template <int S, bool COMP>
__global__ void __launch_bounds__(BatchCfg<S, COMP>::THREADS, BatchCfg<S, COMP>::MINB)
    batched_pass_kernel(BatchClass bc)
{
    using C = SweepCfg<S>;
    using B = BatchCfg<S, COMP>;
    constexpr int M = C::M, NG = C::NG, NSTAT = C::NSTAT;
    constexpr int NS = COMP ? C::NSTATC : C::NSTAT;        // columns of a partial row
    constexpr int NGRP = COMP ? C::NGRPC : C::NGRP;
    constexpr int CW = B::CW, CT = B::CT, T = B::T;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + B::OFF_BAR);
    uint64_t *empty = full + B::MAX_STAGES;
    uint64_t *rdv = empty + B::MAX_STAGES;
    StageMeta *meta = reinterpret_cast<StageMeta *>(smem + B::OFF_META);
    unsigned char *ring = smem + (COMP ? B::FIXED_C : B::FIXED);
    __shared__ int s_abort;
    volatile int *abort_flag = &s_abort;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int mode = bc.mode;
    const int stages = bc.stages;

    if (tid == 0) {
        s_abort = 0;
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], CW);
        }
        mbar_init(rdv, CW);
        fence_mbar_init();
    }
    __syncthreads();                                        // the only block barrier

    if (warp == B::PRODUCER_WARP) {
        if (lane != 0) return;
        Cursor cu{-1, 0, 0, 0, 0, 1, 0, nullptr, nullptr};
        long long k = 0;
        int s = 0, round = 0;                               // unit k = round * stages + s
        bool bad = false;
        for (;; ++k) {
            if (round > 0 && !mbar_wait_bounded(&empty[s], uint32_t((round - 1) & 1), BATCH_WAIT_NS)) {
                bad = true;
                break;
            }
            if (*abort_flag) {
                bad = true;
                break;
            }
            if (!issue_unit<S, COMP>(cu, bc, mode, ring + size_t(s) * B::STAGE_BYTES, &full[s], &meta[s])) break;
            if (++s == stages) {
                s = 0;
                ++round;
            }
        }
        if (bad) {
            // a wait ran out: record it, then let the copies of the last units
            // issued on each stage land before the block exits (bounded)
            batch_abort(bc, abort_flag);
            for (long long kk = (k > stages ? k - stages : 0); kk < k; ++kk)
                (void)mbar_wait_bounded(&full[kk % stages], uint32_t((kk / stages) & 1), 100000000ull);
        }
        return;
    }

    // ---------------- compute warps ----------------
    // One iteration of the outer loop per chunk: the statistics start at zero
    // (each chunk's last unit flushed them into this warp's partial row), so
    // a data-set switch at the chunk's first unit holds no accumulator live.
    // plain form: L~ (L) and kappa~ (kap) in registers; compensated form: the
    // split globals of the current data set (copy cur & 1) and its table of
    // profile terms in shared memory
    float L[COMP ? 1 : C::NGA], kap[COMP ? 1 : C::MA], erho = 0.0f;
    L[0] = 0.0f;
    kap[0] = 0.0f;
    float4 *tab = reinterpret_cast<float4 *>(smem + B::OFF_TAB);
    float *split = reinterpret_cast<float *>(smem + B::OFF_SPLIT);
    int cur_ds = -1, nswitch = 0;
    uint32_t rv = 0;                                        // rendezvous phases passed
    // every compute warp arrives; true once all seven have (bounded)
    auto rendezvous = [&]() -> bool {
        __syncwarp();
        if (lane == 0) mbar_arrive(rdv);
        const bool ok = mbar_wait_bounded(rdv, rv & 1u, BATCH_WAIT_NS);
        ++rv;
        return __all_sync(0xffffffffu, ok);
    };
    // the next unit is in stage cs, whose fill has parity cph
    int cs = 0;
    uint32_t cph = 0;
    // wait for the next unit (its stage and metadata); false on a timeout (recorded)
    auto take = [&](StageMeta &m) -> bool {
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[cs], cph, BATCH_WAIT_NS))) {
            if (lane == 0) batch_abort(bc, abort_flag);
            return false;
        }
        m = meta[cs];                                       // the same for every thread once the stage is full
        return true;
    };

    while (true) {
        float acc[NSTAT];
        double acc64[NGRP];
        float prod = 1.0f, pl = 0.0f, uh = 0.0f, ul = 0.0f;
        int ex = 0, ftile = 0;
#pragma unroll
        for (int i = 0; i < NSTAT; ++i) acc[i] = 0.0f;
#pragma unroll
        for (int g = 0; g < NGRP; ++g) acc64[g] = 0.0;
        StageMeta m;
        if (!take(m) || m.chunk < 0) break;                 // a timeout, or the end mark
        if (m.ds != cur_ds) {
            const DevState *st = bc.states + m.ds;
            erho = (mode == MODE_INIT) ? 0.0f : st->sw.erho;
            if constexpr (COMP) {
                // the spare copy of the split globals is free: every warp passed the
                // previous switch's first rendezvous, so none reads it any more
                float *sp = split + (nswitch & 1) * (B::SPLIT_AL / 4);
                for (int i = tid; i < C::SPLIT_FLOATS; i += CT) {
                    float v;
                    if (i < NG) v = st->sw.Sh[i];
                    else if (i < 2 * NG) v = st->sw.Sl[i - NG];
                    else if (i < 2 * NG + M) v = st->sw.kh[i - 2 * NG];
                    else v = st->sw.kl[i - 2 * NG - M];
                    sp[i] = v;
                }
                if (!rendezvous()) {                        // done with the old table; new split written
                    if (lane == 0) batch_abort(bc, abort_flag);
                    break;
                }
                build_profile_table<S>(tab, sp, erho, tid, CT);
                if (!rendezvous()) {                        // the table is complete
                    if (lane == 0) batch_abort(bc, abort_flag);
                    break;
                }
                ++nswitch;
            } else {
#pragma unroll
                for (int i = 0; i < NG; ++i) L[i] = st->sw.L[i];
#pragma unroll
                for (int i = 0; i < M; ++i) kap[i] = st->sw.kappa[i];
            }
            cur_ds = m.ds;
        }
        const float *sp = split + ((nswitch + 1) & 1) * (B::SPLIT_AL / 4);   // copy of the current data set
        bool ok = true;
        while (true) {                                      // the units of chunk m.chunk
            if (!(m.flags & UNIT_TAIL)) {
                const float *rt = reinterpret_cast<const float *>(ring + size_t(cs) * B::STAGE_BYTES);
                const float *dt = rt + T;
#pragma unroll
                for (int u = 0; u < B::OPT; ++u) {
                    const int j = tid + u * CT;
                    float x[S];
                    load_row<S>(dt, j, x);
                    if constexpr (COMP) {
                        observe_comp<S>(x, rt[j], tab, sp, erho, acc, prod, pl, uh, ul);
                        if (u & 1) peel_exponent2(prod, pl, ex);
                    } else {
                        observe<S>(x, rt[j], L, kap, erho, acc, prod);
                        if (u & 1) peel_exponent(prod, ex);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[cs]);         // this warp's reads of stage cs are done
            if (++cs == stages) {
                cs = 0;
                cph ^= 1u;
            }
            if (m.flags & UNIT_TAIL) {
                const float *rg = bc.r[m.ds];
                const float *dg = bc.d[m.ds];
                const long long hi = bc.chunk_hi[m.chunk];
                for (long long i = m.obs0 + tid; i < hi; i += CT) {
                    float x[S];
#pragma unroll
                    for (int q = 0; q < S; ++q) x[q] = __ldg(dg + i * S + q);
                    if constexpr (COMP) {
                        observe_comp<S>(x, __ldg(rg + i), tab, sp, erho, acc, prod, pl, uh, ul);
                        peel_exponent2(prod, pl, ex);
                    } else {
                        observe<S>(x, __ldg(rg + i), L, kap, erho, acc, prod);
                        peel_exponent(prod, ex);
                    }
                }
            }
            if (m.flags & UNIT_LAST) break;
            if (++ftile == 16) {
                if constexpr (COMP)
                    flush_warp_comp<S>(acc, acc64, prod, pl, ex, uh, ul, lane);
                else
                    flush_warp<S>(acc, acc64, prod, ex, lane);
                ftile = 0;
            }
            if (!take(m)) {                                 // the chunk's next unit
                ok = false;
                break;
            }
        }
        if (!ok) break;
        // chunk done: this warp's row of its partial
        if constexpr (COMP)
            flush_warp_comp<S>(acc, acc64, prod, pl, ex, uh, ul, lane);
        else
            flush_warp<S>(acc, acc64, prod, ex, lane);
        double *row = bc.partials + (size_t(m.chunk) * CW + warp) * NS;
#pragma unroll
        for (int g = 0; g < NGRP; ++g)
            if (g * 32 + lane < NS) row[g * 32 + lane] = acc64[g];
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
    // the data set's chunk partials: rows_per_chunk rows per chunk (one per compute warp of the pass)
    global_update<M>(st, bc.partials + size_t(bc.ds_first_chunk[b]) * bc.rows_per_chunk * bc.nstat,
                     bc.ds_nchunks[b] * bc.rows_per_chunk, a, reinterpret_cast<double *>(smem));
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
