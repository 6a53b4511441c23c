"""Throughput of the fused CAVI sweep on one GB300 (or N independent replicas).

A step is one sweep of the whole hot path over the at-scale synthetic data set
(N = 4,194,304 cells x G = 96 genes = V = 402,653,184 observations, S = 8
subpopulations, 5 % constant profiles, K_true ~ Dirichlet(0.5), seed 2):
Q(beta) for every observation -> reduction of the sufficient statistics ->
Q(rho), Q(K, Lambda) -> ELBO and convergence test.  The metric is
observation x subpopulation CAVI updates per second (cell . gene . K updates/s
with V = N G and S = K), V * S * steps / time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the FP64 CPU oracle (the reference arm) on a
bounded prefix of the same data set on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = {"name": "at-scale single data set", "cells": 4_194_304, "genes": 96, "S": 8, "p_const": 0.05,
            "alpha": 0.5, "seed": 2}
V_FULL = WORKLOAD["cells"] * WORKLOAD["genes"]
METRIC = "cell.gene.K CAVI updates/s (observation x subpopulation updates per second, FP32 fused sweep)"
UNIT = "updates/s"
CPU_SAMPLE_V = 1 << 20          # oracle prefix for the single-core cpu_baseline leg
CPU_SAMPLE_SWEEPS = 5
CPU_ALL_V = 1 << 22             # oracle prefix for the all-cores cpu_baseline leg
REF_SAMPLE_V = 1 << 17          # oracle prefix per step of the reference arm (single process)
REF_ALL_V = 1 << 21             # oracle prefix per step of the reference arm (all host cores)


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def whole_job(seconds_rank, units_rank, dist, world, device):
    """Whole-job timing of N replicas: the maximum of the per-rank times over
    the ranks (all-reduce MAX; every rank receives it) and the units of all
    ranks divided by that time.  Returns (max seconds, units/s)."""
    import torch
    t = torch.tensor([float(seconds_rank)], device=device, dtype=torch.float64)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    t_max = float(t.item())
    return t_max, float(units_rank) * world / t_max


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


SWEEP_SOURCES = ("vbh_sweep.cuh", "vbh_internal.cuh", "vbh_dispatch.cuh", "vbh_sweep_s5_8.cu")


def _kernel_hash():
    """Hash of the sources that define sweep_kernel<8> (the timed kernel)."""
    h = hashlib.sha256()
    for name in SWEEP_SOURCES:
        with open(os.path.join(ROOT, "paper_2401_10068_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(bytes_alg):
    """DRAM bytes per launch of the sweep kernel from the committed ncu capture,
    or None if the kernel source changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "sweep_kernel_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        j = json.load(f)
    if j.get("kernel_hash") != _kernel_hash():
        return None
    return float(j["dram_read_bytes_per_obs"]) * V_FULL + float(j["dram_write_bytes_per_launch"])


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,utilization.gpu,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(device_index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [ln.strip().split(",") for ln in self.f.read().splitlines() if ln.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for row in rows:
            try:
                clk, cmax, util = float(row[0]), float(row[1]), float(row[2])
            except (ValueError, IndexError):
                continue
            mx.append(cmax)
            if util < 50:            # keep samples taken under load
                continue
            sm.append(clk)
            for nm, v in zip(names, row[3:7]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples_under_load": len(sm), "samples": len(rows)}


def _oracle_sweeps(V, S, sweeps, warm=1):
    """Time `sweeps` oracle sweeps (Q(beta), sums, Q(rho), Q(K,Lambda), ELBO) on
    the first V observations of the workload in this process; returns (wall
    seconds, CPU seconds of this process over the same sweeps)."""
    from oracle import oracle as O
    from paper_2401_10068_gb300 import synth
    r, d, _ = synth.generate(V, S, seed=WORKLOAD["seed"], alpha=WORKLOAD["alpha"], p_const=WORKLOAD["p_const"])
    p = O.paper_prior(S)
    g = O.fit(r, d, p, tol=0.0, max_iter=warm)
    c0, t0 = time.process_time(), time.perf_counter()
    for _ in range(sweeps):
        mu, Sig = O.beta_update(r, d, p, g)
        s = O.sums_from_beta(r, d, p, mu, Sig)
        g = O.KLambda_update(p, s, O.rho_update(p, s, g))
        O.elbo(p, s, g)
    return time.perf_counter() - t0, time.process_time() - c0


def _oracle_worker(conn, S, lo, hi):
    """One host core of the all-cores oracle leg.  It generates observations
    [lo, hi) of the workload (the generator is counter-based, so these are the
    prefix's own values) and answers each message with the oracle's Q(beta)
    and sufficient statistics of its chunk under the globals sent (sweep 0's
    initial Q(beta) for None), flattened, and the CPU seconds it spent."""
    from oracle import oracle as O
    from paper_2401_10068_gb300 import synth
    r, d, _ = synth.generate(hi - lo, S, seed=WORKLOAD["seed"], alpha=WORKLOAD["alpha"],
                             p_const=WORKLOAD["p_const"], start=lo)
    p = O.paper_prior(S)
    conn.send("ready")
    while True:
        msg = conn.recv()
        if msg == "stop":
            break
        c0 = time.process_time()
        g = msg["g"]
        if g is None:
            mu, Sig = O.beta_init(p, hi - lo)
        else:
            mu, Sig = O.beta_update(r, d, p, g)
        s = O.sums_from_beta(r, d, p, mu, Sig)
        flat = np.concatenate([[s["V"], s["sum_S"], s["sum_logdet"]], np.ravel(s["sum_mu"]), np.ravel(s["sum_Ebb"])])
        conn.send((flat, time.process_time() - c0))
    conn.close()


class OraclePool:
    """The oracle on `procs` host cores: one spawn-started process per
    contiguous chunk of the first V observations of the workload runs Q(beta)
    and the sums of its chunk; the parent adds the chunks' FP64 statistics in
    chunk order (the same bits whatever the timing) and runs Q(rho),
    Q(K, Lambda) and the ELBO."""

    def __init__(self, V, S, procs):
        import multiprocessing as mp
        from oracle import oracle as O
        O.build()                                       # built once here, loaded by every worker
        self.O, self.S, self.M = O, S, S - 1
        self.p = O.paper_prior(S)
        ctx = mp.get_context("spawn")
        self.conns, self.workers = [], []
        try:
            for k in range(procs):
                a, b = ctx.Pipe()
                w = ctx.Process(target=_oracle_worker, args=(b, S, k * V // procs, (k + 1) * V // procs),
                                daemon=True)
                w.start()
                b.close()
                self.conns.append(a)
                self.workers.append(w)
            for c in self.conns:
                if c.recv() != "ready":
                    raise RuntimeError("oracle worker failed to start")
        except BaseException:
            self.close()
            raise

    def sweep(self, g):
        """One sweep from globals g (None: sweep 0 from the initial Q(beta));
        returns (new globals, the workers' CPU seconds)."""
        O, M = self.O, self.M
        for c in self.conns:
            c.send({"g": g})
        total, cpu = None, 0.0
        for c in self.conns:                            # chunk order
            flat, t = c.recv()
            total = flat.copy() if total is None else total + flat
            cpu += t
        s = {"V": total[0], "sum_S": total[1], "sum_logdet": total[2], "sum_mu": total[3:3 + M],
             "sum_Ebb": total[3 + M:].reshape(M, M)}
        g2 = O.KLambda_update(self.p, s, O.rho_update(self.p, s, g))
        if g is not None:
            O.elbo(self.p, s, g2)
        return g2, cpu

    def close(self):
        for c in self.conns:
            try:
                c.send("stop")
            except (OSError, ValueError):
                pass
        for w in self.workers:
            w.join(timeout=30)
            if w.is_alive():
                w.terminate()
        self.conns, self.workers = [], []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False


def _oracle_sweeps_all_cores(V, S, sweeps, procs, warm=1):
    """`OraclePool` over the first V observations: sweep 0 and `warm` sweeps
    untimed, then `sweeps` timed.  Returns (wall seconds of the timed sweeps,
    the workers' CPU seconds in them, final globals)."""
    with OraclePool(V, S, procs) as pool:
        g, _ = pool.sweep(None)
        for _ in range(warm):
            g, _ = pool.sweep(g)
        cpu, t0 = 0.0, time.perf_counter()
        for _ in range(sweeps):
            g, c = pool.sweep(g)
            cpu += c
        wall = time.perf_counter() - t0
    return wall, cpu, g


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


def cpu_baseline(S):
    """The oracle timed on the host cores: single-threaded on a 2^20 prefix,
    and on all cores on a 2^22 prefix of the workload (the main figure)."""
    sec, csec = _oracle_sweeps(CPU_SAMPLE_V, S, CPU_SAMPLE_SWEEPS)
    single = {"value": CPU_SAMPLE_V * S * CPU_SAMPLE_SWEEPS / sec, "unit": UNIT, "cores": 1,
              "effective_cores": csec / sec,
              "sample": f"first {CPU_SAMPLE_V} observations of the workload, {CPU_SAMPLE_SWEEPS} sweeps after "
                        f"sweep 0, single-process FP64 oracle ({sec:.1f} s)"}
    host = {"nproc": os.cpu_count(), "cpu_model": _cpu_model()}
    procs = max(1, os.cpu_count() or 1)
    try:
        wall, cpu, _ = _oracle_sweeps_all_cores(CPU_ALL_V, S, CPU_SAMPLE_SWEEPS, procs)
    except Exception as e:                              # report the single-core leg alone
        return dict(single, kind="oracle", host=host, all_cores_error=f"{type(e).__name__}: {e}")
    return {"value": CPU_ALL_V * S * CPU_SAMPLE_SWEEPS / wall, "unit": UNIT, "cores": procs, "kind": "oracle",
            "effective_cores": cpu / wall,
            "sample": f"first {CPU_ALL_V} observations of the workload, {CPU_SAMPLE_SWEEPS} sweeps after sweep 0 "
                      f"and one warm-up sweep; the FP64 oracle in {procs} processes over contiguous chunks, the "
                      f"chunks' statistics summed in chunk order, the global update in the parent "
                      f"({wall:.1f} s, {cpu:.1f} CPU s)",
            "single_core": single, "host": host}


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands on the host cores, each
    step a sweep over a bounded prefix of the at-scale data set (2^21
    observations over every core with `OraclePool`; 2^17 in one process if
    the pool cannot start).  Under torchrun only rank 0 runs it."""
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    S = WORKLOAD["S"]
    procs = max(1, os.cpu_count() or 1)
    try:
        with OraclePool(REF_ALL_V, S, procs) as pool:
            g, _ = pool.sweep(None)
            for _ in range(args.warmup):
                g, _ = pool.sweep(g)
            cpu, t0 = 0.0, time.perf_counter()
            for _ in range(args.steps):
                g, c = pool.sweep(g)
                cpu += c
            el = time.perf_counter() - t0
        V, cores = REF_ALL_V, procs
        how = (f"the FP64 oracle in {procs} processes over contiguous chunks, the chunks' statistics summed in "
               f"chunk order, the global update in the parent ({cpu / el:.1f} effective cores)")
    except Exception as e:                              # one process
        V, cores, el = REF_SAMPLE_V, 1, _reference_one_process(args, S)
        how = f"the FP64 oracle in one process (all-cores pool unavailable: {type(e).__name__}: {e})"
    value = V * S * args.steps / el
    sample = f"first {V} of the {V_FULL} observations per step (same seeded recipe), S = {S}; {how}"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "N_cells": WORKLOAD["cells"], "G_genes": WORKLOAD["genes"],
                       "S": S, "V": V_FULL, "sample_V": V},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "host": {"nproc": os.cpu_count(), "cpu_model": _cpu_model()}},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _reference_one_process(args, S):
    """The reference arm's steps in one process on the first 2^17 observations;
    returns the seconds of the timed steps."""
    from oracle import oracle as O
    from paper_2401_10068_gb300 import synth
    V = REF_SAMPLE_V
    r, d, _ = synth.generate(V, S, seed=WORKLOAD["seed"], alpha=WORKLOAD["alpha"], p_const=WORKLOAD["p_const"])
    p = O.paper_prior(S)
    g = O.fit(r, d, p, tol=0.0, max_iter=0)

    def step(g):
        mu, Sig = O.beta_update(r, d, p, g)
        s = O.sums_from_beta(r, d, p, mu, Sig)
        g = O.KLambda_update(p, s, O.rho_update(p, s, g))
        O.elbo(p, s, g)
        return g

    for _ in range(args.warmup):
        g = step(g)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        g = step(g)
    return time.perf_counter() - t0


def run_ours(args):
    import torch
    rank, world, local = _dist()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2401_10068_gb300 import _build
    _build.build_all()
    from paper_2401_10068_gb300 import synth, vbh

    S, V = WORKLOAD["S"], V_FULL
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        r, d, _ = synth.generate_device(V, S, seed=WORKLOAD["seed"], alpha=WORKLOAD["alpha"],
                                        p_const=WORKLOAD["p_const"], device=dev)
    stream.synchronize()
    h = vbh.Handle(local, stream)
    total = args.warmup + args.steps
    h.fit_begin(r, d, S, None, tol=0.0, max_iter=total)
    clocks = Clocks(local)
    time.sleep(0.3)                                     # let the sampler start
    if args.warmup:
        h.fit_step(args.warmup)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    h.fit_step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    res = h.fit_result()
    assert res["iters"] == total, res["iters"]
    t_max, value = whole_job(ms * 1e-3, float(V) * S * args.steps, dist, world, dev)
    ms_max = t_max * 1e3
    ms_step = ms_max / args.steps

    # roofline of the dominant kernel (the fused sweep: one launch per step)
    bytes_alg = float(V) * (S + 1) * 4
    peak, peak_kind = _peaks()
    achieved = bytes_alg / (ms_step * 1e-3) / 1e9
    traffic = _traffic(bytes_alg)

    # end to end through the C ABI from pinned host buffers: one vbh_fit call
    # per timed repetition (H2D of r and d, sweep 0 + `steps` sweeps, result D2H)
    e2e_steps = args.steps
    e2e = None
    if not args.no_e2e:
        e2e = _e2e(h, r, d, V, S, e2e_steps, dev, dist, world)
    del r, d

    h.close()
    extra = None
    if rank == 0 and world == 1 and not args.no_extra:
        extra = other_workloads(dev, stream)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(S)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD["name"], "N_cells": WORKLOAD["cells"], "G_genes": WORKLOAD["genes"],
                           "S": S, "V": V, "p_const": WORKLOAD["p_const"], "seed": WORKLOAD["seed"],
                           "inputs_bytes": bytes_alg, "l2": "inputs larger than L2 (129 MB), no flush",
                           "parallelism": f"replicas x{world}",
                           "e2e": "one vbh_fit call from pinned host buffers per repetition: H2D of r and d once, "
                                  f"sweep 0 + {e2e_steps} sweeps, result D2H; bytes per step = per call / steps"},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": traffic,
                             "kernel": f"sweep_kernel<{S}>", "peak_kind": peak_kind,
                             "bytes_per_launch": bytes_alg},
                "cpu_baseline": cpu,
                "e2e": e2e,
                # the sweeps, the budget kernel of fit_step and, for an odd step count, the
                # second (idle) sweep launch of the graph's last loop iteration
                "gpu_launches": args.steps + 1 + (args.steps % 2),
                "clocks": clk,
                "other_workloads": extra}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


SINGLE = {"name": "single data set: N=2,000 cells x G=48 genes, S=3", "cells": 2000, "genes": 48, "S": 3,
          "alpha": 1.0, "seed": 1, "tol": 1e-8, "cap": 200, "cap_raised": 2000, "reps": 5}


def single_workload(h, dev, stream):
    """The single data set (N = 2,000 cells x G = 48 genes, S = 3): fits/s
    through vbh_fit at the workload's rule (rel dELBO < 1e-8 or 200 sweeps)
    and with the cap raised to 2,000 (converged data sets/s), and the device
    time per sweep of the resident and the streaming sweep loops."""
    import torch
    from paper_2401_10068_gb300 import synth, vbh
    V1 = SINGLE["cells"] * SINGLE["genes"]
    with torch.cuda.stream(stream):
        r1, d1, _ = synth.generate_device(V1, SINGLE["S"], seed=SINGLE["seed"], alpha=SINGLE["alpha"], device=dev)
    stream.synchronize()
    row = {"workload": SINGLE["name"], "V": V1, "tol": SINGLE["tol"]}
    for key, cap in (("rule_cap_200", SINGLE["cap"]), ("cap_2000", SINGLE["cap_raised"])):
        res = h.fit(r1, d1, SINGLE["S"], None, tol=SINGLE["tol"], max_iter=cap)          # warm (graph, buffers)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(SINGLE["reps"]):
            res = h.fit(r1, d1, SINGLE["S"], None, tol=SINGLE["tol"], max_iter=cap)
        sec = (time.perf_counter() - t0) / SINGLE["reps"]
        row[key] = {"fits_per_s": 1.0 / sec, "converged_datasets_per_s": (1.0 / sec) if res["converged"] else 0.0,
                    "converged": bool(res["converged"]), "sweeps": res["iters"], "us_per_sweep": 1e6 * sec /
                    (res["iters"] + 1), "elbo": res["elbo"]}
    # device time per sweep of the two sweep loops (200 sweeps in one vbh_fit_step, statistics as at tol > 0);
    # vbh_fit above runs the resident loop (VBH_LOOP_AUTO: the data set fits in shared memory)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, loop in (("resident_loop", vbh.LOOP_RESIDENT), ("stream_loop", vbh.LOOP_STREAM)):
        h.fit_begin(r1, d1, SINGLE["S"], None, tol=0.0, max_iter=205, stats=vbh.STATS_COMPENSATED, loop=loop)
        h.fit_step(5)
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        h.fit_step(200)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        row[name] = {"us_per_sweep": ev0.elapsed_time(ev1) * 1e3 / 200}
    return row


def run_single(args):
    """``--workload single``: the single-data-set figures alone (the small
    case for captures of the resident kernel)."""
    import torch
    from paper_2401_10068_gb300 import _build
    _build.build_all()
    from paper_2401_10068_gb300 import vbh
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    h = vbh.Handle(0, stream)
    clocks = Clocks(0)
    time.sleep(0.3)
    row = single_workload(h, dev, stream)
    h.close()
    line = {"metric": "converged datasets/s (single data set)",
            "value": row["cap_2000"]["converged_datasets_per_s"], "unit": "datasets/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic", "config": {"workload": SINGLE["name"]},
            "single": row, "clocks": clocks.stop()}
    print(json.dumps(line), flush=True)
    return 0


def other_workloads(dev, stream):
    """The other workloads' headline figures, measured after the timed region
    of the default step (each its own timing, CUDA events or wall clock around
    synchronous vbh_* calls with device-resident inputs):
      single data set: fits/s through vbh_fit at the workload's rule
        (rel dELBO < 1e-8 or 200 sweeps) and with the cap raised to 2,000 so
        that the fit converges (converged data sets/s);
      batched: the 4,096-data-set fit to rel dELBO < 1e-8 (cap 1,000),
        converged data sets/s and how many converged;
      precision: the S = 32 tensor-core sweep, ms per sweep of the BF16 and
        FP32 forms and the BF16 form's fraction of the HBM copy peak."""
    import torch
    from paper_2401_10068_gb300 import synth, vbh
    out = {}
    h = vbh.Handle(dev.index or 0, stream)
    clocks = Clocks(dev.index or 0)
    time.sleep(0.3)
    out["single"] = single_workload(h, dev, stream)
    # batched
    V, Sb = batch_specs(BATCH["datasets"])
    rs, ds = [], []
    with torch.cuda.stream(stream):
        for b in range(BATCH["datasets"]):
            r, d, _ = synth.generate_device(int(V[b]), int(Sb[b]), seed=BATCH["seed0"] + b, alpha=BATCH["alpha"],
                                            device=dev)
            rs.append(r)
            ds.append(d)
    stream.synchronize()
    Ss = [int(x) for x in Sb]
    h.fit_batched(rs[:64], ds[:64], Ss[:64], None, tol=0.0, max_iter=3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    res = h.fit_batched(rs, ds, Ss, None, tol=BATCH["tol"], max_iter=BATCH["cap"])
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    sec = ev0.elapsed_time(ev1) * 1e-3
    iters = np.array([x["iters"] for x in res])
    conv = np.array([x["converged"] for x in res])
    plan = h.batched_plan()
    for p in plan:                           # the class's data-pass bandwidth in the autotuner's timing
        cls = Sb == p["S"]
        p["pass_gbs"] = (float(np.sum(V[cls].astype(np.float64) * (p["S"] + 1) * 4)) / (p["pass_ms"] * 1e6)
                         if p["pass_ms"] > 0 else None)
    out["batched"] = {"workload": BATCH["name"], "V_total": int(V.sum()), "tol": BATCH["tol"], "cap": BATCH["cap"],
                      "seconds": sec, "converged": int(conv.sum()), "datasets": len(res),
                      "converged_datasets_per_s": float(conv.sum()) / sec, "datasets_per_s": len(res) / sec,
                      "sweeps_mean": float(iters.mean()), "sweeps_max": int(iters.max()),
                      "fit_average_gbs": float(np.sum(V.astype(np.float64) * (Sb + 1) * 4 * (iters + 1))) / sec / 1e9,
                      "pass_plan": plan}
    del rs, ds, res
    torch.cuda.empty_cache()
    # precision form
    S3, V3 = PREC["S"], PREC["cells"] * PREC["genes"]
    with torch.cuda.stream(stream):
        r3, d3, _ = synth.generate_device(V3, S3, seed=PREC["seed"], alpha=PREC["alpha"], p_const=PREC["p_const"],
                                          device=dev)
    stream.synchronize()
    n3 = 20
    peak, peak_kind = _peaks()
    row = {"workload": PREC["name"], "V": V3, "S": S3, "sweeps_timed": n3}
    for name, prec in (("bf16_form", vbh.BF16), ("fp32_form", vbh.FP32)):
        h.fit_begin(r3, d3, S3, None, tol=0.0, max_iter=n3 + 4, precision=prec, refine_iters=0)
        h.fit_step(4)
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        h.fit_step(n3)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        ms = ev0.elapsed_time(ev1) / n3
        gbs = V3 * 68.0 / (ms * 1e-3) / 1e9
        row[name] = {"ms_per_sweep": ms, "hbm_gbs": gbs, "frac": gbs / peak}
    row["peak"], row["peak_kind"] = peak, peak_kind
    out["precision"] = row
    del r3, d3
    h.close()
    out["clocks"] = clocks.stop()
    torch.cuda.empty_cache()
    return out


def _e2e(h, r, d, V, S, e2e_steps, dev, dist, world):
    import torch
    rh = torch.empty(V, dtype=torch.float32, pin_memory=True)
    dh = torch.empty((V, S), dtype=torch.float32, pin_memory=True)
    rh.copy_(r)
    dh.copy_(d)
    torch.cuda.synchronize(dev)
    h.fit(rh, dh, S, None, tol=0.0, max_iter=2)            # staging buffers + graph warm
    reps = 2
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(reps):
        out = h.fit(rh, dh, S, None, tol=0.0, max_iter=e2e_steps)
    t_e2e = (time.perf_counter() - t0) / reps
    assert out["iters"] == e2e_steps
    _, e2e_value = whole_job(t_e2e, float(V) * S * e2e_steps, dist, world, dev)
    h2d = V * 4 + V * S * 4
    d2h = ctypes_result_bytes()
    return {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d / e2e_steps,
            "d2h_bytes_per_step": d2h / e2e_steps}


def ctypes_result_bytes():
    """Device -> host bytes of one vbh_fit call: three read-backs of the fit state."""
    from paper_2401_10068_gb300 import vbh
    return 3 * vbh.state_bytes()


BATCH = {"name": "batched: 4,096 independent data sets", "datasets": 4096, "n_lo": 200, "n_hi": 50000,
         "genes": (48, 96), "S_lo": 2, "S_hi": 10, "alpha": 0.5, "seed0": 1000, "tol": 1e-8, "cap": 1000}


def batch_specs(B):
    """Data set shapes of the batched workload: N ~ log-uniform[200, 50000]
    cells, G uniform on {48, 96} genes (V = N G), S uniform on 2..10."""
    rng = np.random.default_rng(7)
    N = np.floor(np.exp(rng.uniform(np.log(BATCH["n_lo"]), np.log(BATCH["n_hi"]), size=B))).astype(np.int64)
    G = rng.choice(np.array(BATCH["genes"]), size=B)
    S = rng.integers(BATCH["S_lo"], BATCH["S_hi"] + 1, size=B)
    return N * G, S


def run_batched(args):
    """Converged data sets per second of the batched form, with the plain
    single-data-set form timed on a sample of the same data sets."""
    import torch
    from paper_2401_10068_gb300 import _build
    _build.build_all()
    from paper_2401_10068_gb300 import synth, vbh
    dev = torch.device("cuda", 0)
    B = args.datasets
    V, S = batch_specs(B)
    stream = torch.cuda.Stream(dev)
    rs, ds = [], []
    with torch.cuda.stream(stream):
        for b in range(B):
            r, d, _ = synth.generate_device(int(V[b]), int(S[b]), seed=BATCH["seed0"] + b, alpha=BATCH["alpha"],
                                            device=dev)
            rs.append(r)
            ds.append(d)
    stream.synchronize()
    h = vbh.Handle(0, stream)
    Ss = [int(x) for x in S]
    h.fit_batched(rs[:64], ds[:64], Ss[:64], None, tol=0.0, max_iter=args.warmup)       # warm-up
    clocks = Clocks(0)
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    stats = {"auto": vbh.STATS_AUTO, "plain": vbh.STATS_PLAIN, "compensated": vbh.STATS_COMPENSATED}[args.stats]
    res = h.fit_batched(rs, ds, Ss, None, tol=BATCH["tol"], max_iter=BATCH["cap"], stats=stats)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    sec = ev0.elapsed_time(ev1) * 1e-3
    clk = clocks.stop()
    plan = h.batched_plan()                  # per class: the autotuned pass shape and its pass time
    for p in plan:                           # the class's data-pass bandwidth in the autotuner's timing
        cls = S == p["S"]
        p["pass_gbs"] = (float(np.sum(V[cls].astype(np.float64) * (p["S"] + 1) * 4)) / (p["pass_ms"] * 1e6)
                         if p["pass_ms"] > 0 else None)
    pk, pk_kind = _peaks()
    iters = np.array([x["iters"] for x in res])
    conv = np.array([x["converged"] for x in res])
    upd = float(np.sum(V.astype(np.float64) * S * (iters + 1)))
    byts = float(np.sum(V.astype(np.float64) * (S + 1) * 4 * (iters + 1)))
    # the plain form on a sample, same tolerance and cap
    sample = list(range(0, B, max(1, B // args.plain_sample)))[:args.plain_sample]
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    plain = [h.fit(rs[b], ds[b], Ss[b], None, tol=BATCH["tol"], max_iter=BATCH["cap"]) for b in sample]
    torch.cuda.synchronize(dev)
    sec_plain = time.perf_counter() - t0
    gap = max(abs(res[b]["elbo"] - p["elbo"]) / abs(p["elbo"]) for b, p in zip(sample, plain))
    # the same data sets by the plain form for exactly the batched form's sweep counts
    same = [h.fit(rs[b], ds[b], Ss[b], None, tol=0.0, max_iter=res[b]["iters"]) for b in sample]
    gap_same = max(abs(res[b]["elbo"] - p["elbo"]) / abs(p["elbo"]) for b, p in zip(sample, same))
    stop_spread = [res[b]["iters"] - p["iters"] for b, p in zip(sample, plain)]
    h.close()
    line = {"metric": "converged datasets/s (batched form)", "value": float(conv.sum()) / sec, "unit": "datasets/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": BATCH["name"], "datasets": B, "V_total": int(V.sum()),
                       "bytes_resident": float(np.sum(V.astype(np.float64) * (S + 1) * 4)),
                       "tol": BATCH["tol"], "cap": BATCH["cap"], "stats": args.stats, "pass_plan": plan},
            "pass_bandwidth_frac": {str(p["S"]): (p["pass_gbs"] / pk if p["pass_gbs"] else None) for p in plan},
            "peak": {"hbm_gbs": pk, "kind": pk_kind},
            "seconds": sec, "converged": int(conv.sum()), "iters_mean": float(iters.mean()),
            "iters_max": int(iters.max()), "datasets_per_s_all": B / sec,
            "updates_per_s": upd / sec, "achieved_gbs_fit_average": byts / sec / 1e9,
            "plain": {"sample": len(sample), "seconds": sec_plain, "datasets_per_s": len(sample) / sec_plain,
                      "max_rel_elbo_gap_vs_batched": gap, "max_rel_elbo_gap_same_sweeps": gap_same,
                      "stop_sweep_difference_min_max": [int(min(stop_spread)), int(max(stop_spread))]},
            "speedup_vs_plain": (B / sec) / (len(sample) / sec_plain), "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


PREC = {"name": "precision form: N=1,048,576 cells x G=512 genes, S=32", "cells": 1 << 20, "genes": 512, "S": 32,
        "p_const": 0.05, "alpha": 0.5, "seed": 3, "refine": 10}


def run_precision(args):
    """The precision form on one data set of V = N G = 536,870,912 observations
    and S = 32: the tensor-core sweep with 16-bit operands (VBH_BF16) for all
    but the last `refine` sweeps, which run with FP32 operands; the same number
    of sweeps of the FP32 form alone for the speedup and the error of the
    BF16 schedule against it."""
    import torch
    from paper_2401_10068_gb300 import _build
    _build.build_all()
    from paper_2401_10068_gb300 import synth, vbh
    dev = torch.device("cuda", 0)
    S, V = PREC["S"], PREC["cells"] * PREC["genes"]
    refine = PREC["refine"]
    if args.steps <= refine:
        raise SystemExit(f"--steps must exceed the {refine} refinement sweeps")
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        r, d, _ = synth.generate_device(V, S, seed=PREC["seed"], alpha=PREC["alpha"], p_const=PREC["p_const"],
                                        device=dev)
    stream.synchronize()
    h = vbh.Handle(0, stream)
    total = args.warmup + args.steps
    clocks = Clocks(0)
    time.sleep(0.3)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

    h.fit_begin(r, d, S, None, tol=0.0, max_iter=total, precision=vbh.BF16, refine_iters=refine)
    h.fit_step(args.warmup)
    torch.cuda.synchronize(dev)
    ev[0].record(stream)
    h.fit_step(args.steps - refine)
    ev[1].record(stream)
    h.fit_step(refine)
    ev[2].record(stream)
    torch.cuda.synchronize(dev)
    res_bf16 = h.fit_result()
    assert res_bf16["iters"] == total, res_bf16["iters"]
    ms_bf16 = ev[0].elapsed_time(ev[1]) / (args.steps - refine)
    ms_ref = ev[1].elapsed_time(ev[2]) / refine
    ms_sched = ev[0].elapsed_time(ev[2]) / args.steps

    h.fit_begin(r, d, S, None, tol=0.0, max_iter=total, precision=vbh.FP32)
    h.fit_step(args.warmup)
    torch.cuda.synchronize(dev)
    ev[0].record(stream)
    h.fit_step(args.steps)
    ev[3].record(stream)
    torch.cuda.synchronize(dev)
    res_fp32 = h.fit_result()
    ms_fp32 = ev[0].elapsed_time(ev[3]) / args.steps
    clk = clocks.stop()
    h.close()

    def relerr(a, b):
        a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    err = {k: relerr(res_bf16[k], res_fp32[k]) for k in ("kappa", "Winv", "b_rho")}
    err["elbo"] = abs(res_bf16["elbo"] - res_fp32["elbo"]) / abs(res_fp32["elbo"])
    peak, peak_kind = _peaks()
    bytes_obs = 68.0                     # BF16 profile row (32 x 2 B) + r (4 B)
    # MMA work per tile of 128 observations: U = d (128 x 32) . B1 (32 x N1) and
    # G' = A2 (128 x 128) . d (128 x 32)
    flops_tile = lambda n1: 2 * 128 * n1 * 32 + 2 * 128 * 32 * 128
    tiles = (V + 127) // 128
    upd = float(V) * S
    line = {"metric": "cell.gene.K CAVI updates/s (precision form, S = 32)", "unit": UNIT,
            "value": upd / (ms_sched * 1e-3), "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_sched, "higher_is_better": True, "dtype": "bf16 operands, f32 accumulation",
            "data": "synthetic",
            "config": {"workload": PREC["name"], "V": V, "S": S, "p_const": PREC["p_const"], "seed": PREC["seed"],
                       "schedule": f"{args.steps - refine} BF16-form sweeps + {refine} FP32-form sweeps",
                       "l2": "inputs larger than L2 (129 MB), no flush"},
            "bf16_form": {"ms_per_sweep": ms_bf16, "updates_per_s": upd / (ms_bf16 * 1e-3),
                          "hbm_gbs": V * bytes_obs / (ms_bf16 * 1e-3) / 1e9,
                          "tensor_tflops": tiles * flops_tile(80) / (ms_bf16 * 1e-3) / 1e12},
            "fp32_form": {"ms_per_sweep": ms_fp32, "updates_per_s": upd / (ms_fp32 * 1e-3),
                          "hbm_gbs": V * bytes_obs / (ms_fp32 * 1e-3) / 1e9,
                          "tensor_tflops": tiles * flops_tile(112) / (ms_fp32 * 1e-3) / 1e12,
                          "ms_per_sweep_in_schedule": ms_ref},
            "speedup_schedule_vs_fp32_form": ms_fp32 / ms_sched,
            "rel_error_bf16_schedule_vs_fp32_form": err,
            "roofline": {"bound": "hbm", "achieved": V * bytes_obs / (ms_bf16 * 1e-3) / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": V * bytes_obs / (ms_bf16 * 1e-3) / 1e9 / peak,
                         "kernel": "tc_sweep_kernel<2>", "peak_kind": peak_kind, "bytes_per_obs": bytes_obs},
            "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_grouped(args):
    """The exact profile-grouped form on the at-scale data set (binary profiles,
    S = 8): the histogram pass, then sweeps over the 2^S profiles; against the
    per-observation sweep, per sweep and for a whole fit to rel dELBO < 1e-8
    (cap 1000 sweeps), with the gap between the two converged ELBOs."""
    import torch
    from paper_2401_10068_gb300 import _build
    _build.build_all()
    from paper_2401_10068_gb300 import synth, vbh
    dev = torch.device("cuda", 0)
    S, V = WORKLOAD["S"], V_FULL
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        r, d, _ = synth.generate_device(V, S, seed=WORKLOAD["seed"], alpha=WORKLOAD["alpha"],
                                        p_const=WORKLOAD["p_const"], device=dev)
    stream.synchronize()
    h = vbh.Handle(0, stream)
    clocks = Clocks(0)
    time.sleep(0.3)
    total = args.warmup + args.steps
    h.fit(r, d, S, None, tol=0.0, max_iter=2, grouped=True)                  # buffers, graph
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    h.fit_begin(r, d, S, None, tol=0.0, max_iter=total, grouped=True)       # histogram + sweep 0
    t_begin = time.perf_counter() - t0
    h.fit_step(args.warmup)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    h.fit_step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms_grouped = ev0.elapsed_time(ev1) / args.steps
    tol, cap = 1e-8, 1000
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    g = h.fit(r, d, S, None, tol=tol, max_iter=cap, grouped=True)
    t_g = time.perf_counter() - t0
    t0 = time.perf_counter()
    p = h.fit(r, d, S, None, tol=tol, max_iter=cap)
    t_p = time.perf_counter() - t0
    same = h.fit(r, d, S, None, tol=0.0, max_iter=g["iters"])
    clk = clocks.stop()
    h.close()
    line = {"metric": "converged fits/s, at-scale data set (profile-grouped vs per-observation sweep)",
            "value": 1.0 / t_g, "unit": "fits/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f64 groups",
            "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "V": V, "S": S, "profiles": 1 << S, "tol": tol, "cap": cap},
            "grouped": {"fit_begin_s_incl_histogram": t_begin, "ms_per_sweep": ms_grouped,
                        "fit_s": t_g, "iters": g["iters"], "converged": bool(g["converged"]), "elbo": g["elbo"]},
            "per_observation": {"fit_s": t_p, "iters": p["iters"], "converged": bool(p["converged"]),
                                "elbo": p["elbo"]},
            "speedup_fit": t_p / t_g,
            "rel_elbo_gap_converged": abs(g["elbo"] - p["elbo"]) / abs(p["elbo"]),
            "rel_elbo_gap_same_sweeps": abs(g["elbo"] - same["elbo"]) / abs(same["elbo"]),
            "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


WARM = {"name": "learned warm start: held-out batch of the batched workload's shape", "train_sets": 8192,
        "train_seed": 7, "train_n_lo": 200, "train_n_hi": 20000, "eval_sets": 1024, "eval_seed": 900, "n_lo": 200,
        "n_hi": 50000, "tol": 1e-8, "cap": 4000, "epochs": 150, "batch": 64, "lr": 2e-3, "n_cap": 16384}


def run_warmstart(args):
    """The learned warm start (set encoder on the tensor cores): trained on
    generator data sets against their CAVI fixed points (or loaded with
    --ws-load), then a held-out batch shaped like the batched workload is fitted
    from the paper's start and from the encoder's start to rel dELBO < 1e-8:
    converged data sets per second of both, sweeps per S, the ELBO gap between
    the two converged fits, the error of each predicted factor against the
    converged fixed point next to the error of the per-S training mean (what a
    predictor with no information about the data set would give), and the
    encoder's tensor-core throughput."""
    import torch
    from paper_2401_10068_gb300 import _build
    _build.build_all()
    from paper_2401_10068_gb300 import vbh, warmstart
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    h = vbh.Handle(0, stream)
    W = WARM
    train = None
    if args.ws_load:
        ws = warmstart.load(args.ws_load, stream=stream)
    else:
        ws = vbh.WarmStart(seed=W["train_seed"], stream=stream)
        info = warmstart.fit_and_train(h, ws, W["train_sets"], W["train_seed"], W["train_n_lo"], W["train_n_hi"],
                                       W["tol"], W["cap"], W["epochs"], W["batch"], W["lr"], W["n_cap"])
        train = {k: v for k, v in info.items() if k not in ("T", "W", "losses")}
        train["loss_first_last"] = [info["losses"][0], info["losses"][-1]]
        if args.ws_save:
            warmstart.save(ws, args.ws_save)
    rs, ds, Ss = warmstart.make_sets(W["eval_sets"], W["eval_seed"], W["n_lo"], W["n_hi"])
    clocks = Clocks(0)
    time.sleep(0.3)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    torch.cuda.synchronize(dev)
    ev[0].record(stream)
    preds = warmstart.predict(ws, rs, ds, Ss)
    ev[1].record(stream)
    cold = h.fit_batched(rs, ds, Ss, None, tol=W["tol"], max_iter=W["cap"])
    ev[2].record(stream)
    ev[3].record(stream)
    warm = h.fit_batched(rs, ds, Ss, None, tol=W["tol"], max_iter=W["cap"], init_states=preds)
    ev[4].record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    t_pred = ev[0].elapsed_time(ev[1]) * 1e-3
    t_cold = ev[1].elapsed_time(ev[2]) * 1e-3
    t_warm = ev[3].elapsed_time(ev[4]) * 1e-3
    Sa = np.asarray(Ss)
    ic = np.array([x["iters"] for x in cold])
    iw = np.array([x["iters"] for x in warm])
    cc = np.array([x["converged"] for x in cold])
    cw = np.array([x["converged"] for x in warm])
    both = cc & cw
    gaps = np.array([abs(w["elbo"] - c["elbo"]) / abs(c["elbo"]) for c, w in zip(cold, warm)])[both]
    # predicted factors against the converged fixed points, and the per-S mean of the training targets
    mean = ws.mean
    err = {"kappa": [], "Sigma0": [], "E_rho": []}
    err_mean = {"kappa": [], "Sigma0": [], "E_rho": []}
    for p, c, S in zip(preds, cold, Ss):
        if not c["converged"]:
            continue
        M = S - 1
        sc = np.asarray(c["Winv"]) / c["nu"]
        rc = c["a_rho"] / c["b_rho"]
        err["kappa"].append(np.linalg.norm(p["kappa"] - c["kappa"]) / np.linalg.norm(c["kappa"]))
        err["Sigma0"].append(np.linalg.norm(np.asarray(p["Winv"]) / p["nu"] - sc) / np.linalg.norm(sc))
        err["E_rho"].append(abs(p["a_rho"] / p["b_rho"] - rc) / rc)
        m = mean[S]
        Lm = np.zeros((M, M))
        for j in range(M):
            for k in range(j + 1):
                Lm[j, k] = np.exp(m[10 + j * (j + 1) // 2 + k]) if j == k else m[10 + j * (j + 1) // 2 + k]
        err_mean["kappa"].append(np.linalg.norm(m[:M] - c["kappa"]) / np.linalg.norm(c["kappa"]))
        err_mean["Sigma0"].append(np.linalg.norm(Lm @ Lm.T - sc) / np.linalg.norm(sc))
        err_mean["E_rho"].append(abs(np.exp(m[9]) - rc) / rc)
    rows = sum(int(r.shape[0]) for r in rs)
    flops = rows * 2.0 * (64 * 256 + 256 * 256)
    per_s = {int(S): {"sets": int((Sa == S).sum()), "cold_sweeps_median": float(np.median(ic[Sa == S])),
                      "warm_sweeps_median": float(np.median(iw[Sa == S])), "cold_converged": int(cc[Sa == S].sum()),
                      "warm_converged": int(cw[Sa == S].sum())} for S in range(2, 11) if (Sa == S).any()}
    line = {"metric": "converged datasets/s, learned vs paper's start (held-out batch)", "unit": "datasets/s",
            "value": float(cw.sum()) / (t_warm + t_pred), "n_gpus": 1, "higher_is_better": True,
            "dtype": "bf16 encoder (f32 accumulation), f32 sweeps", "data": "synthetic",
            "config": {"workload": W["name"], "eval_sets": W["eval_sets"], "V_total": rows, "tol": W["tol"],
                       "cap": W["cap"], "train": None if train is None else {k: W[k] for k in (
                           "train_sets", "train_n_lo", "train_n_hi", "epochs", "batch", "lr", "n_cap")}},
            "cold": {"seconds": t_cold, "converged": int(cc.sum()), "converged_datasets_per_s": float(cc.sum()) / t_cold,
                     "sweeps_mean": float(ic.mean())},
            "warm": {"seconds_fit": t_warm, "seconds_predict": t_pred, "converged": int(cw.sum()),
                     "converged_datasets_per_s": float(cw.sum()) / (t_warm + t_pred), "sweeps_mean": float(iw.mean())},
            "speedup_converged_datasets_per_s": (float(cw.sum()) / (t_warm + t_pred)) / max(float(cc.sum()) / t_cold,
                                                                                          1e-30),
            "elbo_gap_both_converged": {"median": float(np.median(gaps)) if gaps.size else None,
                                        "max": float(gaps.max()) if gaps.size else None, "sets": int(both.sum())},
            "factor_error_median": {k: float(np.median(v)) for k, v in err.items()},
            "factor_error_median_per_S_mean": {k: float(np.median(v)) for k, v in err_mean.items()},
            "per_S": per_s,
            "encoder": {"pooled_observations": rows, "seconds": t_pred, "tensor_tflops": flops / t_pred / 1e12},
            "train": train, "clocks": clk}
    h.close()
    ws.close()
    print(json.dumps(line), flush=True)
    return 0


PER_S = {"V": 1 << 27, "S": (2, 3, 4, 6, 8, 10, 11), "seed": 9, "alpha": 0.5, "warm": 4, "sweeps": 20}


def run_per_s(args):
    """Bandwidth of the FP32 sweep kernel across S (one data set of 2^27
    observations per S, the same recipe without constant profiles), in its
    plain and its compensated form: per S and form, 4 untimed sweeps, then 20
    sweeps timed with CUDA events on the handle's stream; algorithmic bytes
    4 (S + 1) per observation."""
    import torch
    from paper_2401_10068_gb300 import _build
    _build.build_all()
    from paper_2401_10068_gb300 import synth, vbh
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(dev)
    h = vbh.Handle(0, stream)
    peak, peak_kind = _peaks()
    V, n = PER_S["V"], PER_S["sweeps"]
    clocks = Clocks(0)
    time.sleep(0.3)
    rows = []
    for S in PER_S["S"]:
        with torch.cuda.stream(stream):
            r, d, _ = synth.generate_device(V, S, seed=PER_S["seed"], alpha=PER_S["alpha"], device=dev)
        stream.synchronize()
        row = {"S": S}
        for form, stats in (("plain", vbh.STATS_PLAIN), ("compensated", vbh.STATS_COMPENSATED)):
            h.fit_begin(r, d, S, None, tol=0.0, max_iter=PER_S["warm"] + n, stats=stats)
            h.fit_step(PER_S["warm"])
            torch.cuda.synchronize(dev)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            h.fit_step(n)
            ev1.record(stream)
            torch.cuda.synchronize(dev)
            ms = ev0.elapsed_time(ev1) / n
            gbs = V * 4.0 * (S + 1) / (ms * 1e-3) / 1e9
            if form == "plain":
                row.update({"ms_per_sweep": ms, "achieved_gbs": gbs, "frac": gbs / peak})
            else:
                row["compensated"] = {"ms_per_sweep": ms, "achieved_gbs": gbs, "frac": gbs / peak}
        rows.append(row)
        del r, d
    clk = clocks.stop()
    h.close()
    line = {"metric": "FP32 sweep kernel bandwidth across S", "unit": "GB/s", "n_gpus": 1, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "one data set per S", "V": V, "S": list(PER_S["S"]), "seed": PER_S["seed"],
                       "warmup": PER_S["warm"], "sweeps": n, "l2": "inputs larger than L2 (129 MB), no flush"},
            "peak": peak, "peak_kind": peak_kind, "rows": rows, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cells", type=int, default=WORKLOAD["cells"],
                    help="N cells (x 96 genes); smaller values give the small case used for ncu captures")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other workloads' figures (single data set, batched, precision)")
    ap.add_argument("--ws-load", default=None, help="warmstart workload: load the encoder instead of training it")
    ap.add_argument("--ws-save", default=None, help="warmstart workload: save the trained encoder")
    ap.add_argument("--workload", default="at-scale",
                    choices=["at-scale", "single", "batched", "precision", "grouped", "per-s", "warmstart"],
                    help="batched: the 4,096-data-set form; precision: the S = 32 tensor-core form; grouped: "
                         "the profile-grouped form; per-s: the FP32 sweep's bandwidth for S = 2..11; warmstart: "
                         "the learned warm start (separate measurements, not the default step)")
    ap.add_argument("--datasets", type=int, default=BATCH["datasets"])
    ap.add_argument("--plain-sample", type=int, default=32)
    ap.add_argument("--stats", default="auto", choices=["auto", "plain", "compensated"],
                    help="batched workload: the statistics of the data passes (auto: compensated, as tol > 0)")
    args = ap.parse_args()
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "single":
        return run_single(args)
    if args.workload == "grouped":
        return run_grouped(args)
    if args.workload == "per-s":
        return run_per_s(args)
    if args.workload == "warmstart":
        return run_warmstart(args)
    if args.workload == "precision":
        if args.cells != WORKLOAD["cells"]:
            PREC["cells"] = args.cells
            PREC["name"] = "precision recipe, reduced N (profiling case)"
        return run_precision(args)
    global V_FULL
    if args.cells != WORKLOAD["cells"]:
        WORKLOAD["cells"] = args.cells
        WORKLOAD["name"] = "at-scale recipe, reduced N (profiling case)"
        V_FULL = WORKLOAD["cells"] * WORKLOAD["genes"]
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
