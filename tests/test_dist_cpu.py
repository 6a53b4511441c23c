"""The N > 1 paths on CPU ranks (gloo, world size 2; no GPU).

* `bench.whole_job`: the max-over-ranks time and the whole-job throughput
  that every multi-rank bench line reports.
* Partition and sum: the sufficient statistics of a sweep (Eq. 17, 24, 25)
  are sums over observations, so a contiguous split of the observations over
  ranks, one reduction of the per-rank FP64 sums in rank order and the
  closed-form updates run redundantly on every rank give the single-rank
  result (the design a sharded fit of one data set would follow; the build
  runs replicas only).  Checked with the oracle's sums.
* The reference arm under torchrun: rank 0 alone prints one line.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _w_whole_job(rank, world, port, out):
    _init(rank, world, port)
    import bench
    t_max, value = bench.whole_job([0.5, 0.8][rank], 1000.0, dist, world, torch.device("cpu"))
    with open(os.path.join(out, f"r{rank}.json"), "w") as f:
        json.dump({"t": t_max, "v": value}, f)
    dist.destroy_process_group()


def test_whole_job_takes_the_slowest_rank(tmp_path):
    mp.spawn(_w_whole_job, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for rank in range(2):
        with open(tmp_path / f"r{rank}.json") as f:
            j = json.load(f)
        assert j["t"] == 0.8
        assert j["v"] == pytest.approx(2 * 1000.0 / 0.8, rel=1e-15)


S_SHARD, V_SHARD = 4, 3001          # ragged: the ranks get 1500 and 1501 observations


def _state(O, synth):
    r, d, _ = synth.generate(V_SHARD, S_SHARD, seed=7)
    p = O.paper_prior(S_SHARD)
    mu, Sig = O.beta_init(p, V_SHARD)
    s = O.sums_from_beta(r, d, p, mu, Sig)
    g = O.KLambda_update(p, s, O.rho_update(p, s))
    return r, d, p, g


def _flat(s):
    return np.concatenate([[s["V"], s["sum_S"], s["sum_logdet"]], np.ravel(s["sum_mu"]), np.ravel(s["sum_Ebb"])])


def _unflat(v, M):
    return {"V": v[0], "sum_S": v[1], "sum_logdet": v[2], "sum_mu": v[3:3 + M],
            "sum_Ebb": v[3 + M:].reshape(M, M)}


def _shard_sums(O, r, d, p, g, rank, world):
    V = r.shape[0]
    lo, hi = rank * V // world, (rank + 1) * V // world
    mu, Sig = O.beta_update(r[lo:hi], d[lo:hi], p, g)
    return _flat(O.sums_from_beta(r[lo:hi], d[lo:hi], p, mu, Sig))


def _w_shard(rank, world, port, out):
    _init(rank, world, port)
    from oracle import oracle as O
    from paper_2401_10068_gb300 import synth
    r, d, p, g = _state(O, synth)
    mine = torch.from_numpy(_shard_sums(O, r, d, p, g, rank, world))
    parts = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine)
    total = parts[0].clone()
    for k in range(1, world):                       # rank order: the same bits on every rank
        total += parts[k]
    M = S_SHARD - 1
    s = _unflat(total.numpy(), M)
    g2 = O.KLambda_update(p, s, O.rho_update(p, s, g))
    np.savez(os.path.join(out, f"r{rank}.npz"), total=total.numpy(), kappa=g2["kappa"], Winv=g2["Winv"],
             b_rho=g2["b_rho"], elbo=O.elbo(p, s, g2)[0])
    dist.destroy_process_group()


def test_partition_and_sum_equals_one_rank(tmp_path):
    from oracle import oracle as O
    from paper_2401_10068_gb300 import synth
    mp.spawn(_w_shard, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    z = [np.load(tmp_path / f"r{k}.npz") for k in range(2)]
    # every rank holds the same reduced statistics and runs the same update
    for key in ("total", "kappa", "Winv", "b_rho", "elbo"):
        assert np.array_equal(z[0][key], z[1][key]), key
    # the rank-order sum is the sum of the two shard sums taken in one process
    r, d, p, g = _state(O, synth)
    seq = _shard_sums(O, r, d, p, g, 0, 2) + _shard_sums(O, r, d, p, g, 1, 2)
    assert np.array_equal(z[0]["total"], seq)
    # and equals the single-rank sums up to the order of the FP64 additions
    mu, Sig = O.beta_update(r, d, p, g)
    s1 = O.sums_from_beta(r, d, p, mu, Sig)
    full = _flat(s1)
    assert full[0] == z[0]["total"][0] == V_SHARD
    assert np.allclose(z[0]["total"], full, rtol=1e-12, atol=1e-12 * np.max(np.abs(full)))
    g1 = O.KLambda_update(p, s1, O.rho_update(p, s1, g))
    assert np.allclose(z[0]["kappa"], g1["kappa"], rtol=1e-12, atol=0)
    assert np.allclose(z[0]["Winv"], g1["Winv"], rtol=1e-12, atol=0)
    assert float(z[0]["elbo"]) == pytest.approx(O.elbo(p, s1, g1)[0], rel=1e-12)


def test_reference_arm_prints_once_under_torchrun():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    j = json.loads(lines[0])
    assert j["impl"] == "reference" and j["n_gpus"] == 2 and j["value"] > 0
    assert j["cpu_baseline"]["kind"] == "oracle"
    assert j["e2e"]["h2d_bytes_per_step"] == 0 and j["e2e"]["d2h_bytes_per_step"] == 0
