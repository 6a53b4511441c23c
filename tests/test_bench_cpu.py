"""The oracle legs of bench.py on CPU (no GPU).

* The all-cores oracle (contiguous chunks in spawn-started processes, the
  chunks' FP64 statistics summed in chunk order) follows the single-process
  oracle fit (Section 3.5 schedule) up to the order of the FP64 additions,
  and gives the same bits on every run.
* The reference arm runs it on every host core and prints one line, and
  falls back to one process when the pool cannot start."""
import argparse
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2401_10068_gb300 import synth  # noqa: E402


def test_all_cores_oracle_follows_the_single_process_fit():
    V, S, procs, warm, sweeps = 3001, 4, 3, 1, 2        # ragged: chunks of 1000, 1000 and 1001
    _, _, g = bench._oracle_sweeps_all_cores(V, S, sweeps, procs, warm=warm)
    W = bench.WORKLOAD
    r, d, _ = synth.generate(V, S, seed=W["seed"], alpha=W["alpha"], p_const=W["p_const"])
    ref = O.fit(r, d, O.paper_prior(S), tol=0.0, max_iter=warm + sweeps)
    assert ref["iters"] == warm + sweeps
    assert np.allclose(g["kappa"], ref["kappa"], rtol=1e-12, atol=0)
    assert np.allclose(g["Winv"], ref["Winv"], rtol=1e-12, atol=0)
    for k in ("a_rho", "b_rho", "nu", "lam"):
        assert g[k] == pytest.approx(ref[k], rel=1e-12), k
    # chunk-order sums: identical bits on a second run
    _, _, g2 = bench._oracle_sweeps_all_cores(V, S, sweeps, procs, warm=warm)
    assert np.array_equal(g["kappa"], g2["kappa"]) and np.array_equal(g["Winv"], g2["Winv"])
    assert g["b_rho"] == g2["b_rho"]


def test_cpu_model_is_reported():
    assert isinstance(bench._cpu_model(), str) and bench._cpu_model()


def test_reference_arm_on_every_core(capsys):
    args = argparse.Namespace(steps=1, warmup=3)
    assert bench.run_reference(args) == 0
    j = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert j["impl"] == "reference" and j["value"] > 0
    assert j["cpu_baseline"]["cores"] == (os.cpu_count() or 1) and j["config"]["sample_V"] == bench.REF_ALL_V
    assert j["e2e"]["h2d_bytes_per_step"] == 0 and j["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_arm_falls_back_to_one_process(monkeypatch, capsys):
    class NoPool:
        def __init__(self, *a, **k):
            raise RuntimeError("no pool")

    monkeypatch.setattr(bench, "OraclePool", NoPool)
    monkeypatch.setattr(bench, "REF_SAMPLE_V", 2048)
    args = argparse.Namespace(steps=1, warmup=3)
    assert bench.run_reference(args) == 0
    j = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert j["cpu_baseline"]["cores"] == 1 and j["config"]["sample_V"] == 2048
    assert "no pool" in j["cpu_baseline"]["sample"] and j["value"] > 0
