"""The cpu_baseline leg of bench.py on CPU (no GPU): the oracle run over
contiguous chunks in spawn-started processes, with the chunks' FP64
statistics summed in chunk order, follows the single-process oracle fit
(Section 3.5 schedule) up to the order of the FP64 additions, and gives the
same bits on every run."""
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
