"""Parity at the full at-scale size, in the launch configuration bench.py times.

N = 4,194,304 cells x G = 96 genes = 402,653,184 observations, S = 8, 5 %
constant profiles, 100 sweeps: far beyond what the per-observation oracle can
run, so the oracle runs its profile-grouped form (exact for binary profiles:
every sum it needs is a polynomial of degree <= 2 in y_i within a profile,
pinned against the per-observation form by test_oracle_pins).  Its input, the
per-profile (n, sum y, sum y^2), is computed here on the CPU from the raw data
copied back from the device, in FP64."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2401_10068_gb300 import _build, synth, vbh

pytestmark = pytest.mark.gpu

CELLS, GENES, S, SWEEPS = 4_194_304, 96, 8, 100


def _histogram(r, d, S, chunk=1 << 24):
    V = r.shape[0]
    P = 1 << S
    n, sy, syy = np.zeros(P), np.zeros(P), np.zeros(P)
    for s0 in range(0, V, chunk):
        rc = r[s0:s0 + chunk].cpu().numpy().astype(np.float64)
        dc = d[s0:s0 + chunk].cpu().numpy()
        assert np.all((dc == 0) | (dc == 1))
        code = np.packbits(dc.astype(np.uint8), axis=1, bitorder="little")[:, 0].astype(np.int64)
        y = rc - dc[:, S - 1].astype(np.float64)
        n += np.bincount(code, minlength=P)
        sy += np.bincount(code, weights=y, minlength=P)
        syy += np.bincount(code, weights=y * y, minlength=P)
    keep = n > 0
    codes = np.nonzero(keep)[0]
    dprof = ((codes[:, None] >> np.arange(S)[None, :]) & 1).astype(np.float64)
    return {"dprof": dprof, "n": n[keep], "sy": sy[keep], "syy": syy[keep]}


def test_fullsize_parity_against_grouped_oracle():
    _build.build_all()
    V = CELLS * GENES
    stream = torch.cuda.current_stream()
    r, d, truth = synth.generate_device(V, S, seed=2, alpha=0.5, p_const=0.05)
    prior = O.paper_prior(S)
    with vbh.Handle(0, stream) as h:
        got = h.fit(r, d, S, prior, tol=0.0, max_iter=SWEEPS, trace=True)
    assert got["iters"] == SWEEPS
    groups = _histogram(r, d, S)
    assert groups["n"].sum() == V
    ref = O.fit_grouped(groups, prior, tol=0.0, max_iter=SWEEPS)
    rel = lambda a, b: np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))
    assert rel(got["kappa"], ref["kappa"]) < 1e-4
    assert rel(got["Winv"], ref["Winv"]) < 1e-4
    assert rel(got["b_rho"], ref["b_rho"]) < 1e-4
    assert abs(got["elbo"] - ref["elbo"]) <= 1e-6 * abs(ref["elbo"])
    for t, (x, y) in enumerate(zip(got["trace"], ref["trace"])):
        assert abs(x - y) <= 1e-6 * max(abs(y), V), t
    # coordinate ascent: the ELBO does not decrease (up to the FP32 rounding floor)
    assert np.all(np.diff(got["trace"]) >= -1e-8 * V)
    assert abs(got["weights"].sum() - 1.0) < 1e-12
