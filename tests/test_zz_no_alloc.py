"""vbh_fit_static: the allocation-free fit, for callers that cannot allocate
device memory (the device allocator synchronises the GPU, or the memory is
owned by the caller's own pool or budget).  It must give the results of the
handle-based vbh_fit within the tolerances of the other parity tests, on
consecutive calls that share its static scratch array.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2401_10068_gb300 import _build, synth, vbh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build_all()


def _rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _close(got, ref, V):
    assert got["iters"] == ref["iters"] and got["converged"] == ref["converged"]
    assert _rel(got["kappa"], ref["kappa"]) < 1e-4
    assert _rel(got["Winv"], ref["Winv"]) < 1e-4
    assert _rel(got["b_rho"], ref["b_rho"]) < 1e-4
    assert abs(got["elbo"] - ref["elbo"]) <= 1e-6 * max(abs(ref["elbo"]), V)
    for t, (x, y) in enumerate(zip(got["trace"], ref["trace"])):
        assert abs(x - y) <= 1e-6 * max(abs(y), V), t


def test_static_fit_matches_handle_fit_on_consecutive_calls():
    stream = torch.cuda.current_stream()
    cases = [(8, 300_007, 21, 0.05, 12), (3, 96_000, 22, 0.0, 30)]   # different S: the shared array is reused
    results = []
    for S, V, seed, p_const, sweeps in cases:
        r, d, _ = synth.generate_device(V, S, seed=seed, alpha=0.5, p_const=p_const)
        prior = O.paper_prior(S)
        got = vbh.fit_static(r, d, S, prior, tol=0.0, max_iter=sweeps, trace=True, stream=stream)
        with vbh.Handle(0, stream) as h:
            ref = h.fit(r, d, S, prior, tol=0.0, max_iter=sweeps, trace=True)
        _close(got, ref, V)
        results.append(got)
    # a repeat of the first case after the second gives the first case's result
    S, V, seed, p_const, sweeps = cases[0]
    r, d, _ = synth.generate_device(V, S, seed=seed, alpha=0.5, p_const=p_const)
    again = vbh.fit_static(r, d, S, O.paper_prior(S), tol=0.0, max_iter=sweeps, trace=True, stream=stream)
    np.testing.assert_array_equal(again["kappa"], results[0]["kappa"])
    np.testing.assert_array_equal(again["trace"], results[0]["trace"])


def test_static_fit_allocates_no_device_memory():
    S, V = 5, 200_000
    r, d, _ = synth.generate_device(V, S, seed=5)
    prior = O.paper_prior(S)
    vbh.fit_static(r, d, S, prior, tol=1e-6, max_iter=50)          # first call on the device: address look-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    out = vbh.fit_static(r, d, S, prior, tol=1e-6, max_iter=50)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert out["iters"] > 0


def test_static_fit_rejects_what_it_cannot_hold():
    S, V = 3, 10_000
    r, d, _ = synth.generate(V, S, seed=1)
    rg, dg = torch.from_numpy(r).cuda(), torch.from_numpy(d).cuda()
    with pytest.raises(vbh.VBHError) as e:                            # trace longer than the static array holds
        vbh.fit_static(rg, dg, S, None, tol=0.0, max_iter=vbh.STATIC_TRACE_MAX, trace=True)
    assert e.value.status == -1
    with pytest.raises(vbh.VBHError) as e:                            # host inputs would need a staging buffer
        vbh.fit_static(r, d, S, None, tol=0.0, max_iter=3)
    assert e.value.status == -1
    ok = vbh.fit_static(rg, dg, S, None, tol=0.0, max_iter=vbh.STATIC_TRACE_MAX - 1, trace=True)
    assert ok["iters"] == vbh.STATIC_TRACE_MAX - 1
