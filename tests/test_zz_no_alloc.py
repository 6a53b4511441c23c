"""vbh_fit_static: the allocation-free fit, for callers that cannot allocate
device memory (the device allocator synchronises the GPU, or the memory is
owned by the caller's own pool or budget).  It must give the results of the
handle-based vbh_fit within the tolerances of the other parity tests, on
consecutive calls that share its static scratch array.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes

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


def test_static_fit_matches_the_oracle():
    """Parity with the FP64 oracle itself (not only with the handle fit),
    plain and compensated statistics, on two calls in a row."""
    stream = torch.cuda.current_stream()
    for S, V, seed, sweeps, stats in ((4, 70_001, 31, 8, vbh.STATS_PLAIN), (6, 50_000, 32, 6, vbh.STATS_COMPENSATED)):
        r, d, _ = synth.generate(V, S, seed=seed, alpha=0.5, p_const=0.05)
        prior = O.paper_prior(S)
        ref = O.fit(r, d, prior, tol=0.0, max_iter=sweeps)
        got = vbh.fit_static(torch.from_numpy(r).cuda(), torch.from_numpy(d).cuda(), S, prior, tol=0.0,
                             max_iter=sweeps, trace=True, stream=stream, stats=stats)
        assert got["iters"] == sweeps
        assert _rel(got["kappa"], ref["kappa"]) < 1e-4 and _rel(got["Winv"], ref["Winv"]) < 1e-4
        assert _rel(got["b_rho"], ref["b_rho"]) < 1e-4
        for t, (x, y) in enumerate(zip(got["trace"], ref["trace"])):
            assert abs(x - y) <= 1e-6 * max(abs(y), V), (S, t)


def test_static_fit_stops_issuing_sweeps_after_convergence():
    """A sweep budget far beyond convergence costs about nothing: the call
    stops issuing launches once the fit has converged."""
    import time
    S, V = 3, 96_000
    r, d, _ = synth.generate_device(V, S, seed=1)
    out = vbh.fit_static(r, d, S, None, tol=1e-6, max_iter=100_000)
    assert out["converged"] and out["iters"] < 1000
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    same = vbh.fit_static(r, d, S, None, tol=1e-6, max_iter=out["iters"])
    t1 = time.perf_counter()
    big = vbh.fit_static(r, d, S, None, tol=1e-6, max_iter=100_000)
    t2 = time.perf_counter()
    assert same["iters"] == big["iters"] == out["iters"]
    # 100,000 launches would take about a second; the batched issue adds at most 64 idle ones
    assert (t2 - t1) < (t1 - t0) + 0.1, (t1 - t0, t2 - t1)


def test_static_fit_allocates_no_device_memory():
    """After the first call on the device (which loads every kernel of the
    entry point) no call allocates, also not the first call at an S that has
    never run."""
    prior5 = O.paper_prior(5)
    r5, d5, _ = synth.generate_device(200_000, 5, seed=5)
    r9, d9, _ = synth.generate_device(150_000, 9, seed=6)
    vbh.fit_static(r5, d5, 5, prior5, tol=1e-6, max_iter=50)       # first call on the device (no-op if not the first)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    out = vbh.fit_static(r5, d5, 5, prior5, tol=1e-6, max_iter=50)
    out9 = vbh.fit_static(r9, d9, 9, None, tol=1e-6, max_iter=20)   # an S not launched before in this test
    out9p = vbh.fit_static(r9, d9, 9, None, tol=0.0, max_iter=3, stats=vbh.STATS_PLAIN)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert out["iters"] > 0 and out9["iters"] > 0 and out9p["iters"] == 3


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
    o = vbh.Opts()                                                    # the grouped sweep needs a handle
    vbh._lib().vbh_opts_default(ctypes.byref(o))
    o.grouped = 1
    o.max_iter = 3
    pa = vbh._PriorArgs(None, S)
    res = vbh.Result()
    rc = vbh._lib().vbh_fit_static(vbh._ptr(rg), vbh._ptr(dg), V, S, ctypes.byref(pa.c), ctypes.byref(o),
                                   ctypes.byref(res), 0, None)
    assert rc == -7
