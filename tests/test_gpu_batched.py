"""The batched form (vbh_fit_batched): many independent data sets with uneven
V and S in one device loop.  Each data set must follow exactly the schedule of
a single fit: its results match the FP64 oracle (and the single-data-set
CUDA path) after the same number of sweeps, with the parity tolerances of
test_gpu_parity; in convergence mode each data set retires at its own sweep."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2401_10068_gb300 import _build, synth, vbh
from test_gpu_parity import elementwise_errors

pytestmark = pytest.mark.gpu

TOL_P, TOL_E = 1e-4, 1e-6


@pytest.fixture(scope="module")
def handle():
    _build.build_all()
    h = vbh.Handle(0, torch.cuda.current_stream())
    yield h
    h.close()


def _rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    n = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (n if n > 0 else 1.0)


def _check(got, ref, V, what):
    if len(ref["kappa"]):
        assert _rel(got["kappa"], ref["kappa"]) < TOL_P, (what, "kappa")
        assert _rel(got["Winv"], ref["Winv"]) < TOL_P, (what, "Winv")
    assert _rel(got["b_rho"], ref["b_rho"]) < TOL_P, (what, "b_rho")
    assert abs(got["elbo"] - ref["elbo"]) <= TOL_E * max(abs(ref["elbo"]), V, 1.0), (what, got["elbo"], ref["elbo"])


def _mixed_batch(seed0=500):
    # uneven sizes: empty, smaller than a tile, one observation either side of
    # a tile (896 observations), two tiles, ragged, several chunks
    specs = [(3, 0), (1, 1000), (2, 895), (2, 896), (8, 897), (8, 1792), (3, 96000), (4, 50001), (5, 12000),
             (6, 33333), (7, 20000), (8, 60013), (9, 9600), (10, 15000), (11, 8000), (3, 250_000), (8, 700_001)]
    rs, ds, Ss, host = [], [], [], []
    for k, (S, V) in enumerate(specs):
        r, d, _ = synth.generate(max(V, 1), S, seed=seed0 + k, alpha=0.5, p_const=0.05)
        r, d = r[:V], d[:V]
        host.append((r, d))
        rs.append(torch.from_numpy(r).cuda() if V else None)
        ds.append(torch.from_numpy(d).cuda() if V else None)
        Ss.append(S)
    return specs, rs, ds, Ss, host


def test_batched_matches_oracle_fixed_sweeps(handle):
    specs, rs, ds, Ss, host = _mixed_batch()
    sweeps = 6
    priors = [O.paper_prior(S, n0=S + 1.0) if V == 0 else O.paper_prior(S) for S, V in specs]
    got = handle.fit_batched(rs, ds, Ss, priors, tol=0.0, max_iter=sweeps, trace=True)
    for (S, V), g, (r, d), p in zip(specs, got, host, priors):
        ref = O.fit(r, d, p, tol=0.0, max_iter=sweeps)
        assert g["iters"] == sweeps
        _check(g, ref, V, (S, V))
        if V > 0:
            ew = elementwise_errors(g, ref)
            assert all(v < TOL_P for v in ew.values()), (S, V, ew)
        for t, (a, b) in enumerate(zip(g["trace"], ref["trace"])):
            assert abs(a - b) <= TOL_E * max(abs(b), V, 1.0), (S, V, t)


def test_batched_matches_single_fits_with_retirement(handle):
    """tol > 0: data sets converge after different numbers of sweeps.  Each
    data set stops exactly where its own ELBO trace meets the rule, and its
    state equals a single fit run for that many sweeps."""
    specs, rs, ds, Ss, host = _mixed_batch(seed0=900)
    keep = [i for i, (S, V) in enumerate(specs) if V > 0]
    rs, ds, Ss = [rs[i] for i in keep], [ds[i] for i in keep], [Ss[i] for i in keep]
    tol = 1e-6
    got = handle.fit_batched(rs, ds, Ss, None, tol=tol, max_iter=600, trace=True)
    iters = set()
    for g, r, d, S in zip(got, rs, ds, Ss):
        tr = g["trace"]
        rel = np.abs(np.diff(tr)) / np.abs(tr[1:])
        if g["converged"]:
            assert rel[-1] < tol and np.all(rel[:-1] >= tol), S
        else:
            assert g["iters"] == 600 and np.all(rel >= tol)
        one = handle.fit(r, d, S, None, tol=0.0, max_iter=g["iters"])
        _check(g, one, r.shape[0], S)
        iters.add(g["iters"])
    assert len(iters) > 3            # retirement really happened at different sweeps


def test_batched_given_init_and_host_inputs(handle):
    specs, rs, ds, Ss, host = _mixed_batch(seed0=1300)
    keep = [i for i, (S, V) in enumerate(specs) if V > 0][:6]
    rs, ds, Ss = [rs[i] for i in keep], [ds[i] for i in keep], [Ss[i] for i in keep]
    hr = [host[i][0] for i in keep]
    hd = [host[i][1] for i in keep]
    a = handle.fit_batched(rs, ds, Ss, None, tol=0.0, max_iter=5)
    b = handle.fit_batched(hr, hd, Ss, None, tol=0.0, max_iter=5)          # host numpy inputs, staged
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x["kappa"], y["kappa"])
        assert x["elbo"] == y["elbo"]
    # resume from the 5-sweep states for 4 more sweeps = 9 sweeps in one go
    c = handle.fit_batched(rs, ds, Ss, None, tol=0.0, max_iter=4, init_states=a)
    full = handle.fit_batched(rs, ds, Ss, None, tol=0.0, max_iter=9)
    for x, y in zip(c, full):
        np.testing.assert_array_equal(x["kappa"], y["kappa"])
        np.testing.assert_array_equal(x["Winv"], y["Winv"])


def test_batched_direct_mode_and_determinism(monkeypatch):
    specs, rs, ds, Ss, host = _mixed_batch(seed0=1700)
    keep = [i for i, (S, V) in enumerate(specs) if V > 0]     # V = 0 with the improper default prior: no ELBO
    rs, ds, Ss = [rs[i] for i in keep], [ds[i] for i in keep], [Ss[i] for i in keep]
    with vbh.Handle(0, torch.cuda.current_stream()) as h1:
        a = h1.fit_batched(rs, ds, Ss, None, tol=1e-6, max_iter=300, trace=True)
        a2 = h1.fit_batched(rs, ds, Ss, None, tol=1e-6, max_iter=300, trace=True)
    monkeypatch.setenv("VBH_LAUNCH", "direct")
    with vbh.Handle(0, torch.cuda.current_stream()) as h2:
        b = h2.fit_batched(rs, ds, Ss, None, tol=1e-6, max_iter=300, trace=True)
    for x, y, z in zip(a, a2, b):
        assert x["iters"] == y["iters"] == z["iters"]
        np.testing.assert_array_equal(x["trace"], y["trace"])
        np.testing.assert_array_equal(x["trace"], z["trace"])


def test_batched_improper_empty_data_set_is_reported(handle):
    """V = 0 with n0 = 1 <= M - 1: the posterior is the improper prior, the ELBO
    is not finite, the data set reports VBH_ENONFINITE, the others are fine."""
    r, d, _ = synth.generate(5000, 3, seed=3)
    with pytest.raises(vbh.VBHError) as e:
        handle.fit_batched([torch.from_numpy(r).cuda(), None], [torch.from_numpy(d).cuda(), None], [3, 3], None,
                           tol=0.0, max_iter=3)
    assert e.value.status == -4
    assert e.value.results[0]["status"] == 0 and e.value.results[1]["status"] == -4


def test_batched_errors(handle):
    r, d, _ = synth.generate(1000, 12, seed=1)
    with pytest.raises(vbh.VBHError) as e:
        handle.fit_batched([torch.from_numpy(r).cuda()], [torch.from_numpy(d).cuda()], [12], None, tol=0.0,
                           max_iter=2)
    assert e.value.status == -7
    r, d, _ = synth.generate(1000, 3, seed=1)
    with pytest.raises(vbh.VBHError) as e:              # r on the device, d on the host
        handle.fit_batched([torch.from_numpy(r).cuda()], [d], [3], None, tol=0.0, max_iter=2)
    assert e.value.status == -1
    assert handle.fit_batched([], [], [], None) == []


def test_batched_many_small_data_sets_compensated(handle):
    """Dozens of small data sets per class: a pass block changes data set
    every few tiles, so the compensated form rebuilds its table of profile
    terms at nearly every chunk (the compute warps' rendezvous), and chunks
    of one tile or only a tail are common.  Each data set against the oracle
    at equal sweeps."""
    rng = np.random.default_rng(77)
    specs = [(4, int(v)) for v in rng.integers(100, 6000, 40)] + [(9, int(v)) for v in rng.integers(800, 5000, 16)]
    specs += [(4, 896), (4, 1), (9, 895)]
    rs, ds, Ss, host = [], [], [], []
    for k, (S, V) in enumerate(specs):
        r, d, _ = synth.generate(V, S, seed=4000 + k, alpha=0.5)
        host.append((r, d))
        rs.append(torch.from_numpy(r).cuda())
        ds.append(torch.from_numpy(d).cuda())
        Ss.append(S)
    sweeps = 4
    priors = [O.paper_prior(S, n0=S + 1.0) for S, _ in specs]     # proper even at V = 1
    got = handle.fit_batched(rs, ds, Ss, priors, tol=0.0, max_iter=sweeps, trace=True, stats=vbh.STATS_COMPENSATED)
    for (S, V), g, (r, d), p in zip(specs, got, host, priors):
        ref = O.fit(r, d, p, tol=0.0, max_iter=sweeps)
        assert g["iters"] == sweeps
        _check(g, ref, V, (S, V))
        for t, (a, b) in enumerate(zip(g["trace"], ref["trace"])):
            assert abs(a - b) <= TOL_E * max(abs(b), V, 1.0), (S, V, t)
    plan = handle.batched_plan()
    assert [p["S"] for p in plan] == [4, 9]
    for p in plan:           # below 2^26 observations: the default shape, not timed
        assert p["tile"] == 896 and p["chunk_tiles"] == 32 and p["stages"] == 3 and p["pass_ms"] == 0.0
        assert p["blocks_per_sm"] >= 1


def test_batched_autotuned_shape_matches_default_shape(handle):
    """At >= 2^26 observations the pass shape (tiles per chunk, stages) is
    autotuned per class; the statistics do not depend on the stage count and
    the chunk rows are summed in order, so the fit equals the oracle's as
    before, and the plan reports a timed candidate for every class."""
    specs = [(3, 30_000_000), (6, 20_000_000), (6, 7_000_001), (10, 12_000_000)]
    rs, ds, Ss = [], [], []
    for k, (S, V) in enumerate(specs):
        r, d, _ = synth.generate_device(V, S, seed=5100 + k, alpha=0.5)
        rs.append(r)
        ds.append(d)
        Ss.append(S)
    got = handle.fit_batched(rs, ds, Ss, None, tol=0.0, max_iter=2, trace=True)
    plan = handle.batched_plan()
    assert [p["S"] for p in plan] == [3, 6, 10]
    for p in plan:
        assert p["chunk_tiles"] in (8, 32, 128) and 2 <= p["stages"] <= 8 and p["pass_ms"] > 0.0
    for (S, V), g, r, d in zip(specs, got, rs, ds):
        one = handle.fit(r, d, S, None, tol=0.0, max_iter=2, trace=True)
        _check(g, one, V, (S, V))
        for t, (a, b) in enumerate(zip(g["trace"], one["trace"])):
            assert abs(a - b) <= TOL_E * max(abs(b), V, 1.0), (S, V, t)
