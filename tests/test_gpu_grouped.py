"""The exact profile-grouped sweep (binary profiles) against the FP64 oracle.

The grouped form histograms (count, sum y, sum y^2) per profile once and runs
each sweep over the 2^S profiles; the oracle's profile-grouped fit (pinned
against its per-observation fit) is the reference, and the GPU's own
per-observation sweep is compared as well.  Same tolerances as the other
parity tests: parameters within 1e-4 relative, ELBO / log-likelihood within
1e-6 of max(|L|, V)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2401_10068_gb300 import synth, vbh

pytestmark = pytest.mark.gpu

TOL_PARAM = 1e-4
TOL_ELBO = 1e-6


@pytest.fixture(scope="module")
def handle():
    from paper_2401_10068_gb300 import _build
    _build.build_all()
    h = vbh.Handle(0, torch.cuda.current_stream())
    yield h
    h.close()


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def close(a, b, V, tol=TOL_ELBO):
    return abs(a - b) <= tol * max(abs(b), float(V), 1.0)


def assert_parity(got, ref, V, tol=TOL_PARAM, what=""):
    if len(ref["kappa"]):
        assert rel(got["kappa"], ref["kappa"]) < tol, (what, "kappa")
        assert rel(got["Winv"], ref["Winv"]) < tol, (what, "Winv", rel(got["Winv"], ref["Winv"]))
    assert rel(got["b_rho"], ref["b_rho"]) < tol, (what, "b_rho")
    assert close(got["elbo"], ref["elbo"], V), (what, got["elbo"], ref["elbo"])


CASES = [
    # (S, V, seed, sweeps, p_const)
    (1, 5003, 1, 3, 0.0),
    (2, 20011, 2, 10, 0.0),
    (3, 96000, 3, 25, 0.05),
    (8, 1_000_003, 4, 10, 0.05),
    (11, 150_001, 10, 5, 0.05),         # the last S of the warp-per-code form
    (12, 300_007, 5, 6, 0.0),           # from here a lane per code
    (14, 500_009, 11, 4, 0.0),
    (16, 200_003, 6, 4, 0.05),
]


@pytest.mark.parametrize("S,V,seed,sweeps,p_const", CASES)
def test_grouped_parity_fixed_sweeps(handle, S, V, seed, sweeps, p_const):
    r, d, _ = synth.generate(V, S, seed=seed, alpha=0.5, p_const=p_const)
    prior = O.paper_prior(S)
    ref = O.fit_grouped(O.group_profiles(r, d, S), prior, tol=0.0, max_iter=sweeps)
    rd, dd = _dev(r), _dev(d)
    got = handle.fit(rd, dd, S, prior, tol=0.0, max_iter=sweeps, trace=True, grouped=True)
    assert got["iters"] == sweeps
    assert_parity(got, ref, V, what=(S, V))
    for t, (a, b) in enumerate(zip(got["trace"], ref["trace"])):
        assert close(a, b, V), (t, a, b)
    # and the GPU's per-observation sweep (same FP32 globals per pass)
    if S <= 12:
        per_obs = handle.fit(rd, dd, S, prior, tol=0.0, max_iter=sweeps)
        assert_parity(got, per_obs, V, what=("per-observation", S))


def test_grouped_converged(handle):
    S, V = 3, 2_000_000
    r, d, _ = synth.generate(V, S, seed=7, alpha=1.0)
    prior = O.paper_prior(S)
    ref = O.fit_grouped(O.group_profiles(r, d, S), prior, tol=1e-7, max_iter=3000)
    got = handle.fit(_dev(r), _dev(d), S, prior, tol=1e-7, max_iter=3000, trace=True, grouped=True)
    assert ref["converged"] and got["converged"]
    assert abs(got["iters"] - ref["iters"]) <= max(5, ref["iters"] // 20), (got["iters"], ref["iters"])
    same = O.fit_grouped(O.group_profiles(r, d, S), prior, tol=0.0, max_iter=got["iters"])
    assert_parity(got, same, V, what="converged")


def test_grouped_em(handle):
    S, V, iters = 5, 200_003, 12
    r, d, _ = synth.generate(V, S, seed=8, alpha=0.5, p_const=0.05)
    prior = O.paper_prior(S)
    ref = O.em_fit(r, d, S, O.em_init(prior), tol=0.0, max_iter=iters)
    got = handle.fit(_dev(r), _dev(d), S, prior, tol=0.0, max_iter=iters, trace=True, grouped=True, method=vbh.EM)
    assert rel(got["kappa"], ref["K"]) < TOL_PARAM and rel(got["Winv"], ref["Linv"]) < TOL_PARAM
    assert rel(got["rho_mean"], ref["rho"]) < TOL_PARAM
    for t, (a, b) in enumerate(zip(got["trace"], ref["trace"])):
        assert close(a, b, V), (t, a, b)


def test_grouped_em_lane_per_code(handle):
    """EM through the lane-per-code form of the grouped sweep (S = 13)."""
    S, V, iters = 13, 300_007, 5
    r, d, _ = synth.generate(V, S, seed=12, alpha=0.5)
    prior = O.paper_prior(S)
    ref = O.em_fit(r, d, S, O.em_init(prior), tol=0.0, max_iter=iters)
    got = handle.fit(_dev(r), _dev(d), S, prior, tol=0.0, max_iter=iters, trace=True, grouped=True, method=vbh.EM)
    assert rel(got["kappa"], ref["K"]) < TOL_PARAM and rel(got["Winv"], ref["Linv"]) < TOL_PARAM
    assert rel(got["rho_mean"], ref["rho"]) < TOL_PARAM
    for t, (a, b) in enumerate(zip(got["trace"], ref["trace"])):
        assert close(a, b, V), (t, a, b)


def test_grouped_refuses_non_binary_profiles(handle):
    S, V = 4, 10000
    r, d, _ = synth.generate(V, S, seed=9)
    d = d.copy()
    d[123, 2] = 0.5
    with pytest.raises(vbh.VBHError) as ei:
        handle.fit(_dev(r), _dev(d), S, O.paper_prior(S), tol=0.0, max_iter=2, grouped=True)
    assert ei.value.status == -1
    with pytest.raises(vbh.VBHError) as ei:
        r2, d2, _ = synth.generate(100, 17, seed=9)
        handle.fit(_dev(r2), _dev(d2), 17, O.paper_prior(17), tol=0.0, max_iter=2, grouped=True)
    assert ei.value.status == -7
