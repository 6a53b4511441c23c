"""Parity of the EM form (Section 4.2, Eq. 42-47) of the CUDA path with the
FP64 CPU oracle.

Same seeded inputs, same start (K0, Lambda_0^{-1}, rho = a0 / b0 from the
prior) and the same number of iterations.  The CUDA path runs EM through the
CAVI sweep kernels (the per-observation sums are the same) with the EM global
update; its log-likelihood comes from the sums of the pass, the oracle's from
the marginal Gaussian directly.  Tolerances as for CAVI: K, Lambda^{-1}, rho
within 1e-4 relative; ln p(r | theta) within 1e-6 of max(|ln p|, V)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2401_10068_gb300 import synth, vbh

pytestmark = pytest.mark.gpu

TOL_PARAM = 1e-4
TOL_LL = 1e-6


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


def ll_close(a, b, V, tol=TOL_LL):
    return abs(a - b) <= tol * max(abs(b), float(V), 1.0)


def assert_em_parity(got, ref, V, what=""):
    M = len(ref["K"])
    if M:
        assert rel(got["kappa"], ref["K"]) < TOL_PARAM, (what, "K", got["kappa"], ref["K"])
        assert rel(got["Winv"], ref["Linv"]) < TOL_PARAM, (what, "Lambda^-1", rel(got["Winv"], ref["Linv"]))
    assert rel(got["rho_mean"], ref["rho"]) < TOL_PARAM, (what, "rho", got["rho_mean"], ref["rho"])
    assert got["rho_mode"] == got["rho_mean"] and got["b_rho"] == 1.0 and got["nu"] == 1.0


CASES = [
    # (S, V, seed, iterations, p_const)
    (1, 5003, 1, 3, 0.0),
    (3, 96000, 2, 20, 0.0),
    (4, 33333, 3, 10, 0.05),
    (8, 60013, 4, 8, 0.05),
    (11, 20011, 5, 5, 0.0),
    (12, 20011, 6, 5, 0.05),            # tensor-core sweep
    (32, 12000, 7, 3, 0.0),
]


@pytest.mark.parametrize("S,V,seed,iters,p_const", CASES)
def test_em_parity_fixed_iterations(handle, S, V, seed, iters, p_const):
    r, d, _ = synth.generate(V, S, seed=seed, alpha=0.5, p_const=p_const)
    prior = O.paper_prior(S)
    ref = O.em_fit(r, d, S, O.em_init(prior), tol=0.0, max_iter=iters)
    got = handle.fit(_dev(r), _dev(d), S, prior, tol=0.0, max_iter=iters, trace=True, method=vbh.EM)
    assert got["iters"] == iters and not got["converged"]
    assert_em_parity(got, ref, V, what=(S, V))
    for t, (a, b) in enumerate(zip(got["trace"], ref["trace"])):
        assert ll_close(a, b, V), (t, a, b)
    assert ll_close(got["elbo"], ref["loglik"], V)


def test_em_loglik_ascends_and_converges(handle):
    S, V = 3, 96000
    r, d, _ = synth.generate(V, S, seed=12, alpha=0.5)
    prior = O.paper_prior(S)
    ref = O.em_fit(r, d, S, O.em_init(prior), tol=1e-7, max_iter=3000)
    got = handle.fit(_dev(r), _dev(d), S, prior, tol=1e-7, max_iter=3000, trace=True, method=vbh.EM)
    assert ref["converged"] and got["converged"]
    # near the stop |dL| / |L| decays slowly, so the FP32 rounding floor of ln p (~1e-8 relative)
    # moves the crossing of 1e-7 by a few iterations
    assert abs(got["iters"] - ref["iters"]) <= max(5, ref["iters"] // 20), (got["iters"], ref["iters"])
    tr = got["trace"]
    assert np.all(np.diff(tr) >= -1e-7 * V)                  # ascent, up to the FP32 rounding floor
    assert abs(tr[-1] - tr[-2]) < 1e-7 * abs(tr[-1])         # the GPU's own stopping test
    same = O.em_fit(r, d, S, O.em_init(prior), tol=0.0, max_iter=got["iters"])
    assert_em_parity(got, same, V, what="converged")
    assert abs(got["elbo"] - same["loglik"]) <= TOL_LL * abs(same["loglik"])
    # against the oracle's own stopping point (a few iterations apart on a slow tail)
    assert rel(got["kappa"], ref["K"]) < 1e-3 and rel(got["Winv"], ref["Linv"]) < 1e-3


def test_em_resume_is_bitwise(handle):
    S, V, T = 5, 40000, 6
    r, d, _ = synth.generate(V, S, seed=13, alpha=0.5)
    rd, dd = _dev(r), _dev(d)
    prior = O.paper_prior(S)
    whole = handle.fit(rd, dd, S, prior, tol=0.0, max_iter=2 * T + 1, method=vbh.EM)
    half = handle.fit(rd, dd, S, prior, tol=0.0, max_iter=T, method=vbh.EM)
    rest = handle.fit(rd, dd, S, prior, tol=0.0, max_iter=T, method=vbh.EM, init_state=half)
    for key in ("kappa", "Winv", "rho_mean"):
        assert np.array_equal(np.asarray(rest[key]), np.asarray(whole[key])), key


def test_em_bf16_form(handle):
    """EM through the tensor-core sweep's BF16 form, last 3 iterations FP32."""
    S, V, iters = 16, 30011, 8
    r, d, _ = synth.generate(V, S, seed=14, alpha=0.5)
    prior = O.paper_prior(S)
    ref = O.em_fit(r, d, S, O.em_init(prior), tol=0.0, max_iter=iters)
    got = handle.fit(_dev(r), _dev(d), S, prior, tol=0.0, max_iter=iters, method=vbh.EM, precision=vbh.BF16,
                     refine_iters=3)
    assert got["iters"] == iters
    assert rel(got["kappa"], ref["K"]) < 1e-3 and rel(got["Winv"], ref["Linv"]) < 1e-3
    assert rel(got["rho_mean"], ref["rho"]) < 1e-3


def test_em_is_refused_where_unsupported(handle):
    S, V = 3, 1000
    r, d, _ = synth.generate(V, S, seed=15)
    with pytest.raises(vbh.VBHError) as ei:
        o, keep, buf = vbh.Handle._opts(0.0, 2, None, S, False, method=vbh.EM)
        res = (vbh.Result * 1)()
        import ctypes
        pa = vbh._PriorArgs(None, S)
        Vs = (ctypes.c_int64 * 1)(V)
        Ss = (ctypes.c_int * 1)(S)
        rt, dt = _dev(r), _dev(d)
        rp = (ctypes.c_void_p * 1)(rt.data_ptr())
        dp = (ctypes.c_void_p * 1)(dt.data_ptr())
        rc = vbh._lib().vbh_fit_batched(handle._h, 1, Vs, Ss, rp, dp, None, ctypes.byref(o), res)
        if rc != 0:
            raise vbh.VBHError(rc, "vbh_fit_batched")
    assert ei.value.status == -7
