"""The resident sweep loop (vbh_opts.loop = VBH_LOOP_RESIDENT): every sweep of
a step in one cooperative launch, each block holding its slice of (r, d) in
shared memory, one grid barrier per sweep and the FP64 global update run by
every block on the same partial sums.

Against the FP64 oracle at the parity bar of the streaming loop (every
parameter block within 1e-4, the ELBO trace within 1e-6), at sizes that give
one block, many blocks with a ragged last one, and slices long enough for the
FP32 chunk flushes inside a sweep; against the streaming loop; and the
properties the one-launch design has to keep: a fit split into steps is
bitwise the fit in one step, runs repeat bitwise, and requests it cannot
serve are refused."""

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2401_10068_gb300 import synth, vbh

from test_gpu_parity import assert_parity, elbo_close, late_delta_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def handle():
    from paper_2401_10068_gb300 import _build
    _build.build_all()
    h = vbh.Handle(0, torch.cuda.current_stream())
    yield h
    h.close()


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


RES_CASES = [
    # (S, V, seed, sweeps, p_const, stats)
    (1, 700, 1, 5, 0.0, vbh.STATS_PLAIN),                  # one block
    (2, 2_700_001, 2, 4, 0.0, vbh.STATS_PLAIN),            # ~17,800 observations per block: flushes inside a sweep
    (1, 3_000_017, 3, 3, 0.0, vbh.STATS_COMPENSATED),      # the same in the compensated form
    (3, 96_000, 4, 30, 0.0, vbh.STATS_PLAIN),              # the single-data-set workload: 47 blocks, ragged last
    (3, 96_000, 4, 30, 0.0, vbh.STATS_COMPENSATED),
    (5, 250_003, 5, 8, 0.05, vbh.STATS_COMPENSATED),
    (8, 650_000, 6, 5, 0.05, vbh.STATS_PLAIN),             # near the S = 8 capacity (152 blocks)
    (11, 140_000, 7, 4, 0.0, vbh.STATS_COMPENSATED),       # near the S = 11 compensated capacity (64 KB table)
    (11, 40_000, 8, 6, 0.05, vbh.STATS_PLAIN),
]


@pytest.mark.parametrize("S,V,seed,sweeps,p_const,stats", RES_CASES)
def test_resident_parity(handle, S, V, seed, sweeps, p_const, stats):
    alpha = 1.0 if S == 3 else 0.5
    r, d, _ = synth.generate(V, S, seed=seed, alpha=alpha, p_const=p_const)
    prior = O.paper_prior(S)
    ref = O.fit(r, d, prior, tol=0.0, max_iter=sweeps)
    got = handle.fit(_dev(r), _dev(d), S, prior, tol=0.0, max_iter=sweeps, trace=True, stats=stats,
                     loop=vbh.LOOP_RESIDENT)
    assert got["iters"] == sweeps and not got["converged"] and got["status"] == 0
    assert_parity(got, ref, what=(S, V, stats))
    for t, (a, b) in enumerate(zip(got["trace"], ref["trace"])):
        assert elbo_close(a, b, V), (t, a, b)


def test_resident_converged_fit_matches_streaming_and_oracle(handle):
    """96,000 observations, S = 3, rel dELBO < 1e-8 (cap 2,000): the resident
    loop stops where the oracle stops (within 2 %) and where the streaming loop
    stops, and the ELBO changes the stopping test reads match the oracle's."""
    S, V = 3, 96000
    r, d, _ = synth.generate(V, S, seed=1)
    rd, dd = _dev(r), _dev(d)
    prior = O.paper_prior(S)
    ref = O.fit(r, d, prior, tol=1e-8, max_iter=2000)
    res = handle.fit(rd, dd, S, prior, tol=1e-8, max_iter=2000, trace=True, loop=vbh.LOOP_RESIDENT)
    stm = handle.fit(rd, dd, S, prior, tol=1e-8, max_iter=2000, trace=True, loop=vbh.LOOP_STREAM)
    assert ref["converged"] and res["converged"] and stm["converged"]
    assert abs(res["iters"] - ref["iters"]) <= max(2, ref["iters"] // 50), (res["iters"], ref["iters"])
    assert abs(res["iters"] - stm["iters"]) <= 2, (res["iters"], stm["iters"])
    err, n = late_delta_error(res["trace"], ref["trace"], abs(ref["elbo"]))
    assert n >= 20 and err < 5e-10, (n, err)
    assert_parity(res, ref)


def test_resident_steps_are_bitwise_one_call(handle):
    """A fit run as steps of 7 sweeps (one launch each, the data reloaded into
    shared memory every time) equals the fit run in one step, bit for bit:
    the blocks, their slices and every order of summation are the same."""
    S, V, T = 4, 150_001, 35
    r, d, _ = synth.generate(V, S, seed=21, alpha=0.5)
    rd, dd = _dev(r), _dev(d)
    prior = O.paper_prior(S)
    whole = handle.fit(rd, dd, S, prior, tol=0.0, max_iter=T, trace=True, loop=vbh.LOOP_RESIDENT)
    handle.fit_begin(rd, dd, S, prior, tol=0.0, max_iter=T, trace=True, loop=vbh.LOOP_RESIDENT)
    for _ in range(T // 7):
        handle.fit_step(7)
    parts = handle.fit_result()
    assert parts["iters"] == whole["iters"] == T
    for key in ("kappa", "Winv", "b_rho", "elbo"):
        assert np.array_equal(np.asarray(parts[key]), np.asarray(whole[key])), key
    assert np.array_equal(parts["trace"], whole["trace"])
    again = handle.fit(rd, dd, S, prior, tol=0.0, max_iter=T, trace=True, loop=vbh.LOOP_RESIDENT)
    assert np.array_equal(again["trace"], whole["trace"])


def test_resident_stops_on_the_tolerance_mid_step(handle):
    """The stopping test ends the launch in every block at the same sweep: a
    step budget far above the stopping sweep leaves iters at that sweep."""
    S, V = 2, 40_000
    r, d, _ = synth.generate(V, S, seed=3, alpha=0.5)
    rd, dd = _dev(r), _dev(d)
    prior = O.paper_prior(S)
    ref = O.fit(r, d, prior, tol=1e-6, max_iter=5000)
    got = handle.fit(rd, dd, S, prior, tol=1e-6, max_iter=5000, trace=True, loop=vbh.LOOP_RESIDENT)
    assert ref["converged"] and got["converged"] and got["status"] == 0
    assert abs(got["iters"] - ref["iters"]) <= max(2, ref["iters"] // 50), (got["iters"], ref["iters"])
    tr = got["trace"]
    assert abs(tr[-1] - tr[-2]) < 1e-6 * abs(tr[-1]) and abs(tr[-2] - tr[-3]) >= 1e-6 * abs(tr[-2])


@pytest.mark.parametrize("S,V,iters", [(3, 96_000, 20), (8, 60_013, 8)])
def test_resident_em(handle, S, V, iters):
    """EM (Eq. 42-47) through the resident loop against the EM oracle."""
    r, d, _ = synth.generate(V, S, seed=S + 40, alpha=0.5, p_const=0.05)
    prior = O.paper_prior(S)
    ref = O.em_fit(r, d, S, O.em_init(prior), tol=0.0, max_iter=iters)
    got = handle.fit(_dev(r), _dev(d), S, prior, tol=0.0, max_iter=iters, trace=True, method=vbh.EM,
                     loop=vbh.LOOP_RESIDENT)
    assert got["iters"] == iters
    M = S - 1
    nk = np.linalg.norm(ref["K"])
    assert np.linalg.norm(np.asarray(got["kappa"]) - ref["K"]) < 1e-4 * nk
    nl = np.linalg.norm(ref["Linv"])
    assert np.linalg.norm(np.asarray(got["Winv"]).reshape(M, M) - np.asarray(ref["Linv"]).reshape(M, M)) < 1e-4 * nl
    assert abs(got["rho_mean"] - ref["rho"]) < 1e-4 * ref["rho"]
    for t, (a, b) in enumerate(zip(got["trace"], ref["trace"])):
        assert abs(a - b) <= 1e-6 * max(abs(b), float(V)), (t, a, b)


def test_resident_resume_from_given_state(handle):
    """A warm start (VBH_INIT_GIVEN) then resident sweeps equals the oracle's
    continuation of the same state."""
    S, V, T = 5, 60_000, 6
    r, d, _ = synth.generate(V, S, seed=31, alpha=0.5)
    rd, dd = _dev(r), _dev(d)
    prior = O.paper_prior(S)
    half = handle.fit(rd, dd, S, prior, tol=0.0, max_iter=T, loop=vbh.LOOP_STREAM)
    whole = O.fit(r, d, prior, tol=0.0, max_iter=2 * T)
    rest = handle.fit(rd, dd, S, prior, tol=0.0, max_iter=T, init_state=half, loop=vbh.LOOP_RESIDENT)
    assert_parity(rest, whole, what="resumed")


def test_resident_refusals(handle):
    """VBH_LOOP_RESIDENT where the loop cannot run: VBH_EUNSUPPORTED (the data
    set does not fit in shared memory, the tensor-core sweep, the grouped
    sweep); VBH_LOOP_AUTO streams in the same cases."""
    cases = [(11, 500_000, {}), (12, 5_000, {}), (4, 5_000, {"grouped": True})]
    for S, V, kw in cases:
        r, d, _ = synth.generate(V, S, seed=5)
        rd, dd = _dev(r), _dev(d)
        prior = O.paper_prior(S)
        with pytest.raises(vbh.VBHError) as ei:
            handle.fit(rd, dd, S, prior, tol=1e-8, max_iter=3, loop=vbh.LOOP_RESIDENT, **kw)
        assert ei.value.status == -7, (S, V, kw)
        got = handle.fit(rd, dd, S, prior, tol=0.0, max_iter=3, loop=vbh.LOOP_AUTO, **kw)
        assert got["iters"] == 3 and got["status"] == 0
    # an unknown loop value
    r, d, _ = synth.generate(100, 3, seed=6)
    with pytest.raises(vbh.VBHError) as ei:
        handle.fit(_dev(r), _dev(d), 3, None, loop=7)
    assert ei.value.status == -1


def test_table_driven_log_against_numpy(handle):
    """The ELBO of the resident loop takes its logarithms from Tang's
    table-driven method (vbh_selftest_math runs it): within 4 units in the
    last place of max(|ln x|, 1) of numpy's log over the whole exponent range,
    near 1 and at the table's breakpoints; zero, negative, subnormal and
    non-finite inputs give what the library logarithm gives."""
    rng = np.random.default_rng(0)
    j = np.arange(128)
    x = np.concatenate([
        np.exp(rng.uniform(-700.0, 700.0, 200_000)),
        rng.uniform(0.5, 2.0, 200_000),
        1.0 + rng.normal(0.0, 1e-6, 20_000),
        1.0 + j / 128.0, np.nextafter(1.0 + j / 128.0, 0.0), np.nextafter(1.0 + j / 128.0, 3.0),
        [1.0, 2.0, 0.5, 2.0 ** -1022, np.finfo(np.float64).max, 7e4, 4.8e4],
    ])
    out = np.empty_like(x)
    dp = vbh._dp
    rc = vbh._lib().vbh_selftest_math(0, None, 0, x.ctypes.data_as(dp), out.ctypes.data_as(dp), x.size)
    assert rc == 0
    ref = np.log(x)
    err = np.abs(out - ref) / np.maximum(np.abs(ref), 1.0)
    print(f"max error {err.max() / 2.0 ** -52:.2f} units of 2^-52 max(|ln x|, 1)")
    assert err.max() <= 4 * 2.0 ** -52
    assert np.array_equal(out[-7:-4], [0.0, np.log(2.0), -np.log(2.0)]) or np.all(err[-7:-4] <= 2 * 2.0 ** -52)
    special = np.array([0.0, -1.0, np.inf, np.nan, 5e-324, 1e-310])
    so = np.empty_like(special)
    assert vbh._lib().vbh_selftest_math(0, None, 0, special.ctypes.data_as(dp), so.ctypes.data_as(dp), special.size) == 0
    assert so[0] == -np.inf and np.isnan(so[1]) and so[2] == np.inf and np.isnan(so[3])
    np.testing.assert_allclose(so[4:], np.log(special[4:]), rtol=1e-15)


def test_fast_rsqrt_against_numpy(handle):
    """The Cholesky factorisations take 1/sqrt(p) from the PTX approximation
    and one third-order correction: within one unit in the last place of the exact
    value (an extended-precision reference) over the whole exponent range;
    special inputs as the library's rsqrt."""
    rng = np.random.default_rng(1)
    x = np.concatenate([np.exp(rng.uniform(-700.0, 700.0, 200_000)), rng.uniform(0.25, 4.0, 200_000),
                        [1.0, 2.0, 4.0, 0.5, 3.999999999999999, 2.0 ** -1022, np.finfo(np.float64).max]])
    out = np.empty_like(x)
    dp = vbh._dp
    assert vbh._lib().vbh_selftest_math(0, None, 1, x.ctypes.data_as(dp), out.ctypes.data_as(dp), x.size) == 0
    # reference in extended precision (long double: 64 or 113 significant bits)
    xl = x.astype(np.longdouble)
    refl = 1 / np.sqrt(xl)
    ulps = np.abs((out.astype(np.longdouble) - refl) / np.spacing(refl.astype(np.float64)).astype(np.longdouble))
    print(f"max error {float(ulps.max()):.3f} ulp (long double with {np.finfo(np.longdouble).nmant} fraction bits)")
    assert float(ulps.max()) <= 1.0
    assert out[-7] == 1.0 and out[-5] == 0.5            # 1/sqrt(1), 1/sqrt(4)
    special = np.array([0.0, -1.0, np.inf, np.nan, 5e-324])
    so = np.empty_like(special)
    assert vbh._lib().vbh_selftest_math(0, None, 1, special.ctypes.data_as(dp), so.ctypes.data_as(dp), special.size) == 0
    assert so[0] == np.inf and np.isnan(so[1]) and so[2] == 0.0 and np.isnan(so[3])
    np.testing.assert_allclose(so[4], 1.0 / np.sqrt(5e-324), rtol=1e-12)
