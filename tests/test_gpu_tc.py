"""Parity of the tensor-core sweep (12 <= S <= 32) with the FP64 CPU oracle.

The sweep for these S runs the two M^2 contractions per observation as BF16
tcgen05 MMAs with FP32 accumulation; every FP32 operand is split into BF16
parts.  VBH_FP32 (three parts) carries the FP32 values and is held to the same
bar as the CUDA-core sweep: parameters within 1e-4 relative, the ELBO within
1e-6 relative (of max(|L|, V)).  VBH_BF16 (two parts, 16 significant bits) is
the fast form: a 16-bit operand moves q_i, t_i and each (w_i^2 - c_i) D_i D_i^T
term by about 2^-17 relative, so a fixed number of its sweeps stays within
1e-3 of the oracle; with its FP32 refinement sweeps a converged fit reaches
the oracle's optimum (ELBO within 1e-6).
"""
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


def elbo_close(a, b, V, tol=TOL_ELBO):
    return abs(a - b) <= tol * max(abs(b), float(V), 1.0)


def errors(got, ref):
    return {"kappa": rel(got["kappa"], ref["kappa"]), "Winv": rel(got["Winv"], ref["Winv"]),
            "b_rho": rel(got["b_rho"], ref["b_rho"]),
            "elbo": abs(got["elbo"] - ref["elbo"]) / max(abs(ref["elbo"]), ref["nu"], 1.0)}


def assert_parity(got, ref, tol_param=TOL_PARAM, tol_elbo=TOL_ELBO, what=""):
    e = errors(got, ref)
    for key in ("kappa", "Winv", "b_rho"):
        assert e[key] < tol_param, (what, key, e)
    for key in ("a_rho", "nu", "lam"):
        assert got[key] == pytest.approx(ref[key], rel=1e-14), (what, key)
    assert e["elbo"] <= tol_elbo, (what, "elbo", got["elbo"], ref["elbo"])


CASES = [
    # (S, V, seed, sweeps, p_const)
    (12, 20011, 21, 8, 0.05),
    (13, 77, 22, 4, 0.0),               # one partial tile
    (16, 50021, 23, 6, 0.0),
    (20, 30000, 24, 5, 0.05),
    (32, 20000, 25, 4, 0.0),            # the largest S
    (12, 700_003, 26, 3, 0.05),         # ~36 tiles per block: several G' epochs, ragged tail
    (24, 400_001, 27, 2, 0.0),
]


@pytest.mark.parametrize("S,V,seed,sweeps,p_const", CASES)
def test_fp32_form_parity_fixed_sweeps(handle, S, V, seed, sweeps, p_const):
    r, d, _ = synth.generate(V, S, seed=seed, alpha=0.5, p_const=p_const)
    prior = O.paper_prior(S)
    ref = O.fit(r, d, prior, tol=0.0, max_iter=sweeps)
    got = handle.fit(_dev(r), _dev(d), S, prior, tol=0.0, max_iter=sweeps, trace=True)
    assert got["iters"] == sweeps and not got["converged"]
    assert_parity(got, ref, what=(S, V))
    for t, (a, b) in enumerate(zip(got["trace"], ref["trace"])):
        assert elbo_close(a, b, V), (t, a, b)


def test_fp32_form_host_inputs_and_determinism(handle):
    S, V = 16, 30011
    r, d, _ = synth.generate(V, S, seed=31, alpha=0.5)
    prior = O.paper_prior(S)
    a = handle.fit(r, d, S, prior, tol=0.0, max_iter=5, trace=True)          # host pointers: staged
    b = handle.fit(_dev(r), _dev(d), S, prior, tol=0.0, max_iter=5, trace=True)
    for key in ("kappa", "Winv", "b_rho", "elbo", "trace"):
        assert np.array_equal(np.asarray(a[key]), np.asarray(b[key])), key


def test_zero_observations_give_the_prior(handle):
    S = 12
    prior = O.paper_prior(S, n0=14.0)          # proper Wishart prior: with V = 0 the ELBO is finite (0)
    got = handle.fit(None, None, S, prior, tol=0.0, max_iter=2, V=0)
    ref = O.fit(np.zeros(0, np.float32), np.zeros((0, S), np.float32), prior, tol=0.0, max_iter=2)
    assert_parity(got, ref, what="V=0")


def test_non_binary_profiles_exact_in_bf16(handle):
    """Profiles in {0, 1/4, 1/2, 3/4, 1}: exact in BF16, not binary, so the
    sweep forms each (w_i^2 - c_i) d_ij in FP32 before splitting it."""
    S, V = 14, 40009
    r, d, _ = synth.generate(V, S, seed=41, alpha=0.5)
    q = (np.arange(V * S).reshape(V, S) * 2654435761 % 5).astype(np.float32) * 0.25
    d = np.where(d > 0, np.maximum(q, 0.25), 0.0).astype(np.float32)
    assert set(np.unique(d)) <= {0.0, 0.25, 0.5, 0.75, 1.0} and np.any((d != 0) & (d != 1))
    prior = O.paper_prior(S)
    ref = O.fit(r, d, prior, tol=0.0, max_iter=5)
    got = handle.fit(_dev(r), _dev(d), S, prior, tol=0.0, max_iter=5)
    assert_parity(got, ref, what="quarters")


def test_profiles_inexact_in_bf16(handle):
    """VBH_FP32 refuses profiles whose differences d_j - d_S BF16 cannot hold;
    VBH_BF16 rounds those differences."""
    S, V = 12, 20000
    r, d, _ = synth.generate(V, S, seed=42, alpha=0.5)
    d = (d * np.float32(0.3)).astype(np.float32)
    prior = O.paper_prior(S)
    with pytest.raises(vbh.VBHError) as ei:
        handle.fit(_dev(r), _dev(d), S, prior, tol=0.0, max_iter=2)
    assert ei.value.status == -7
    # the BF16 form rounds D_j = d_j - d_S to BF16 and keeps y = r - d_S in FP32: the oracle
    # gets the profiles d_S + bf16(d_j - d_S), which reproduce exactly those values
    dS = d[:, S - 1:]
    D16 = torch.from_numpy((d[:, :S - 1] - dS).astype(np.float32)).to(torch.bfloat16).to(torch.float32).numpy()
    d16 = np.concatenate([(dS + D16).astype(np.float32), dS], axis=1)
    assert np.array_equal((d16[:, :S - 1] - dS).astype(np.float32), D16)
    ref = O.fit(r, d16, prior, tol=0.0, max_iter=4)
    got = handle.fit(_dev(r), _dev(d), S, prior, tol=0.0, max_iter=4, precision=vbh.BF16, refine_iters=0)
    e = errors(got, ref)
    assert max(e["kappa"], e["Winv"], e["b_rho"]) < 1e-3 and e["elbo"] < 1e-4, e


@pytest.mark.parametrize("S,V,seed", [(12, 50021, 51), (20, 30011, 52), (32, 20000, 53)])
def test_bf16_form_error_fixed_sweeps(handle, S, V, seed):
    r, d, _ = synth.generate(V, S, seed=seed, alpha=0.5, p_const=0.05)
    prior = O.paper_prior(S)
    ref = O.fit(r, d, prior, tol=0.0, max_iter=6)
    got = handle.fit(_dev(r), _dev(d), S, prior, tol=0.0, max_iter=6, precision=vbh.BF16, refine_iters=0)
    e = errors(got, ref)
    print(f"BF16 form, S={S}, V={V}, 6 sweeps: {e}")
    assert max(e["kappa"], e["Winv"], e["b_rho"]) < 1e-3 and e["elbo"] < 1e-4, e
    # refinement: the last two of the six sweeps in FP32
    got2 = handle.fit(_dev(r), _dev(d), S, prior, tol=0.0, max_iter=6, precision=vbh.BF16, refine_iters=2)
    assert got2["iters"] == 6
    e2 = errors(got2, ref)
    assert max(e2["kappa"], e2["Winv"], e2["b_rho"]) < 1e-3 and e2["elbo"] < 1e-4, e2


@pytest.fixture(scope="module")
def converged_case():
    """S = 12, V = 500,000 (4,096 profiles, ~26 tiles per block), run to rel dELBO < 1e-7."""
    S, V = 12, 500_000
    r, d, _ = synth.generate(V, S, seed=5, alpha=0.5)
    prior = O.paper_prior(S)
    ref = O.fit_grouped(O.group_profiles(r, d, S), prior, tol=1e-7, max_iter=3000)
    assert ref["converged"]
    return S, V, r, d, prior, ref


def test_fp32_form_converged_fit(handle, converged_case):
    S, V, r, d, prior, ref = converged_case
    got = handle.fit(_dev(r), _dev(d), S, prior, tol=1e-7, max_iter=3000, trace=True)
    assert got["converged"]
    assert abs(got["iters"] - ref["iters"]) <= max(3, ref["iters"] // 50), (got["iters"], ref["iters"])
    assert_parity(got, ref, what="converged")
    assert np.all(np.diff(got["trace"]) >= -1e-7 * V)


def test_bf16_form_with_refinement_reaches_the_optimum(handle, converged_case):
    S, V, r, d, prior, ref = converged_case
    got = handle.fit(_dev(r), _dev(d), S, prior, tol=1e-7, max_iter=3000, precision=vbh.BF16,
                     refine_iters=50, trace=True)
    assert got["converged"]
    e = errors(got, ref)
    print(f"BF16 + FP32 refinement, converged: iters {got['iters']} (oracle {ref['iters']}), {e}")
    assert e["elbo"] <= TOL_ELBO, e
    assert max(e["kappa"], e["Winv"], e["b_rho"]) < 1e-3, e


def test_bf16_stepwise_equals_one_call(handle):
    S, V = 16, 40000
    r, d, _ = synth.generate(V, S, seed=61, alpha=0.5)
    prior = O.paper_prior(S)
    rd, dd = _dev(r), _dev(d)
    one = handle.fit(rd, dd, S, prior, tol=1e-6, max_iter=60, precision=vbh.BF16, refine_iters=7, trace=True)
    handle.fit_begin(rd, dd, S, prior, tol=1e-6, max_iter=60, precision=vbh.BF16, refine_iters=7, trace=True)
    conv = False
    for _ in range(30):
        conv = handle.fit_step(5)
    steps = handle.fit_result()
    assert steps["iters"] == one["iters"] and bool(conv) == bool(one["converged"])
    for key in ("kappa", "Winv", "b_rho", "elbo"):
        assert np.array_equal(np.asarray(steps[key]), np.asarray(one[key])), key


def test_elbo_entry_point(handle):
    S, V = 18, 25000
    r, d, _ = synth.generate(V, S, seed=71, alpha=0.5)
    prior = O.paper_prior(S)
    ref = O.fit(r, d, prior, tol=0.0, max_iter=3)
    want, _ = O.elbo_at(r, d, prior, ref)
    got = handle.elbo(_dev(r), _dev(d), S, ref, prior)
    assert elbo_close(got, want, V), (got, want)


def per_entry(got, ref):
    """Largest per-entry relative error of kappa and W^{-1} (entries whose
    reference is below 1e-12 of the block's largest are skipped)."""
    out = {}
    for key in ("kappa", "Winv"):
        a, b = np.ravel(np.asarray(got[key], np.float64)), np.ravel(np.asarray(ref[key], np.float64))
        keep = np.abs(b) > 1e-12 * np.abs(b).max()
        out[key] = float(np.max(np.abs(a[keep] - b[keep]) / np.abs(b[keep])))
    return out


@pytest.fixture(scope="module")
def s32_multi_epoch():
    """S = 32 at V = 700,001: about 36 tiles of 128 observations per block on
    152 blocks, so every block runs two full 16-tile epochs of tensor-memory
    accumulation, the compensated FP32 sums across epochs and a partial third
    epoch; the last tile is ragged.  Oracle: sweep 0 and two sweeps."""
    S, V, sweeps = 32, 700_001, 2
    r, d, _ = synth.generate(V, S, seed=81, alpha=0.5, p_const=0.05)
    prior = O.paper_prior(S)
    ref = O.fit(r, d, prior, tol=0.0, max_iter=sweeps)
    return S, V, sweeps, r, d, prior, ref


def test_s32_fp32_form_parity_multi_epoch(handle, s32_multi_epoch):
    S, V, sweeps, r, d, prior, ref = s32_multi_epoch
    got = handle.fit(_dev(r), _dev(d), S, prior, tol=0.0, max_iter=sweeps, trace=True)
    e, pe = errors(got, ref), per_entry(got, ref)
    print(f"FP32 form, S=32, V={V}: norm-wise {e}, per-entry max {pe}")
    assert_parity(got, ref, what="S=32 multi-epoch")
    for t, (a, b) in enumerate(zip(got["trace"], ref["trace"])):
        assert elbo_close(a, b, V), (t, a, b)


def test_s32_bf16_form_error_multi_epoch(handle, s32_multi_epoch):
    """The BF16 form without refinement against the FP64 oracle at the same
    multi-epoch size.  Stated bound per parameter block: 1e-3 relative
    (norm-wise) for kappa, W^{-1} and b_rho, 1e-4 for the ELBO."""
    S, V, sweeps, r, d, prior, ref = s32_multi_epoch
    got = handle.fit(_dev(r), _dev(d), S, prior, tol=0.0, max_iter=sweeps, precision=vbh.BF16, refine_iters=0)
    e, pe = errors(got, ref), per_entry(got, ref)
    print(f"BF16 form, S=32, V={V}: norm-wise {e}, per-entry max {pe}")
    assert max(e["kappa"], e["Winv"], e["b_rho"]) < 1e-3 and e["elbo"] < 1e-4, e


def test_s32_full_size_invariants(handle):
    """The precision workload at full size (N = 1,048,576 cells x G = 512
    genes = 536,870,912 observations, S = 32), where the per-observation oracle
    is out of reach: properties that hold at any size.  a_rho, nu and lambda
    are exact functions of V (Eq. 16, 22, 23); W^{-1} stays symmetric positive
    definite; the ELBO does not decrease over the FP32-form sweeps (coordinate
    ascent, Eq. 12, to 1e-9 |L|); and the BF16 schedule (BF16-form sweeps,
    then FP32-form refinement) ends within 1e-4 (parameters) and 1e-6 (ELBO)
    of the same number of FP32-form sweeps."""
    S, V = 32, (1 << 20) * 512
    sweeps, refine = 8, 3
    r, d, _ = synth.generate_device(V, S, seed=3, alpha=0.5, p_const=0.05)
    prior = O.paper_prior(S)
    fp32 = handle.fit(r, d, S, prior, tol=0.0, max_iter=sweeps, trace=True)
    sched = handle.fit(r, d, S, prior, tol=0.0, max_iter=sweeps, precision=vbh.BF16, refine_iters=refine)
    del r, d
    torch.cuda.empty_cache()
    M = S - 1
    for res in (fp32, sched):
        assert res["iters"] == sweeps and res["status"] == 0
        assert res["a_rho"] == 0.5 + V / 2 and res["nu"] == 1.0 + V and res["lam"] == 1e-3 + V
        W = np.asarray(res["Winv"])
        assert np.allclose(W, W.T, rtol=0, atol=1e-12 * np.abs(W).max())
        np.linalg.cholesky(W)                                    # raises unless positive definite
        assert np.all(np.isfinite(res["kappa"])) and len(res["kappa"]) == M
    tr = np.asarray(fp32["trace"])
    assert np.all(np.diff(tr) >= -1e-9 * np.abs(tr[1:])), np.diff(tr)
    e = errors(sched, fp32)
    print(f"BF16 schedule ({sweeps - refine} + {refine}) vs FP32 form at V={V}: {e}, per-entry {per_entry(sched, fp32)}")
    assert max(e["kappa"], e["Winv"], e["b_rho"]) < 1e-4 and e["elbo"] < 1e-6, e
