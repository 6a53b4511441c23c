"""Pins of the expectation-maximisation oracle (Section 4.2, Eq. 42-47).

EM maximises the marginal likelihood p(r | K, Lambda, rho) with beta_i
integrated out.  The pins come from outside the oracle's own formulas:
the EM ascent property, a closed form at S = 1, one-dimensional quadrature of
the marginal, and stationarity of the likelihood at the EM fixed point
(checked by finite differences, with a perturbed point as the control)."""
import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_2401_10068_gb300 import synth


@pytest.mark.parametrize("S", [2, 3, 4])
def test_em_loglik_never_decreases(S):
    r, d, _ = synth.generate(3000, S, seed=20 + S, alpha=0.5, p_const=0.05)
    res = O.em_fit(r, d, S, O.em_init(O.paper_prior(S)), tol=0.0, max_iter=80)
    tr = res["trace"]
    assert res["iters"] == 80 and tr.shape == (81,)
    assert np.all(np.diff(tr) >= -1e-10 * np.abs(tr[1:])), np.min(np.diff(tr))
    assert tr[-1] > tr[0]


def test_em_single_component_closed_form():
    """S = 1: no beta; r_i ~ N(d_i, 1/rho), so one step gives the maximum-
    likelihood precision V / sum (r_i - d_i)^2, after which the iteration stays
    there and ln p = -V/2 (ln 2 pi - ln rho + 1)."""
    r, d, _ = synth.generate(5000, 1, seed=3)
    y = r.astype(np.float64) - d[:, 0].astype(np.float64)
    rho = len(y) / np.sum(y * y)
    t1 = O.em_step(r, d, 1, {"rho": 0.37, "K": np.zeros(0), "Linv": np.zeros((0, 0))})
    assert t1["rho"] == pytest.approx(rho, rel=1e-12)
    ll = O.em_loglik(r, d, 1, t1)
    assert ll == pytest.approx(-0.5 * len(y) * (np.log(2 * np.pi) - np.log(rho) + 1.0), rel=1e-12)
    res = O.em_fit(r, d, 1, {"rho": 0.37, "K": np.zeros(0), "Linv": np.zeros((0, 0))}, tol=1e-15, max_iter=5)
    assert res["converged"] and res["rho"] == pytest.approx(rho, rel=1e-12)


def test_em_marginal_matches_quadrature():
    """S = 2: ln of the integral over beta of N(r | D beta + mu, 1/rho) N(beta | K, 1/Lambda),
    by adaptive quadrature, observation by observation."""
    r, d, _ = synth.generate(6, 2, seed=5, alpha=0.5)
    theta = {"rho": 37.0, "K": np.array([0.31]), "Linv": np.array([[0.02]])}
    for i in range(6):
        D = float(d[i, 0]) - float(d[i, 1])
        mu = float(d[i, 1])
        s_b = np.sqrt(theta["Linv"][0, 0])

        def f(b):
            return (np.sqrt(theta["rho"] / (2 * np.pi)) * np.exp(-0.5 * theta["rho"] * (float(r[i]) - D * b - mu) ** 2)
                    * np.exp(-0.5 * (b - theta["K"][0]) ** 2 / s_b ** 2) / (s_b * np.sqrt(2 * np.pi)))
        val, _ = integrate.quad(f, theta["K"][0] - 12 * s_b, theta["K"][0] + 12 * s_b, epsabs=0, epsrel=1e-13,
                                limit=400)
        ll = O.em_loglik(r[i:i + 1], d[i:i + 1], 2, theta)
        assert ll == pytest.approx(np.log(val), abs=1e-9)


def _grad_scaled(r, d, S, th):
    """Finite-difference derivatives of ln p(r | theta), each times the size of
    its parameter: rho, every K_j, every symmetric pair of Lambda^{-1}."""
    out = []
    h = 1e-4 * th["rho"]
    tp, tm = dict(th, rho=th["rho"] + h), dict(th, rho=th["rho"] - h)
    out.append((O.em_loglik(r, d, S, tp) - O.em_loglik(r, d, S, tm)) / (2 * h) * th["rho"])
    M = S - 1
    for j in range(M):
        e = np.zeros(M)
        e[j] = 1e-5
        tp, tm = dict(th, K=th["K"] + e), dict(th, K=th["K"] - e)
        out.append((O.em_loglik(r, d, S, tp) - O.em_loglik(r, d, S, tm)) / 2e-5 * 0.1)
    scale = float(np.mean(np.diag(th["Linv"])))
    for j in range(M):
        for k in range(j + 1):
            E = np.zeros((M, M))
            E[j, k] = E[k, j] = 1e-4 * scale
            tp, tm = dict(th, Linv=th["Linv"] + E), dict(th, Linv=th["Linv"] - E)
            out.append((O.em_loglik(r, d, S, tp) - O.em_loglik(r, d, S, tm)) / (2e-4 * scale) * scale)
    return np.array(out)


@pytest.mark.parametrize("S,seed", [(2, 11), (3, 12)])
def test_em_fixed_point_is_stationary(S, seed):
    """(Data sets on which EM reaches its fixed point in a few thousand steps;
    where a variance component of Lambda^{-1} heads for zero EM creeps.)"""
    V = 2000
    r, d, _ = synth.generate(V, S, seed=seed, alpha=0.5)
    res = O.em_fit(r, d, S, O.em_init(O.paper_prior(S)), tol=1e-14, max_iter=20000)
    assert res["converged"]
    th = {"rho": res["rho"], "K": res["K"], "Linv": res["Linv"]}
    g = _grad_scaled(r, d, S, th)
    assert np.max(np.abs(g)) < 1e-5 * V, g
    # control: a point off the fixed point has a clearly non-zero gradient
    off = dict(th, K=th["K"] + 0.02)
    assert np.max(np.abs(_grad_scaled(r, d, S, off))) > 1e-2 * V
