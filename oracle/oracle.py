"""Python binding of the FP64 CPU oracle in ``vbh_oracle.c``.

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
cpu_baseline / reference legs of ``bench.py`` may import this module.  It never
imports the CUDA package and the CUDA package never imports it.

The C library is compiled on first use with plain ``gcc -O2`` (no fast-math, no
FMA contraction, no architecture flags), so it gives the same results on x86-64
and aarch64 hosts.  Every function here only marshals numpy arrays; the
arithmetic is in the C file, whose functions cite the equations they follow.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

MMAX = 31
SMAX = MMAX + 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vbh_oracle.c")
_LIB = os.path.join(_HERE, "libvbh_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``vbh_oracle.c`` into ``libvbh_oracle.so`` next to it."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                                   _SRC, "-lm", "-o", tmp])
            os.replace(tmp, _LIB)
    return _LIB


class _Prior(ctypes.Structure):
    _fields_ = [("S", ctypes.c_int), ("K0", ctypes.c_double * MMAX), ("q0", ctypes.c_double),
                ("n0", ctypes.c_double), ("a0", ctypes.c_double), ("b0", ctypes.c_double),
                ("L0inv", ctypes.c_double * (MMAX * MMAX))]


class _Glob(ctypes.Structure):
    _fields_ = [("a_rho", ctypes.c_double), ("b_rho", ctypes.c_double), ("nu", ctypes.c_double),
                ("lam", ctypes.c_double), ("kappa", ctypes.c_double * MMAX),
                ("Winv", ctypes.c_double * (MMAX * MMAX))]


class _EM(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double), ("K", ctypes.c_double * MMAX), ("Linv", ctypes.c_double * (MMAX * MMAX))]


class _Sums(ctypes.Structure):
    _fields_ = [("V", ctypes.c_double), ("sum_S", ctypes.c_double), ("sum_mu", ctypes.c_double * MMAX),
                ("sum_Ebb", ctypes.c_double * (MMAX * MMAX)), ("sum_logdet", ctypes.c_double)]


_P = ctypes.POINTER
_dp = _P(ctypes.c_double)
_fp = _P(ctypes.c_float)


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, ci = ctypes.c_int64, ctypes.c_int
        sig = {
            "vbo_digamma": (ctypes.c_double, [ctypes.c_double]),
            "vbo_beta_init": (None, [_P(_Prior), i64, _dp, _dp]),
            "vbo_beta_update": (ci, [_P(_Prior), i64, _fp, _fp, _P(_Glob), _dp, _dp]),
            "vbo_sums_from_beta": (ci, [_P(_Prior), i64, _fp, _fp, _dp, _dp, _P(_Sums)]),
            "vbo_rho_update": (None, [_P(_Prior), _P(_Sums), _P(_Glob)]),
            "vbo_KLambda_update": (None, [_P(_Prior), _P(_Sums), _P(_Glob)]),
            "vbo_elbo": (ci, [_P(_Prior), _P(_Sums), _P(_Glob), _dp, _P(ci)]),
            "vbo_fit": (ci, [_P(_Prior), i64, _fp, _fp, ctypes.c_double, ci, _P(_Glob), _dp, _P(ci), _P(ci),
                             _dp, _P(ci)]),
            "vbo_sums_grouped": (ci, [_P(_Prior), ci, _dp, _dp, _dp, _dp, _P(_Glob), ci, _P(_Sums)]),
            "vbo_fit_grouped": (ci, [_P(_Prior), ci, _dp, _dp, _dp, _dp, ctypes.c_double, ci, _P(_Glob), _dp,
                                     _P(ci), _P(ci), _dp, _P(ci)]),
            "vbo_elbo_at": (ci, [_P(_Prior), i64, _fp, _fp, _P(_Glob), _dp, _P(ci)]),
            "vbo_em_loglik": (ci, [ci, i64, _fp, _fp, _P(_EM), _dp]),
            "vbo_em_step": (ci, [ci, i64, _fp, _fp, _P(_EM), _P(_EM)]),
            "vbo_em_fit": (ci, [ci, i64, _fp, _fp, _P(_EM), ctypes.c_double, ci, _P(_EM), _dp, _P(ci), _P(ci)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


# --------------------------------------------------------------------------- #
# Prior constants (Section 3.5) generalised from S = 3 to any S.              #
# --------------------------------------------------------------------------- #
def paper_covariance(M: int) -> np.ndarray:
    """0.005 * 1 1^T + diag(0.005, 0.003, 0.005, 0.003, ...): equals the
    paper's [[0.01, 0.005], [0.005, 0.008]] (Section 3.5 and Section 4) at M = 2
    and is positive definite for every M."""
    diag = np.array([0.005 if j % 2 == 0 else 0.003 for j in range(M)], dtype=np.float64)
    return 0.005 * np.ones((M, M)) + np.diag(diag)


def paper_prior(S: int, **overrides) -> dict:
    """The paper's prior constants (Section 3.5): K0 = (1/S, ...), a0 = b0 = 0.5,
    q0 = 0.001, n0 = 1 and Lambda_0^{-1} = paper_covariance(S - 1)."""
    M = S - 1
    p = {"S": S, "K0": np.full(M, 1.0 / S), "q0": 1e-3, "n0": 1.0, "a0": 0.5, "b0": 0.5,
         "L0inv": paper_covariance(M)}
    p.update(overrides)
    p["K0"] = np.asarray(p["K0"], dtype=np.float64).reshape(M)
    p["L0inv"] = np.asarray(p["L0inv"], dtype=np.float64).reshape(M, M)
    return p


def _prior(p: dict) -> _Prior:
    S = int(p["S"])
    if not 1 <= S <= SMAX:
        raise ValueError("S must be in 1..32")
    M = S - 1
    c = _Prior()
    c.S = S
    c.q0, c.n0, c.a0, c.b0 = float(p["q0"]), float(p["n0"]), float(p["a0"]), float(p["b0"])
    K0 = np.asarray(p["K0"], dtype=np.float64).reshape(M)
    L0 = np.asarray(p["L0inv"], dtype=np.float64).reshape(M * M)
    for j in range(M):
        c.K0[j] = K0[j]
    for j in range(M * M):
        c.L0inv[j] = L0[j]
    return c


def _glob_to_c(g: dict, M: int) -> _Glob:
    c = _Glob()
    c.a_rho, c.b_rho, c.nu, c.lam = float(g["a_rho"]), float(g["b_rho"]), float(g["nu"]), float(g["lam"])
    k = np.asarray(g["kappa"], dtype=np.float64).reshape(M)
    W = np.asarray(g["Winv"], dtype=np.float64).reshape(M * M)
    for j in range(M):
        c.kappa[j] = k[j]
    for j in range(M * M):
        c.Winv[j] = W[j]
    return c


def _glob_from_c(c: _Glob, M: int) -> dict:
    return {"a_rho": c.a_rho, "b_rho": c.b_rho, "nu": c.nu, "lam": c.lam,
            "kappa": np.array(c.kappa[:M]), "Winv": np.array(c.Winv[:M * M]).reshape(M, M)}


def _sums_from_c(c: _Sums, M: int) -> dict:
    return {"V": c.V, "sum_S": c.sum_S, "sum_mu": np.array(c.sum_mu[:M]),
            "sum_Ebb": np.array(c.sum_Ebb[:M * M]).reshape(M, M), "sum_logdet": c.sum_logdet}


def _sums_to_c(s: dict, M: int) -> _Sums:
    c = _Sums()
    c.V, c.sum_S, c.sum_logdet = float(s["V"]), float(s["sum_S"]), float(s["sum_logdet"])
    mu = np.asarray(s["sum_mu"], dtype=np.float64).reshape(M)
    E = np.asarray(s["sum_Ebb"], dtype=np.float64).reshape(M * M)
    for j in range(M):
        c.sum_mu[j] = mu[j]
    for j in range(M * M):
        c.sum_Ebb[j] = E[j]
    return c


def _f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(_fp)


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


# --------------------------------------------------------------------------- #
# Public functions                                                            #
# --------------------------------------------------------------------------- #
def digamma(x: float) -> float:
    return _load().vbo_digamma(float(x))


def fit(r, d, prior: dict, tol: float = 1e-8, max_iter: int = 200) -> dict:
    """Sweep 0 plus up to ``max_iter`` CAVI sweeps (Section 3.5 schedule)."""
    lib = _load()
    S = int(prior["S"])
    r, rp = _f32(r)
    d, dp = _f32(d)
    V = r.shape[0]
    if d.size != V * S:
        raise ValueError("d must hold V*S values")
    pc, gc = _prior(prior), _Glob()
    trace = np.zeros(max_iter + 1)
    iters, conv, dropped = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    elbo = ctypes.c_double()
    rc = lib.vbo_fit(ctypes.byref(pc), V, rp, dp, float(tol), int(max_iter), ctypes.byref(gc),
                     trace.ctypes.data_as(_dp), ctypes.byref(iters), ctypes.byref(conv), ctypes.byref(elbo),
                     ctypes.byref(dropped))
    _check(rc, "fit")
    out = _glob_from_c(gc, S - 1)
    out.update(iters=iters.value, converged=bool(conv.value), elbo=elbo.value,
               trace=trace[:iters.value + 1].copy(), const_dropped=bool(dropped.value))
    return out


def fit_grouped(groups: dict, prior: dict, tol: float = 1e-8, max_iter: int = 200) -> dict:
    """``fit`` on profile-grouped data: ``groups`` holds ``dprof`` (P x S), ``n``,
    ``sy`` = sum of (r - d_S) and ``syy`` = sum of (r - d_S)^2 per profile."""
    lib = _load()
    S = int(prior["S"])
    dprof, dpp = _f64(groups["dprof"])
    n, np_ = _f64(groups["n"])
    sy, syp = _f64(groups["sy"])
    syy, syyp = _f64(groups["syy"])
    P = n.shape[0]
    pc, gc = _prior(prior), _Glob()
    trace = np.zeros(max_iter + 1)
    iters, conv, dropped = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    elbo = ctypes.c_double()
    rc = lib.vbo_fit_grouped(ctypes.byref(pc), P, dpp, np_, syp, syyp, float(tol), int(max_iter),
                             ctypes.byref(gc), trace.ctypes.data_as(_dp), ctypes.byref(iters), ctypes.byref(conv),
                             ctypes.byref(elbo), ctypes.byref(dropped))
    _check(rc, "fit_grouped")
    out = _glob_from_c(gc, S - 1)
    out.update(iters=iters.value, converged=bool(conv.value), elbo=elbo.value,
               trace=trace[:iters.value + 1].copy(), const_dropped=bool(dropped.value))
    return out


def beta_init(prior: dict, V: int):
    lib = _load()
    M = int(prior["S"]) - 1
    mu = np.zeros((V, M))
    Sig = np.zeros((V, M, M))
    lib.vbo_beta_init(ctypes.byref(_prior(prior)), V, mu.ctypes.data_as(_dp), Sig.ctypes.data_as(_dp))
    return mu, Sig


def beta_update(r, d, prior: dict, glob: dict):
    lib = _load()
    M = int(prior["S"]) - 1
    r, rp = _f32(r)
    d, dp = _f32(d)
    V = r.shape[0]
    mu = np.zeros((V, M))
    Sig = np.zeros((V, M, M))
    g = _glob_to_c(glob, M)
    _check(lib.vbo_beta_update(ctypes.byref(_prior(prior)), V, rp, dp, ctypes.byref(g),
                               mu.ctypes.data_as(_dp), Sig.ctypes.data_as(_dp)), "beta_update")
    return mu, Sig


def sums_from_beta(r, d, prior: dict, mu, Sig) -> dict:
    lib = _load()
    M = int(prior["S"]) - 1
    r, rp = _f32(r)
    d, dp = _f32(d)
    mu, mup = _f64(mu)
    Sig, Sp = _f64(Sig)
    s = _Sums()
    _check(lib.vbo_sums_from_beta(ctypes.byref(_prior(prior)), r.shape[0], rp, dp, mup, Sp, ctypes.byref(s)),
           "sums_from_beta")
    return _sums_from_c(s, M)


def sums_grouped(groups: dict, prior: dict, glob: dict | None, init: bool = False) -> dict:
    lib = _load()
    M = int(prior["S"]) - 1
    dprof, dpp = _f64(groups["dprof"])
    n, np_ = _f64(groups["n"])
    sy, syp = _f64(groups["sy"])
    syy, syyp = _f64(groups["syy"])
    g = _glob_to_c(glob, M) if glob is not None else _Glob()
    s = _Sums()
    _check(lib.vbo_sums_grouped(ctypes.byref(_prior(prior)), n.shape[0], dpp, np_, syp, syyp, ctypes.byref(g),
                                int(bool(init)), ctypes.byref(s)), "sums_grouped")
    return _sums_from_c(s, M)


def rho_update(prior: dict, sums: dict, glob: dict | None = None) -> dict:
    lib = _load()
    M = int(prior["S"]) - 1
    g = _glob_to_c(glob, M) if glob is not None else _Glob()
    lib.vbo_rho_update(ctypes.byref(_prior(prior)), ctypes.byref(_sums_to_c(sums, M)), ctypes.byref(g))
    return _glob_from_c(g, M)


def KLambda_update(prior: dict, sums: dict, glob: dict | None = None) -> dict:
    lib = _load()
    M = int(prior["S"]) - 1
    g = _glob_to_c(glob, M) if glob is not None else _Glob()
    lib.vbo_KLambda_update(ctypes.byref(_prior(prior)), ctypes.byref(_sums_to_c(sums, M)), ctypes.byref(g))
    return _glob_from_c(g, M)


def elbo(prior: dict, sums: dict, glob: dict):
    """Returns (ELBO, const_dropped)."""
    lib = _load()
    M = int(prior["S"]) - 1
    out, dropped = ctypes.c_double(), ctypes.c_int()
    _check(lib.vbo_elbo(ctypes.byref(_prior(prior)), ctypes.byref(_sums_to_c(sums, M)),
                        ctypes.byref(_glob_to_c(glob, M)), ctypes.byref(out), ctypes.byref(dropped)), "elbo")
    return out.value, bool(dropped.value)


def elbo_at(r, d, prior: dict, glob: dict):
    """ELBO of the given global factors with Q(beta) from one Eq. 20-21 update."""
    lib = _load()
    M = int(prior["S"]) - 1
    r, rp = _f32(r)
    d, dp = _f32(d)
    out, dropped = ctypes.c_double(), ctypes.c_int()
    _check(lib.vbo_elbo_at(ctypes.byref(_prior(prior)), r.shape[0], rp, dp, ctypes.byref(_glob_to_c(glob, M)),
                           ctypes.byref(out), ctypes.byref(dropped)), "elbo_at")
    return out.value, bool(dropped.value)


def group_profiles(r, d, S: int) -> dict:
    """Per-profile counts and sums of y = r - d_S for binary profiles d (test
    helper for the profile-grouped form).  Works in chunks, FP64 sums."""
    r = np.asarray(r)
    d = np.asarray(d).reshape(-1, S)
    V = r.shape[0]
    P = 1 << S
    n = np.zeros(P)
    sy = np.zeros(P)
    syy = np.zeros(P)
    w = (1 << np.arange(S, dtype=np.int64))
    chunk = 1 << 22
    for s0 in range(0, V, chunk):
        dc = d[s0:s0 + chunk]
        bits = dc > 0.5
        if not np.all(bits == (dc != 0)) or not np.all((dc == 0) | (dc == 1)):
            raise ValueError("group_profiles needs binary profiles")
        code = bits.astype(np.int64) @ w
        y = r[s0:s0 + chunk].astype(np.float64) - dc[:, S - 1].astype(np.float64)
        n += np.bincount(code, minlength=P)
        sy += np.bincount(code, weights=y, minlength=P)
        syy += np.bincount(code, weights=y * y, minlength=P)
    keep = n > 0
    codes = np.nonzero(keep)[0]
    dprof = ((codes[:, None] >> np.arange(S)[None, :]) & 1).astype(np.float64)
    return {"dprof": dprof, "n": n[keep], "sy": sy[keep], "syy": syy[keep]}


# --------------------------------------------------------------------------- #
# Expectation maximisation (Section 4.2, Eq. 42-47).                          #
# --------------------------------------------------------------------------- #
def em_init(prior: dict) -> dict:
    """theta^(0) from the prior constants: K = K0, Lambda^{-1} = Lambda_0^{-1},
    rho = a0 / b0 (the paper gives no starting point; this is the reading the
    CUDA path uses too)."""
    M = int(prior["S"]) - 1
    return {"rho": float(prior["a0"]) / float(prior["b0"]), "K": np.array(prior["K0"], dtype=np.float64).reshape(M),
            "Linv": np.array(prior["L0inv"], dtype=np.float64).reshape(M, M)}


def _em_to_c(t: dict, M: int) -> _EM:
    c = _EM()
    c.rho = float(t["rho"])
    K = np.asarray(t["K"], dtype=np.float64).reshape(M)
    L = np.asarray(t["Linv"], dtype=np.float64).reshape(M * M)
    for j in range(M):
        c.K[j] = K[j]
    for j in range(M * M):
        c.Linv[j] = L[j]
    return c


def _em_from_c(c: _EM, M: int) -> dict:
    return {"rho": c.rho, "K": np.array(c.K[:M]), "Linv": np.array(c.Linv[:M * M]).reshape(M, M)}


def em_loglik(r, d, S: int, theta: dict) -> float:
    """ln p(r | theta): the marginal of Eq. 3 under Eq. 4."""
    lib = _load()
    r, rp = _f32(r)
    d, dp = _f32(d)
    out = ctypes.c_double()
    _check(lib.vbo_em_loglik(int(S), r.shape[0], rp, dp, ctypes.byref(_em_to_c(theta, S - 1)), ctypes.byref(out)),
           "em_loglik")
    return out.value


def em_step(r, d, S: int, theta: dict) -> dict:
    """One EM iteration (Eq. 42-47)."""
    lib = _load()
    r, rp = _f32(r)
    d, dp = _f32(d)
    o = _EM()
    _check(lib.vbo_em_step(int(S), r.shape[0], rp, dp, ctypes.byref(_em_to_c(theta, S - 1)), ctypes.byref(o)),
           "em_step")
    return _em_from_c(o, S - 1)


def em_fit(r, d, S: int, theta0: dict, tol: float = 1e-8, max_iter: int = 200) -> dict:
    """EM from theta0: trace[n] = ln p(r | theta^(n)), n = 0..iters; the result
    holds theta^(iters + 1)."""
    lib = _load()
    r, rp = _f32(r)
    d, dp = _f32(d)
    o = _EM()
    trace = np.zeros(max_iter + 1)
    iters, conv = ctypes.c_int(), ctypes.c_int()
    rc = lib.vbo_em_fit(int(S), r.shape[0], rp, dp, ctypes.byref(_em_to_c(theta0, S - 1)), float(tol), int(max_iter),
                        ctypes.byref(o), trace.ctypes.data_as(_dp), ctypes.byref(iters), ctypes.byref(conv))
    _check(rc, "em_fit")
    out = _em_from_c(o, S - 1)
    out.update(iters=iters.value, converged=bool(conv.value), trace=trace[:iters.value + 1].copy(),
               loglik=float(trace[iters.value]))
    return out
