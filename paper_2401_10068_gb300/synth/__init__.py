"""Seeded synthetic inputs shaped like the paper's workloads (Section 4).

This module holds no arithmetic of the variational method: it only draws data
from the generative model of Eq. 3-4 (profiles d_i, weights beta_i, noise),
and both the CUDA path (tests, bench) and the CPU oracle (tests) consume the
arrays it returns.  It has a host implementation (numpy, here) and a device
implementation (``synth.cu``, library ``libvbh_synth.so``) of the same
counter-based recipe, so that any prefix of a data set can be regenerated.

Recipe for observation i (global index, 64-bit) of a data set keyed by a
64-bit seed; Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11) with key
(seed low word, seed high word) and counter (i low word, i high word, b, 0):

  block b = 0: x0 -> profile bits, d_{i,j} = bit j of x0 (j < S);
               x1 -> constant-profile selector: if (x1 + 1/2) 2^-32 < p_const
               the profile is constant, all zeros if bit 0 of x2 is 0, else
               all ones (D_i = 0: an uninformative measurement).
  blocks b >= 1: four uniforms u = (x + 1/2) 2^-32 each, two Box-Muller pairs
               (R = sqrt(-2 ln u1), z = R cos(2 pi u2), z' = R sin(2 pi u2));
               normal number k comes from block 1 + k // 4.
  z_0..z_{M-1} -> beta_i = K_true + L z (L the Cholesky factor of Sigma_beta)
  z_M          -> noise e_i = z_M / sqrt(rho)
  r_i = sum_j (d_{i,j} - d_{i,S}) beta_{i,j} + d_{i,S} + e_i     (Eq. 3, in FP64)

r is returned as float32 (rounded once), d as float32 (exactly 0 or 1).

The truth: Sigma_beta = 0.005 * 1 1^T + diag(0.005, 0.003, 0.005, ...), which
at S = 3 is the paper's [[0.01, 0.005], [0.005, 0.008]] (Section 4); rho = 100
(Section 4); K_true = the first S - 1 entries of a Dirichlet(alpha 1_S) draw
(Section 4 draws the Table 1 cases from Dirichlet(1, 1, 1)) unless given.
"""
from __future__ import annotations

import numpy as np

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32 with 10 rounds.  Counters are uint32 arrays (or
    scalars), the key two uint32 scalars.  Returns four uint32 arrays."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _MASK for c in (c0, c1, c2, c3))
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    m0, m1 = np.uint64(PHILOX_M0), np.uint64(PHILOX_M1)
    for rnd in range(10):
        if rnd:
            k0 = np.uint64((int(k0) + PHILOX_W0) & 0xFFFFFFFF)
            k1 = np.uint64((int(k1) + PHILOX_W1) & 0xFFFFFFFF)
        p0 = m0 * c0
        p1 = m1 * c2
        c0, c1, c2, c3 = ((p1 >> np.uint64(32)) ^ c1 ^ k0, p1 & _MASK,
                          (p0 >> np.uint64(32)) ^ c3 ^ k1, p0 & _MASK)
    return tuple(x.astype(np.uint32) for x in (c0, c1, c2, c3))


def truth_covariance(M: int) -> np.ndarray:
    diag = np.array([0.005 if j % 2 == 0 else 0.003 for j in range(M)], dtype=np.float64)
    return 0.005 * np.ones((M, M)) + np.diag(diag)


def make_truth(S: int, seed: int, alpha: float = 1.0, K_true=None, rho: float = 100.0) -> dict:
    """Ground truth of a synthetic data set (Section 4)."""
    M = S - 1
    if K_true is None:
        rng = np.random.Generator(np.random.Philox(key=int(seed) & ((1 << 64) - 1)))
        K_true = rng.dirichlet(np.full(S, float(alpha)))[:M]
    K_true = np.asarray(K_true, dtype=np.float64).reshape(M)
    Sb = truth_covariance(M)
    L = np.linalg.cholesky(Sb) if M > 0 else np.zeros((0, 0))
    return {"S": S, "K_true": K_true, "rho": float(rho), "Sigma_beta": Sb, "L_beta": L,
            "weights": np.append(K_true, 1.0 - K_true.sum())}


def _uniform(x):
    return (x.astype(np.float64) + 0.5) * (2.0 ** -32)


def generate(V: int, S: int, seed: int, alpha: float = 1.0, rho: float = 100.0, p_const: float = 0.0,
             K_true=None, start: int = 0, chunk: int = 1 << 20):
    """Host implementation.  Returns (r float32[V], d float32[V, S], truth)."""
    if not 1 <= S <= 32:
        raise ValueError("S must be in 1..32")
    M = S - 1
    truth = make_truth(S, seed, alpha, K_true, rho)
    K, L = truth["K_true"], truth["L_beta"]
    k0, k1 = int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF
    r = np.empty(V, dtype=np.float32)
    d = np.empty((V, S), dtype=np.float32)
    isr = 1.0 / np.sqrt(rho)
    nblk = (S + 3) // 4
    for s0 in range(0, V, chunk):
        n = min(chunk, V - s0)
        idx = np.arange(start + s0, start + s0 + n, dtype=np.uint64)
        lo = (idx & _MASK).astype(np.uint32)
        hi = (idx >> np.uint64(32)).astype(np.uint32)
        zero = np.zeros(n, dtype=np.uint32)
        x0, x1, x2, _ = philox4x32_10(lo, hi, zero, zero, k0, k1)
        bits = ((x0[:, None] >> np.arange(S, dtype=np.uint32)[None, :]) & 1).astype(np.float64)
        const = _uniform(x1) < p_const
        cval = (x2 & 1).astype(np.float64)
        bits[const] = cval[const][:, None]
        z = np.empty((n, 4 * nblk))
        for b in range(nblk):
            y0, y1, y2, y3 = philox4x32_10(lo, hi, np.full(n, b + 1, dtype=np.uint32), zero, k0, k1)
            for h, (ua, ub) in enumerate(((y0, y1), (y2, y3))):
                R = np.sqrt(-2.0 * np.log(_uniform(ua)))
                t = 2.0 * np.pi * _uniform(ub)
                z[:, 4 * b + 2 * h] = R * np.cos(t)
                z[:, 4 * b + 2 * h + 1] = R * np.sin(t)
        dS = bits[:, M]
        acc = np.zeros(n)
        for j in range(M):              # sequential sums: the device kernel uses the same order
            bj = np.full(n, K[j])
            for k in range(j + 1):
                bj = bj + L[j, k] * z[:, k]
            acc = acc + (bits[:, j] - dS) * bj
        rr = (acc + dS) + z[:, M] * isr
        r[s0:s0 + n] = rr.astype(np.float32)
        d[s0:s0 + n] = bits.astype(np.float32)
    return r, d, truth


def generate_device(V: int, S: int, seed: int, alpha: float = 1.0, rho: float = 100.0, p_const: float = 0.0,
                    K_true=None, start: int = 0, device="cuda"):
    """Device implementation of the same recipe (``libvbh_synth.so``); returns
    torch tensors (r [V] float32, d [V, S] float32 row-major) and the truth."""
    import torch
    from . import _device
    truth = make_truth(S, seed, alpha, K_true, rho)
    r = torch.empty(V, dtype=torch.float32, device=device)
    d = torch.empty((V, S), dtype=torch.float32, device=device)
    _device.generate(r, d, V, S, start, seed, truth, p_const)
    return r, d, truth
