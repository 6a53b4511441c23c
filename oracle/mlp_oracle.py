"""FP64 CPU oracle of the learned warm start's set encoder.

TEST INFRASTRUCTURE.  Only the test suite may import this module; it shares no
code with the CUDA path.

The set encoder maps a data set (a set of observations) to a starting point
of the CAVI iteration.  Per observation i a feature vector x_i in R^F goes
through phi(x) = GELU(W2 GELU(W1 x + b1) + b2); the features are mean-pooled
over the set, and the head GELU(W3 p + b3) -> W4 (.) + b4 gives the outputs.
GELU(z) = z Phi(z) with Phi the standard normal CDF (from erfc).  Loss: the mean squared
error against a target vector per set, averaged over sets and outputs.

Parameters are one flat vector in the order W1 (H x F), b1 (H), W2 (H x H),
b2 (H), W3 (H x H), b3 (H), W4 (P x H), b4 (P), matrices row-major.
Everything is FP64 and written out step by step (forward, then the chain rule
backward), so that a reader can check it line by line.
"""
from __future__ import annotations

import math

import numpy as np


def shapes(F: int, H: int, P: int):
    return [("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)), ("b3", (H,)),
            ("W4", (P, H)), ("b4", (P,))]


def num_params(F: int, H: int, P: int) -> int:
    return sum(int(np.prod(s)) for _, s in shapes(F, H, P))


def unpack(theta, F: int, H: int, P: int) -> dict:
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, s in shapes(F, H, P):
        n = int(np.prod(s))
        out[name] = theta[o:o + n].reshape(s)
        o += n
    assert o == theta.size
    return out


def pack(parts: dict, F: int, H: int, P: int) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).reshape(-1) for name, _ in shapes(F, H, P)])


_erfc = np.vectorize(math.erfc)


def _phi_cdf(z):
    # Phi(z) = erfc(-z / sqrt 2) / 2, without the cancellation of 1 + erf at negative z
    return 0.5 * _erfc(-np.asarray(z, dtype=np.float64) / math.sqrt(2.0))


def gelu(z):
    return z * _phi_cdf(z)


def gelu_grad(z):
    # d/dz [z Phi(z)] = Phi(z) + z phi(z)
    return _phi_cdf(z) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(theta, X, F: int, H: int, P: int) -> np.ndarray:
    """X: (B, n, F) -> outputs (B, P)."""
    w = unpack(theta, F, H, P)
    X = np.asarray(X, dtype=np.float64)
    Z1 = X @ w["W1"].T + w["b1"]
    A1 = gelu(Z1)
    Z2 = A1 @ w["W2"].T + w["b2"]
    A2 = gelu(Z2)
    Pool = A2.mean(axis=1)
    Z3 = Pool @ w["W3"].T + w["b3"]
    A3 = gelu(Z3)
    return A3 @ w["W4"].T + w["b4"]


def loss_and_grad(theta, X, T, F: int, H: int, P: int):
    """Mean squared error over (B, P) and its gradient in theta (flat)."""
    w = unpack(theta, F, H, P)
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    B, n, _ = X.shape
    # forward
    Z1 = X @ w["W1"].T + w["b1"]
    A1 = gelu(Z1)
    Z2 = A1 @ w["W2"].T + w["b2"]
    A2 = gelu(Z2)
    Pool = A2.mean(axis=1)
    Z3 = Pool @ w["W3"].T + w["b3"]
    A3 = gelu(Z3)
    Out = A3 @ w["W4"].T + w["b4"]
    R = Out - T
    loss = float(np.sum(R * R) / (B * P))
    # backward
    dOut = 2.0 * R / (B * P)
    g = {"W4": dOut.T @ A3, "b4": dOut.sum(axis=0)}
    dA3 = dOut @ w["W4"]
    dZ3 = dA3 * gelu_grad(Z3)
    g["W3"] = dZ3.T @ Pool
    g["b3"] = dZ3.sum(axis=0)
    dPool = dZ3 @ w["W3"]
    dA2 = np.repeat(dPool[:, None, :] / n, n, axis=1)
    dZ2 = dA2 * gelu_grad(Z2)
    g["W2"] = np.einsum("bnh,bnk->hk", dZ2, A1)
    g["b2"] = dZ2.sum(axis=(0, 1))
    dA1 = dZ2 @ w["W2"]
    dZ1 = dA1 * gelu_grad(Z1)
    g["W1"] = np.einsum("bnh,bnf->hf", dZ1, X)
    g["b1"] = dZ1.sum(axis=(0, 1))
    return loss, pack(g, F, H, P)


def bf16_round(x):
    """Round FP32 values to BF16 (round to nearest even), returned as FP64."""
    a = np.asarray(x, dtype=np.float32).copy()
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return (u.astype(np.uint32)).view(np.float32).astype(np.float64)


def weights_as_bf16(theta, F: int, H: int, P: int) -> np.ndarray:
    """The parameters as the CUDA path's forward sees them: matrices in BF16,
    biases in FP32."""
    w = unpack(theta, F, H, P)
    out = {}
    for name, _ in shapes(F, H, P):
        out[name] = bf16_round(w[name]) if name.startswith("W") else np.asarray(w[name], dtype=np.float32)
    return pack(out, F, H, P)
