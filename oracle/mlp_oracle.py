"""FP64 CPU oracle of the learned warm start's set encoder.

TEST INFRASTRUCTURE.  Only the test suite may import this module; it shares no
code with the CUDA path.

The set encoder maps a data set (a set of observations) to a starting point
of the CAVI iteration.  Per observation i a feature vector x_i (64 slots,
``features``) goes through phi(x) = GELU(W2 GELU(W1 x + b1) + b2) (H = 256);
phi is averaged over the observations of the set, and the head
GELU(W3 p + b3) -> W4 (.) + b4 gives 64 output slots.  GELU is the tanh form
z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))) / 2 (Hendrycks and Gimpel, 2016).
Loss: sum over sets and slots of w (out - t)^2, divided by the number of sets
(w = 0 masks the slots a set with S < 10 does not use).

Parameters are one flat vector in the order W1 (H x F), b1 (H), W2 (H x H),
b2 (H), W3 (H x H), b3 (H), W4 (P x H), b4 (P), matrices row-major.

``quantized=True`` rounds, at the points where the GPU path keeps BF16
values, to BF16 (round to nearest even): the features, W1 and W2, the
layer-1 activations, the pooled gradient dZ2 and the layer-1 gradient dZ1.
Everything else is FP64.  Everything is written out step by step (forward,
then the chain rule backward), so that a reader can check it line by line.
"""
from __future__ import annotations

import math

import numpy as np

F, P, H, SMAX = 64, 64, 256, 10
K0, K1 = math.sqrt(2.0 / math.pi), 0.044715


def shapes(F: int = F, H: int = H, P: int = P):
    return [("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)), ("b3", (H,)),
            ("W4", (P, H)), ("b4", (P,))]


def num_params(F: int = F, H: int = H, P: int = P) -> int:
    return sum(int(np.prod(s)) for _, s in shapes(F, H, P))


def unpack(theta, F: int = F, H: int = H, P: int = P) -> dict:
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, s in shapes(F, H, P):
        n = int(np.prod(s))
        out[name] = theta[o:o + n].reshape(s)
        o += n
    assert o == theta.size
    return out


def pack(parts: dict, F: int = F, H: int = H, P: int = P) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).reshape(-1) for name, _ in shapes(F, H, P)])


def gelu(z):
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * z * (1.0 + np.tanh(K0 * (z + K1 * z ** 3)))


def gelu_grad(z):
    z = np.asarray(z, dtype=np.float64)
    t = np.tanh(K0 * (z + K1 * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * K0 * (1.0 + 3.0 * K1 * z * z)


def bf16_round(x):
    """Round to BF16 (round to nearest even, through FP32), returned as FP64."""
    a = np.asarray(x, dtype=np.float32).copy()
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return (u.astype(np.uint32)).view(np.float32).astype(np.float64)


def pooled_index(V: int, n: int = 0) -> np.ndarray:
    """Observations the encoder pools: all, or floor(j V / n) for j < n."""
    if n <= 0 or n >= V:
        return np.arange(V, dtype=np.int64)
    return (np.arange(n, dtype=np.int64) * V) // n


def features(r, d, S: int, idx=None) -> np.ndarray:
    """The 64 feature slots of the observations idx (FP32 arithmetic, as the
    stored inputs are FP32): D_ij (slots 0-8), the mask j < M (9-17), y (18),
    y^2 (19), y D_ij (20-28), y^2 D_ij (29-37), zeros (38-63)."""
    r = np.asarray(r, dtype=np.float32)
    d = np.asarray(d, dtype=np.float32).reshape(r.shape[0], S)
    if idx is None:
        idx = np.arange(r.shape[0])
    M = S - 1
    dS = d[idx, M]
    y = (r[idx] - dS).astype(np.float32)
    y2 = (y * y).astype(np.float32)
    X = np.zeros((idx.size, F), dtype=np.float32)
    for j in range(M):
        D = (d[idx, j] - dS).astype(np.float32)
        X[:, j] = D
        X[:, 9 + j] = 1.0
        X[:, 20 + j] = y * D
        X[:, 29 + j] = y2 * D
    X[:, 18] = y
    X[:, 19] = y2
    return X.astype(np.float64)


def _q(x, quantized):
    return bf16_round(x) if quantized else np.asarray(x, dtype=np.float64)


def _layers(theta, Xs, quantized):
    w = unpack(theta)
    W1, W2 = _q(w["W1"], quantized), _q(w["W2"], quantized)
    cache = []
    pools = []
    for X in Xs:
        X = _q(X, quantized)
        Z1 = X @ W1.T + w["b1"]
        A1 = _q(gelu(Z1), quantized)
        Z2 = A1 @ W2.T + w["b2"]
        A2 = gelu(Z2)
        pools.append(A2.mean(axis=0))
        cache.append((X, Z1, A1, Z2))
    Pool = np.stack(pools)
    Z3 = Pool @ w["W3"].T + w["b3"]
    A3 = gelu(Z3)
    Out = A3 @ w["W4"].T + w["b4"]
    return w, W1, W2, cache, Pool, Z3, A3, Out


def forward(theta, Xs, quantized: bool = False) -> np.ndarray:
    """Xs: list of (n_b, F) feature arrays, one per set -> outputs (B, P)."""
    return _layers(theta, Xs, quantized)[-1]


def loss_and_grad(theta, Xs, T, Wt, quantized: bool = False):
    """Loss sum w (out - t)^2 / B and its gradient in theta (flat)."""
    w, W1, W2, cache, Pool, Z3, A3, Out = _layers(theta, Xs, quantized)
    T = np.asarray(T, dtype=np.float64)
    Wt = np.asarray(Wt, dtype=np.float64)
    B = len(Xs)
    R = Out - T
    loss = float(np.sum(Wt * R * R) / B)
    # backward
    dOut = 2.0 * Wt * R / B
    g = {"W4": dOut.T @ A3, "b4": dOut.sum(axis=0)}
    dA3 = dOut @ w["W4"]
    dZ3 = dA3 * gelu_grad(Z3)
    g["W3"] = dZ3.T @ Pool
    g["b3"] = dZ3.sum(axis=0)
    dPool = dZ3 @ w["W3"]
    gW2 = np.zeros_like(w["W2"])
    gb2 = np.zeros_like(w["b2"])
    gW1 = np.zeros_like(w["W1"])
    gb1 = np.zeros_like(w["b1"])
    for b, (X, Z1, A1, Z2) in enumerate(cache):
        n = X.shape[0]
        dZ2 = _q(np.repeat(dPool[b][None, :] / n, n, axis=0) * gelu_grad(Z2), quantized)
        gW2 += dZ2.T @ A1
        gb2 += dZ2.sum(axis=0)
        dA1 = dZ2 @ W2
        dZ1 = _q(dA1 * gelu_grad(Z1), quantized)
        gW1 += dZ1.T @ X
        gb1 += dZ1.sum(axis=0)
    g.update(W2=gW2, b2=gb2, W1=gW1, b1=gb1)
    return loss, pack(g)
