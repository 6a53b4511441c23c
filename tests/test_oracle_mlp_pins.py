"""Pins of the FP64 set-encoder oracle (learned warm start): gradients against
central finite differences, GELU against the normal CDF, the set properties
of mean pooling, and BF16 rounding against PyTorch's conversion."""
import numpy as np
import pytest
import torch
from scipy.stats import norm

from oracle import mlp_oracle as MO


def _net(F=4, H=5, P=3, seed=0):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, 0.6, MO.num_params(F, H, P)), F, H, P


def test_gradient_matches_finite_differences():
    theta, F, H, P = _net()
    rng = np.random.default_rng(1)
    X = rng.normal(size=(3, 4, F))
    T = rng.normal(size=(3, P))
    loss, g = MO.loss_and_grad(theta, X, T, F, H, P)
    assert loss == pytest.approx(np.mean((MO.forward(theta, X, F, H, P) - T) ** 2), rel=1e-14)
    h = 1e-6
    num = np.empty_like(theta)
    for j in range(theta.size):
        e = np.zeros_like(theta)
        e[j] = h
        num[j] = (MO.loss_and_grad(theta + e, X, T, F, H, P)[0] - MO.loss_and_grad(theta - e, X, T, F, H, P)[0]) / (2 * h)
    assert np.max(np.abs(num - g)) <= 1e-7 * max(1.0, np.max(np.abs(g)))
    # control: a wrong sign in one block would be caught
    assert np.max(np.abs(num + g)) > 1e-3


def test_gelu_is_z_times_normal_cdf():
    z = np.linspace(-6, 6, 97)
    assert np.allclose(MO.gelu(z), z * norm.cdf(z), rtol=1e-14, atol=1e-300)
    assert MO.gelu(np.array([1.0]))[0] == pytest.approx(0.8413447460685429, rel=1e-15)
    h = 1e-6
    assert np.allclose(MO.gelu_grad(z), (MO.gelu(z + h) - MO.gelu(z - h)) / (2 * h), atol=1e-8)
    assert MO.gelu_grad(np.array([0.0]))[0] == 0.5


def test_set_encoder_is_permutation_invariant_and_size_free():
    theta, F, H, P = _net(seed=2)
    rng = np.random.default_rng(3)
    X = rng.normal(size=(2, 6, F))
    out = MO.forward(theta, X, F, H, P)
    perm = rng.permutation(6)
    assert np.allclose(MO.forward(theta, X[:, perm], F, H, P), out, rtol=1e-13)
    assert np.allclose(MO.forward(theta, np.concatenate([X, X], axis=1), F, H, P), out, rtol=1e-13)


def test_bf16_rounding_matches_torch():
    x = np.random.default_rng(4).normal(0, 3, 10000).astype(np.float32)
    x[:4] = [0.0, -0.0, 1.0, 3.0e38]
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(MO.bf16_round(x), ref)
