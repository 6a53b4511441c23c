"""Pins of the FP64 set-encoder oracle (learned warm start): gradients against
central finite differences (a small network of the same structure), the tanh
form of GELU against its closed form, the exact GELU and its own finite
differences, the set properties of mean pooling, the feature slots against a
hand-written example, the loss weights as masks, and BF16 rounding against
PyTorch's conversion."""
import math

import numpy as np
import pytest
import torch
from scipy.stats import norm

from oracle import mlp_oracle as MO


@pytest.fixture
def small(monkeypatch):
    """A network of the oracle's structure with F = 5, H = 6, P = 4, so that
    finite differences over every parameter stay cheap."""
    monkeypatch.setattr(MO, "F", 5)
    monkeypatch.setattr(MO, "H", 6)
    monkeypatch.setattr(MO, "P", 4)
    orig = (MO.shapes, MO.num_params, MO.unpack, MO.pack)
    monkeypatch.setattr(MO, "shapes", lambda F=5, H=6, P=4: orig[0](F, H, P))
    monkeypatch.setattr(MO, "num_params", lambda F=5, H=6, P=4: orig[1](F, H, P))
    monkeypatch.setattr(MO, "unpack", lambda th, F=5, H=6, P=4: orig[2](th, F, H, P))
    monkeypatch.setattr(MO, "pack", lambda parts, F=5, H=6, P=4: orig[3](parts, F, H, P))
    rng = np.random.default_rng(0)
    return rng.normal(0.0, 0.6, MO.num_params())


def test_gradient_matches_finite_differences(small):
    theta = small
    rng = np.random.default_rng(1)
    Xs = [rng.normal(size=(n, 5)) for n in (3, 5, 2)]           # sets of different sizes
    T = rng.normal(size=(3, 4))
    Wt = (rng.uniform(size=(3, 4)) > 0.3).astype(float)           # some slots masked
    loss, g = MO.loss_and_grad(theta, Xs, T, Wt)
    out = MO.forward(theta, Xs)
    assert loss == pytest.approx(np.sum(Wt * (out - T) ** 2) / 3, rel=1e-14)
    h = 1e-6
    num = np.empty_like(theta)
    for j in range(theta.size):
        e = np.zeros_like(theta)
        e[j] = h
        num[j] = (MO.loss_and_grad(theta + e, Xs, T, Wt)[0] - MO.loss_and_grad(theta - e, Xs, T, Wt)[0]) / (2 * h)
    assert np.max(np.abs(num - g)) <= 1e-7 * max(1.0, np.max(np.abs(g)))
    assert np.max(np.abs(num + g)) > 1e-3                        # control: a wrong sign would be caught


def test_masked_slots_carry_no_gradient(small):
    theta = small
    rng = np.random.default_rng(2)
    Xs = [rng.normal(size=(4, 5))]
    T = rng.normal(size=(1, 4))
    Wt = np.array([[1.0, 1.0, 0.0, 0.0]])
    _, g = MO.loss_and_grad(theta, Xs, T, Wt)
    T2 = T.copy()
    T2[0, 2:] += 5.0                                             # changing masked targets changes nothing
    _, g2 = MO.loss_and_grad(theta, Xs, T2, Wt)
    assert np.array_equal(g, g2)
    w = MO.unpack(g)
    assert np.all(w["W4"][2:] == 0.0) and np.all(w["b4"][2:] == 0.0)


def test_gelu_tanh_form():
    z = np.linspace(-6, 6, 97)
    t = np.tanh(math.sqrt(2 / math.pi) * (z + 0.044715 * z ** 3))
    assert np.allclose(MO.gelu(z), 0.5 * z * (1 + t), rtol=1e-15, atol=0)
    # the tanh form stays within 2e-3 of the exact z Phi(z) (Hendrycks and Gimpel, 2016)
    assert np.max(np.abs(MO.gelu(z) - z * norm.cdf(z))) < 2e-3
    assert MO.gelu(np.array([0.0]))[0] == 0.0
    h = 1e-6
    assert np.allclose(MO.gelu_grad(z), (MO.gelu(z + h) - MO.gelu(z - h)) / (2 * h), atol=1e-8)
    assert MO.gelu_grad(np.array([0.0]))[0] == 0.5


def test_set_encoder_is_permutation_invariant_and_size_free(small):
    theta = small
    rng = np.random.default_rng(3)
    X = rng.normal(size=(6, 5))
    out = MO.forward(theta, [X])
    perm = rng.permutation(6)
    assert np.allclose(MO.forward(theta, [X[perm]]), out, rtol=1e-13)
    assert np.allclose(MO.forward(theta, [np.concatenate([X, X])]), out, rtol=1e-13)


def test_feature_slots_of_a_worked_example():
    # two observations, S = 3 (M = 2): d = (1, 0, 1), r = 1.5 and d = (0, 1, 0), r = -0.25
    r = np.array([1.5, -0.25], dtype=np.float32)
    d = np.array([[1, 0, 1], [0, 1, 0]], dtype=np.float32)
    X = MO.features(r, d, 3)
    want = np.zeros((2, 64))
    # first: D = (0, -1), y = 0.5
    want[0, [0, 1]] = [0.0, -1.0]
    want[0, [9, 10]] = 1.0
    want[0, 18], want[0, 19] = 0.5, 0.25
    want[0, [20, 21]] = [0.0, -0.5]
    want[0, [29, 30]] = [0.0, -0.25]
    # second: D = (0, 1), y = -0.25
    want[1, [0, 1]] = [0.0, 1.0]
    want[1, [9, 10]] = 1.0
    want[1, 18], want[1, 19] = -0.25, 0.0625
    want[1, [20, 21]] = [0.0, -0.25]
    want[1, [29, 30]] = [0.0, 0.0625]
    assert np.array_equal(X, want)
    assert np.array_equal(MO.pooled_index(10, 4), [0, 2, 5, 7]) and np.array_equal(MO.pooled_index(3, 0), [0, 1, 2])


def test_bf16_rounding_matches_torch():
    x = np.random.default_rng(4).normal(0, 3, 10000).astype(np.float32)
    x[:4] = [0.0, -0.0, 1.0, 3.0e38]
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(MO.bf16_round(x), ref)
