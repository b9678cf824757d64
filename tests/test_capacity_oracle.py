"""Pins of the capacity-network oracle: its gradient against central finite
differences of its own loss (an independent check of the chain rule), its
parameter count and packing, and closed forms of the forward pass."""
import numpy as np
import pytest

from oracle import capacity_mlp as mlp


def test_layout():
    assert mlp.N_PARAMS == 64 * 4 + 64 + 64 * 64 + 64 + 64 + 1 == 4545
    flat = np.arange(mlp.N_PARAMS, dtype=np.float64)
    np.testing.assert_array_equal(mlp.pack(mlp.unpack(flat)), flat)
    p = mlp.unpack(flat)
    assert p["W1"][1, 0] == 4 and p["b1"][0] == 256 and p["W2"][0, 1] == 321 and p["b3"][0] == 4544


def test_forward_closed_form():
    # one active path: x0 -> h1_0 -> h2_0 -> y
    p = {k: np.zeros(s) for k, s in mlp.SHAPES}
    p["W1"][0, 0], p["b1"][0] = 2.0, 0.5
    p["W2"][0, 0], p["b2"][0] = 3.0, -1.0
    p["w3"][0], p["b3"][0] = 0.25, 1.0
    X = np.array([[1.0, 9, 9, 9], [-1.0, 0, 0, 0]])
    y, _ = mlp.forward(mlp.pack(p), X)
    # x0 = 1: h1 = 2.5, h2 = 6.5, y = 2.625; x0 = -1: h1 = relu(-1.5) = 0, h2 = relu(-1) = 0, y = 1
    np.testing.assert_allclose(y, [2.625, 1.0], rtol=0, atol=1e-15)
    assert mlp.loss(mlp.pack(p), X, [2.625, 3.0]) == pytest.approx(2.0)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    flat = mlp.init(1)
    X = rng.uniform(-1, 1, (40, 4))
    t = rng.uniform(0, 8, 40)
    _, g = mlp.grad(flat, X, t)
    idx = np.concatenate([rng.choice(256, 25, replace=False), 256 + rng.choice(64, 10, replace=False),
                          320 + rng.choice(4096, 40, replace=False), 4416 + rng.choice(64, 10, replace=False),
                          4480 + rng.choice(64, 10, replace=False), [4544]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(flat)
        e[i] = h
        num = (mlp.loss(flat + e, X, t) - mlp.loss(flat - e, X, t)) / (2 * h)
        assert g[i] == pytest.approx(num, rel=1e-5, abs=1e-8), i


def test_gradient_descent_lowers_the_loss():
    rng = np.random.default_rng(5)
    flat = mlp.init(2)
    X = rng.uniform(0, 1, (64, 4))
    t = 3.0 + 2.0 * X[:, 0] - X[:, 1]
    l0, g = mlp.grad(flat, X, t)
    l1 = mlp.loss(flat - 1e-3 * g, X, t)
    assert l1 < l0
