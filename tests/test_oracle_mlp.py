"""Pins of the oracle's MLP: backpropagation against central finite
differences, GELU against its defining identities.  CPU only."""
import math

import numpy as np
import pytest

from oracle import mlp


def test_gelu_identities():
    z = np.array([-3.0, -1.0, 0.0, 0.5, 2.0, 8.0])
    g = mlp.gelu(z)
    assert g[2] == 0.0
    assert abs(g[-1] - 8.0) < 1e-12                                  # Phi(8) = 1 - 6e-16
    assert np.allclose(g - mlp.gelu(-z), z, atol=1e-15)              # z Phi(z) - (-z) Phi(-z) = z
    assert abs(mlp.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(z), fd, atol=1e-8)


@pytest.mark.parametrize("name", ["W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4"])
def test_backprop_matches_finite_differences(name):
    rng = np.random.default_rng(3)
    p = mlp.init_params(1, sizes=(7, 9, 8, 7, 6))
    X = rng.uniform(-1, 1, (5, 7))
    tgt = rng.uniform(-1, 1, (5, 6))
    _, g = mlp.loss_and_grads(p, X, tgt)
    flat = p[name].reshape(-1)
    gflat = g[name].reshape(-1)
    for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
        old = flat[idx]
        h = 1e-6
        flat[idx] = old + h
        lp, _ = mlp.loss_and_grads(p, X, tgt)
        flat[idx] = old - h
        lm, _ = mlp.loss_and_grads(p, X, tgt)
        flat[idx] = old
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gflat[idx]) <= 1e-7 * max(1.0, abs(fd)), (name, idx, fd, gflat[idx])


def test_apply_map_is_increment():
    p = mlp.init_params(2, sizes=(7, 4, 4, 4, 6))
    for k in p:
        p[k][...] = 0.0
    y0 = np.array([[0.1, -0.2, 0.3, 0.0, 0.5, -0.5]])
    assert np.array_equal(mlp.apply_map(p, y0, 0.25, 0.5, 0.1), y0)   # zero network = identity map
