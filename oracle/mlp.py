"""FP64 statement of the slice-conditioned MLP propagator (the learned map
that stands in for a table when the initial-value space has many dimensions,
Section 4's l^r cost remark and the Conclusion's call for better maps in high
dimension).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Network: x (6 state components scaled by 1/sx, plus the slice time
T_{j-1}/T) -> three hidden layers of 256 with GELU -> 6 outputs, the slice
increment (y_end - y0) scaled by 1/sd.  GELU(z) = z/2 (1 + erf(z/sqrt 2)).
Loss over a batch of B samples: L = (1/B) sum_b sum_o (out_bo - tgt_bo)^2 / 2.

Parameters are a dict W1 (256, 7), b1 (256,), W2, W3 (256, 256), b2, b3,
W4 (6, 256), b4 (6,), weights stored [out, in].
"""
from __future__ import annotations

import math

import numpy as np

SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)
LAYERS = ("1", "2", "3", "4")


def _erf(z):
    return np.vectorize(math.erf, otypes=[np.float64])(z)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / SQRT2))


def gelu_grad(z):
    """d/dz of z Phi(z) = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + _erf(z / SQRT2)) + z * INV_SQRT_2PI * np.exp(-0.5 * z * z)


def init_params(seed: int = 0, sizes=(7, 256, 256, 256, 6)):
    """Uniform(-1/sqrt(in), 1/sqrt(in)) weights and biases (numpy generator;
    the GPU trainer draws its own from SplitMix64)."""
    rng = np.random.default_rng(seed)
    p = {}
    for i, name in enumerate(LAYERS):
        fan_in, fan_out = sizes[i], sizes[i + 1]
        bound = 1.0 / math.sqrt(fan_in)
        p["W" + name] = rng.uniform(-bound, bound, (fan_out, fan_in))
        p["b" + name] = rng.uniform(-bound, bound, fan_out)
    return p


def forward(p, X):
    """X (B, 7) -> (out (B, 6), cache of pre-activations and activations)."""
    cache = {"h0": X}
    h = X
    for name in LAYERS[:3]:
        z = h @ p["W" + name].T + p["b" + name]
        cache["z" + name] = z
        h = gelu(z)
        cache["h" + name] = h
    out = h @ p["W4"].T + p["b4"]
    return out, cache


def loss_and_grads(p, X, tgt):
    """Half mean-squared error over the batch and its gradients (backpropagation
    written out layer by layer)."""
    B = X.shape[0]
    out, c = forward(p, X)
    r = out - tgt
    loss = 0.5 * float(np.sum(r * r)) / B
    g = {}
    d = r / B                                 # dL/dout
    g["W4"] = d.T @ c["h3"]
    g["b4"] = d.sum(axis=0)
    dh = d @ p["W4"]
    for name, prev in (("3", "h2"), ("2", "h1"), ("1", "h0")):
        dz = dh * gelu_grad(c["z" + name])
        g["W" + name] = dz.T @ c[prev]
        g["b" + name] = dz.sum(axis=0)
        dh = dz @ p["W" + name]
    return loss, g


def features(y0, t_frac, sx):
    """Network input: state scaled by 1/sx, then the slice time fraction."""
    y0 = np.atleast_2d(y0)
    return np.concatenate([y0 / sx, np.full((y0.shape[0], 1), t_frac)], axis=1)


def apply_map(p, y0, t_frac, sx, sd):
    """y_end = y0 + sd * MLP((y0 / sx, t_frac))."""
    out, _ = forward(p, features(y0, t_frac, sx))
    return np.atleast_2d(y0) + out * sd
