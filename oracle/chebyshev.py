"""Backward Euler + Chebyshev interpolation: the configuration of the paper's
Table 1 (Section 3) and of its GPU experiment (Table 3).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Not on the GPU path;
it exists so that the oracle's slice grid, step rule and composition can be
pinned against numbers the paper prints.

Readings (Table 1 is reproduced to its printed digits only with these):
  * "M Chebyshev nodes on [0, 2]" are the Gauss-Lobatto points
    1 + cos(i pi / (M - 1)), i = 0..M-1;
  * a non-integer H/dt gives m = ceil(H/dt) steps of size H/m.
"""
from __future__ import annotations

import math

import numpy as np

from .nievergelt import slice_times, step_size, steps_per_slice


def backward_euler_square(y: np.ndarray, h: float, m: int) -> np.ndarray:
    """m backward Euler steps of y' = y^2: y_{i+1} = y_i + h y_{i+1}^2, solved for
    the root that tends to y_i as h -> 0: y_{i+1} = (1 - sqrt(1 - 4 h y_i)) / (2h)."""
    y = np.array(y, dtype=np.float64, copy=True)
    for _ in range(m):
        y = (1.0 - np.sqrt(1.0 - 4.0 * h * y)) / (2.0 * h)
    return y


def lobatto_nodes(a: float, b: float, M: int) -> np.ndarray:
    """Chebyshev-Gauss-Lobatto points mapped to [a, b]."""
    i = np.arange(M)
    return (a + b) / 2 + (b - a) / 2 * np.cos(i * math.pi / (M - 1))


def lagrange_eval(nodes: np.ndarray, values: np.ndarray, x: float) -> float:
    """Lagrange form of the interpolating polynomial through (nodes, values)."""
    total = 0.0
    for k in range(len(nodes)):
        L = 1.0
        for i in range(len(nodes)):
            if i != k:
                L *= (x - nodes[i]) / (nodes[k] - nodes[i])
        total += values[k] * L
    return total


def nievergelt_square_be(dt: float, M: int, S: int = 4, T: float = 0.5, y0: float = 1.0,
                         a: float = 0.0, b: float = 2.0) -> float:
    """y(T) from the method on y' = y^2 with backward Euler and Lagrange
    interpolation on M Chebyshev-Lobatto nodes of [a, b] (Figure "pseudocode")."""
    m = steps_per_slice(0.0, T, S, dt)
    h = step_size(0.0, T, S, m)
    nodes = lobatto_nodes(a, b, M)
    lam = y0
    for _j in range(S):
        vals = backward_euler_square(nodes, h, m)
        lam = lagrange_eval(nodes, vals, lam)
    return float(lam)


def serial_square_be(dt: float, S: int = 4, T: float = 0.5, y0: float = 1.0) -> float:
    """Serial backward Euler over all slices with the same step size."""
    m = steps_per_slice(0.0, T, S, dt)
    h = step_size(0.0, T, S, m)
    return float(backward_euler_square(np.array([y0]), h, m * S)[0])


def square_exact(t: float, y0: float = 1.0) -> float:
    """Exact solution of y' = y^2, y(0) = y0: y = y0 / (1 - y0 t) (Section 3)."""
    return y0 / (1.0 - y0 * t)


__all__ = ["backward_euler_square", "lobatto_nodes", "lagrange_eval", "nievergelt_square_be",
           "serial_square_be", "square_exact", "slice_times"]
