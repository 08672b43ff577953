"""Cost model of the GPU method (Section "A graphics card implementation and
cost model", eqs. gpucostmodel and serialcostmodel).

Time to solution on the GPU, C_G = (M n / N) tau_F + N tau_N + tau_K, and
serially, C_C = n tau_C, where n is the total number of fine steps (T / dt),
N the number of slices, M the samples per slice, tau_F the time to advance
one trajectory by one step, tau_N the time to apply one slice map in the
composition and tau_K a fixed overhead.  The paper reads n this way without
saying so: with it, the printed parameters (Table tauparameters) reproduce the
printed estimates (last column of Table gpuresults) to 0.6 %.

Host-side arithmetic on measured times (plain Python and numpy): no part of
the method's computation.
"""
from __future__ import annotations

import numpy as np


def gpu_cost(n: float, N: int, M: int, tau_F: float, tau_N: float, tau_K: float) -> float:
    """C_G = (M n / N) tau_F + N tau_N + tau_K (eq. gpucostmodel)."""
    return M * n / N * tau_F + N * tau_N + tau_K


def serial_cost(n: float, tau_C: float) -> float:
    """C_C = n tau_C (eq. serialcostmodel)."""
    return n * tau_C


def fit_gpu_cost(rows) -> tuple[float, float, float]:
    """Least-squares (tau_F, tau_N, tau_K) from rows of (n, N, M, time), the
    fit the paper makes for Table tauparameters."""
    rows = list(rows)
    if len(rows) < 3:
        raise ValueError("the fit needs at least three (n, N, M, time) rows")
    X = np.array([[M * n / N, N, 1.0] for n, N, M, _ in rows], dtype=np.float64)
    y = np.array([t for _, _, _, t in rows], dtype=np.float64)
    coef, *_ = np.linalg.lstsq(X, y, rcond=None)
    return float(coef[0]), float(coef[1]), float(coef[2])
