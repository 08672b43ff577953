"""Plain FP64 statement of the wave-equation example of Section 5 (eq.
waveequation, Tables wave40 / wave80).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Model: u_tt = u_xx with homogeneous Dirichlet conditions, discretised in space
with the Chebyshev spectral method on the M + 1 Gauss-Lobatto points
x_i = cos(i pi / M) of [-1, 1] and in time with the explicit second-order
leapfrog method, dt = 8 / M^2.  The unknowns are the M - 1 interior values.

Reading of the domain: the paper writes x in [0, 1] but takes the problem and
the CFL-limited step dt = 8/M^2 from the cited spectral-methods program, whose
domain is [-1, 1]; on [0, 1] the second-derivative matrix is four times larger
and that step is unstable (h sqrt(rho(D2)) / 2 = 1.74 for M = 80, against 0.87
on [-1, 1]).  The domain is therefore [-1, 1].

Two-level state (Section 5, after Table wave40): leapfrog needs the values at
the last two steps, so the state of a slice boundary is Y = (u^n, u^{n-1}) of
dimension 2 (M - 1), the initial-value space doubles, and the affine map of a
slice is the m-th power of the one-step matrix [[2 I + h^2 D2, -I], [I, 0]]
(no forcing, so b_j = 0).

Array convention: states (2d, K), K independent trajectories.
"""
from __future__ import annotations

import math

import numpy as np

from . import nievergelt as nv


def cheb_points(M: int) -> np.ndarray:
    """Gauss-Lobatto points x_i = cos(i pi / M), i = 0..M (x_0 = 1)."""
    return np.array([math.cos(i * math.pi / M) for i in range(M + 1)], dtype=np.float64)


def cheb_diff_matrix(M: int) -> np.ndarray:
    """First-derivative matrix of polynomial interpolation on the Gauss-Lobatto
    points: off the diagonal D_ij = (c_i / c_j) (-1)^(i+j) / (x_i - x_j) with
    c_0 = c_M = 2 and c_i = 1 otherwise (the barycentric weights of these
    points); the diagonal makes every row sum to zero, since the derivative of
    a constant vanishes."""
    x = cheb_points(M)
    c = [2.0 if i in (0, M) else 1.0 for i in range(M + 1)]
    D = np.zeros((M + 1, M + 1))
    for i in range(M + 1):
        for j in range(M + 1):
            if i != j:
                sign = 1.0 if (i + j) % 2 == 0 else -1.0
                D[i, j] = (c[i] / c[j]) * sign / (x[i] - x[j])
    for i in range(M + 1):
        D[i, i] = -sum(D[i, j] for j in range(M + 1) if j != i)
    return D


def interior_second_derivative(M: int) -> np.ndarray:
    """D2 = D D restricted to the interior points 1..M-1: with u = 0 at both
    ends, the boundary columns multiply zeros and the boundary rows are not
    unknowns.  Returns (M-1, M-1)."""
    D = cheb_diff_matrix(M)
    return (D @ D)[1:M, 1:M]


def leapfrog_step(D2: np.ndarray, Y: np.ndarray, h: float) -> np.ndarray:
    """u^{n+1} = 2 u^n - u^{n-1} + h^2 D2 u^n on the stacked state
    Y = (u^n, u^{n-1}); returns (u^{n+1}, u^n)."""
    d = D2.shape[0]
    u, u_old = Y[:d], Y[d:]
    u_new = 2.0 * u - u_old + (h * h) * (D2 @ u)
    return np.concatenate([u_new, u], axis=0)


def integrate(D2: np.ndarray, Y0: np.ndarray, h: float, m: int) -> np.ndarray:
    """m leapfrog steps of every column of Y0 (a slice of Figure "pseudocode")."""
    Y = np.array(Y0, dtype=np.float64, copy=True)
    for _ in range(m):
        Y = leapfrog_step(D2, Y, h)
    return Y


def build_affine(M: int, S: int, m: int, h: float, slices=None):
    """Affine slice maps (eqs. lineardiscrete, linearreconstruct) on the
    doubled state: b_j = solve from 0, column c of A_j = solve from e_c.  The
    operator does not depend on time, so every slice runs the same steps; the
    method still integrates each slice's basis.  Returns A (len, n, n),
    b (len, n) for the requested slices (default all), n = 2 (M - 1)."""
    D2 = interior_second_derivative(M)
    n = 2 * (M - 1)
    js = range(S) if slices is None else slices
    A = np.empty((len(js), n, n))
    b = np.empty((len(js), n))
    for k, _j in enumerate(js):
        b[k] = integrate(D2, np.zeros((n, 1)), h, m)[:, 0]
        A[k] = integrate(D2, np.eye(n), h, m)
    return A, b


def serial_fine(M: int, S: int, m: int, h: float, y0: np.ndarray) -> np.ndarray:
    """The serial leapfrog solve over all S m steps from y0 = (u^0, u^{-1})."""
    D2 = interior_second_derivative(M)
    Y = np.array(y0, dtype=np.float64).reshape(-1, 1)
    for _ in range(S):
        Y = integrate(D2, Y, h, m)
    return Y[:, 0]


def compose(A, b, y0):
    """Communication phase: lambda_j = A_j lambda_{j-1} + b_j."""
    return nv.compose_affine(A, b, y0)
