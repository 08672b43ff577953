"""Pins of the wave-equation oracle (Section 5, eq. waveequation) against the
mathematics: spectral exactness of the differentiation matrix on polynomials,
the Dirichlet eigenvalues -(k pi / 2)^2, the closed form of leapfrog on one
eigenmode, the slice map as a matrix power, composition = serial solve, and
the discrete solution against the exact travelling pulse."""
import math

import numpy as np
import pytest

import workloads
from oracle import nievergelt as nv
from oracle import wave


@pytest.mark.parametrize("M", [4, 9, 16])
def test_differentiation_is_exact_on_polynomials(M):
    """Interpolation on M + 1 points reproduces any polynomial of degree <= M,
    so D maps x^k to k x^(k-1) at the points (up to rounding)."""
    x = wave.cheb_points(M)
    D = wave.cheb_diff_matrix(M)
    for k in range(M + 1):
        exact = k * x ** (k - 1) if k > 0 else np.zeros_like(x)
        assert np.max(np.abs(D @ x ** k - exact)) <= 1e-11 * max(1.0, k * k), k


def test_points_are_gauss_lobatto():
    x = wave.cheb_points(8)
    assert x[0] == 1.0 and x[-1] == -1.0
    assert np.all(np.diff(x) < 0)
    np.testing.assert_allclose(x, -x[::-1], atol=1e-15)


def test_dirichlet_eigenvalues():
    """u'' = lam u, u(+-1) = 0 has lam_k = -(k pi / 2)^2; the spectral matrix
    gets the low modes to near machine precision."""
    D2 = wave.interior_second_derivative(40)
    ev = np.sort(np.linalg.eigvals(D2).real)[::-1]        # least negative first
    for k in range(1, 11):
        lam = -(k * math.pi / 2) ** 2
        assert abs(ev[k - 1] - lam) <= 1e-9 * abs(lam), k


def test_leapfrog_mode_closed_form():
    """On an eigenvector v (D2 v = -w^2 v) the recurrence u^{n+1} = (2 - h^2 w^2)
    u^n - u^{n-1} from (u^0, u^{-1}) = (v, v) is u^n = (cos n t + (cos t - 1)
    / sin t * sin n t) v with cos t = 1 - h^2 w^2 / 2."""
    M, h, m = 24, 8.0 / 24 ** 2, 37
    D2 = wave.interior_second_derivative(M)
    lam, V = np.linalg.eig(D2)
    for k in np.argsort(-lam.real)[[0, 3, 10]]:
        v = V[:, k].real
        w2 = -lam[k].real
        th = math.acos(1.0 - h * h * w2 / 2.0)
        coef = lambda n: math.cos(n * th) + (math.cos(th) - 1.0) / math.sin(th) * math.sin(n * th)
        Y = wave.integrate(D2, np.concatenate([v, v])[:, None], h, m)[:, 0]
        d = M - 1
        np.testing.assert_allclose(Y[:d], coef(m) * v, atol=1e-10)
        np.testing.assert_allclose(Y[d:], coef(m - 1) * v, atol=1e-10)


def test_slice_map_is_matrix_power_and_b_is_zero():
    M, S, m, h = 12, 3, 7, 8.0 / 144
    A, b = wave.build_affine(M, S, m, h)
    D2 = wave.interior_second_derivative(M)
    d = M - 1
    I = np.eye(d)
    P = np.block([[2 * I + h * h * D2, -I], [I, np.zeros((d, d))]])
    Pm = np.linalg.matrix_power(P, m)
    for j in range(S):
        np.testing.assert_allclose(A[j], Pm, rtol=0, atol=1e-12 * np.abs(Pm).max())
        assert np.array_equal(b[j], np.zeros(2 * d))


def test_composition_equals_serial_solve():
    M, S, T = 16, 6, 1.5
    w = workloads.wave1d(M=M, S=S, T=T)
    m = nv.steps_per_slice(w.t0, w.T, S, w.dt)
    h = nv.step_size(w.t0, w.T, S, m)
    y0 = workloads.wave1d_initial(M, h)
    A, b = wave.build_affine(M, S, m, h)
    lam = wave.compose(A, b, y0)
    ys = wave.serial_fine(M, S, m, h, y0)
    assert np.linalg.norm(lam[-1] - ys) <= 1e-12 * np.linalg.norm(ys)


def test_discrete_solution_follows_the_travelling_pulse():
    """Before the peak reaches the boundary, the discrete solution matches the
    exact u(x, t) = exp(-200 (x + t)^2): the model, the [-1, 1] domain, the
    sign of the second-derivative matrix and the two-level start all agree."""
    M, S, T = 80, 16, 0.4
    w = workloads.wave1d(M=M, S=S, T=T)
    m = nv.steps_per_slice(w.t0, w.T, S, w.dt)
    h = nv.step_size(w.t0, w.T, S, m)
    y = wave.serial_fine(M, S, m, h, workloads.wave1d_initial(M, h))
    x = wave.cheb_points(M)[1:M]
    exact = np.exp(-200.0 * (x + T) ** 2)
    d = M - 1
    assert np.max(np.abs(y[:d] - exact)) <= 1e-3       # measured 2.4e-4
    assert abs(x[np.argmax(y[:d])] + T) <= 0.05          # the peak moved left by T


def test_wave_step_rule_matches_table_sizes():
    """Table wave80: M = 80, T = 20, up to N = 512 slices; dt = 8/M^2 gives
    31.25 steps per slice, so m = 32 and h = H/32."""
    w = workloads.wave1d()
    m = nv.steps_per_slice(w.t0, w.T, w.S, w.dt)
    assert (w.dim, m) == (158, 32)
    assert nv.step_size(w.t0, w.T, w.S, m) == 20.0 / 512 / 32
