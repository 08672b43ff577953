"""The cost model of the GPU method against the paper's printed tables
(Section "A graphics card implementation and cost model")."""
import os

import numpy as np

from paper_1304_6514_gb300 import costmodel

HERE = os.path.dirname(os.path.abspath(__file__))


def _table():
    rows, params = [], None
    for line in open(os.path.join(HERE, "golden", "table_gpuresults.txt")):
        if line.startswith("# params"):
            params = [float(v) for v in line.split()[2:]]
        elif line.strip() and not line.startswith("#"):
            e, N, M, t_total, speedup, t_est = line.split()
            rows.append((int(e), int(N), int(M), float(t_total), float(speedup), float(t_est)))
    return rows, params


def test_printed_parameters_reproduce_printed_estimates():
    """eq. gpucostmodel with Table tauparameters and n = T / dt (T = 1/2) gives
    the last column of Table gpuresults to 1 % on every row (0.6 % at most);
    n read as the steps of one slice misses a row by more than 10 % (20 %)."""
    rows, (tau_F, tau_N, tau_K, _) = _table()
    assert len(rows) == 9
    worst_other = 0.0
    for e, N, M, _, _, t_est in rows:
        n = 0.5 * 2 ** e
        assert abs(costmodel.gpu_cost(n, N, M, tau_F, tau_N, tau_K) - t_est) <= 0.01 * t_est
        other = costmodel.gpu_cost(n / N, N, M, tau_F, tau_N, tau_K)
        worst_other = max(worst_other, abs(other - t_est) / t_est)
    assert worst_other > 0.10


def test_serial_parameter_matches_printed_speedups():
    """eq. serialcostmodel: T_total x (T_cpu / T_total) / n on every row is the
    printed tau_C = 0.051 to the two printed digits of the speedup (5 %)."""
    rows, (_, _, _, tau_C) = _table()
    for e, N, M, t_total, speedup, _ in rows:
        n = 0.5 * 2 ** e
        assert abs(t_total * speedup / n - tau_C) <= 0.05 * tau_C
        assert abs(costmodel.serial_cost(n, tau_C) - t_total * speedup) <= 0.05 * t_total * speedup


def test_fit_recovers_parameters_of_synthetic_times():
    """The least-squares fit returns the parameters that generated exact times,
    and fits the printed measurements at least as well as the printed
    parameters do (least squares, by definition)."""
    rows, (tau_F, tau_N, tau_K, _) = _table()
    shapes = [(0.5 * 2 ** e, N, M) for e, N, M, _, _, _ in rows]
    synth = [(n, N, M, costmodel.gpu_cost(n, N, M, 0.02, 0.3, 50.0)) for n, N, M in shapes]
    np.testing.assert_allclose(costmodel.fit_gpu_cost(synth), (0.02, 0.3, 50.0), rtol=1e-10)
    meas = [(n, N, M, t) for (n, N, M), (_, _, _, t, _, _) in zip(shapes, rows)]
    fit = costmodel.fit_gpu_cost(meas)
    sse = lambda p: sum((costmodel.gpu_cost(n, N, M, *p) - t) ** 2 for n, N, M, t in meas)
    assert sse(fit) <= sse((tau_F, tau_N, tau_K)) + 1e-9
