"""GPU parity of the table path (PL1D, BILINEAR2D) against the FP64 oracle.

Tolerances (relative, from the method's stated targets): float64 paths
<= 1e-11, float32 paths <= 1e-5."""
import numpy as np
import pytest

import paper_1304_6514_gb300 as nvp
import workloads
from oracle import nievergelt as nv

from gpu_util import need_gpu, rel_l2, rel_max, run_method

pytestmark = pytest.mark.gpu


def _pl_case(torch, rhs_name, params, t0, T, S, M, lo, hi, scheme, dt, fixed, y0, prec):
    r = nvp.rhs(rhs_name, 1, params)
    smp = nvp.samples("pl1d", M, (lo,), (hi,))
    st = nvp.steps(scheme, dt, fixed, prec)
    maps, tab, yT, lam, oob = run_method(torch, r, t0, T, S, smp, st, [y0])
    m = nv.steps_per_slice(t0, T, S, dt, fixed)
    f = {"cos_cubic": nv.rhs_cos_cubic(), "square": nv.rhs_square(),
         "linear_scalar": nv.rhs_linear_scalar(params[0] if params else 0.0)}[rhs_name]
    otab = nv.build_table_1d(f, scheme, t0, T, S, m, nv.uniform_nodes(lo, hi, M))
    olam, ooob = nv.compose_tables_1d(lo, hi, otab, y0)
    return tab.reshape(S, M), otab, lam[:, 0], olam, oob, ooob


def test_scalar_cos_cubic_full_size_fp64():
    """y' = cos(t) y - y^3, S=16, M=64 on [-2,2], 10^4 Euler steps per slice."""
    torch = need_gpu()
    w = workloads.scalar_cos_cubic()
    tab, otab, lam, olam, oob, ooob = _pl_case(torch, "cos_cubic", (), w.t0, w.T, w.S, w.per_dim,
                                               -2.0, 2.0, "euler", 0.0, w.steps_per_slice, 0.5, "fp64")
    assert rel_max(tab, otab) <= 1e-11
    assert rel_max(lam, olam) <= 1e-11
    assert oob == ooob == 0


def test_scalar_cos_cubic_full_size_fp32():
    torch = need_gpu()
    w = workloads.scalar_cos_cubic()
    tab, otab, lam, olam, oob, _ = _pl_case(torch, "cos_cubic", (), w.t0, w.T, w.S, w.per_dim,
                                            -2.0, 2.0, "euler", 0.0, w.steps_per_slice, 0.5, "fp32")
    assert rel_max(tab, otab) <= 1e-5
    assert rel_l2(lam[-1:], olam[-1:]) <= 1e-5


@pytest.mark.parametrize("scheme", ["euler", "rk4"])
@pytest.mark.parametrize("M", [2, 37, 129])
def test_ragged_pl_sizes(scheme, M):
    """Node counts below, between and above the CTA size; RK4 stages the
    half-step coefficients, Euler the full-step ones (chunk boundary at 2048)."""
    torch = need_gpu()
    tab, otab, lam, olam, oob, ooob = _pl_case(torch, "cos_cubic", (), 0.3, 2.3, 5, M, -1.5, 1.7,
                                               scheme, 0.0, 2100, 0.4, "fp64")
    assert rel_max(tab, otab) <= 1e-11
    assert rel_max(lam, olam) <= 1e-11
    assert oob == ooob


def test_single_slice_table():
    """S = 1: the method degenerates to one table and one lookup."""
    torch = need_gpu()
    tab, otab, lam, olam, oob, ooob = _pl_case(torch, "cos_cubic", (), 0.0, 1.0, 1, 17, -2.0, 2.0,
                                               "rk4", 1e-3, 0, 0.5, "fp64")
    assert rel_max(tab, otab) <= 1e-11
    assert rel_max(lam, olam) <= 1e-11
    assert oob == ooob == 0


def test_out_of_range_extrapolates_and_counts():
    """y' = y^2 from 1.2 leaves [0, 1.5]: the edge segment is extended (as in
    the oracle) and every evaluation outside is counted."""
    torch = need_gpu()
    tab, otab, lam, olam, oob, ooob = _pl_case(torch, "square", (), 0.0, 0.5, 8, 9, 0.0, 1.5,
                                               "rk4", 1e-3, 0, 1.2, "fp64")
    assert ooob > 0 and oob == ooob
    assert rel_max(lam, olam) <= 1e-11


def test_out_of_range_error_policy():
    torch = need_gpu()
    r = nvp.rhs("square", 1)
    smp = nvp.samples("pl1d", 9, (0.0,), (1.5,), oob="error")
    maps = nvp.build_propagators(r, 0.0, 0.5, 8, smp, nvp.steps("rk4", 1e-3))
    y0 = torch.tensor([1.2], dtype=torch.float64, device="cuda")
    yT = torch.empty_like(y0)
    nvp.compose(maps, y0, yT)
    with pytest.raises(nvp.NvError) as e:
        nvp.maps_check(maps)
    assert e.value.status == nvp.NV_EDOMAIN


def test_linear_ode_pl_equals_serial_fine():
    """Linear slice maps are reproduced exactly by the PL table, so the GPU
    composition equals the GPU serial fine solve and the oracle's (Section 4)."""
    torch = need_gpu()
    r = nvp.rhs("linear_scalar", 1, (-0.4,))
    smp = nvp.samples("pl1d", 9, (-2.0,), (2.0,))
    st = nvp.steps("euler", 0.0, 50)
    _, _, yT, _, _ = run_method(torch, r, 0.0, 3.0, 6, smp, st, [3.5])
    y0 = torch.tensor([3.5], dtype=torch.float64, device="cuda")
    ys = torch.empty_like(y0)
    nvp.serial_fine(r, 0.0, 3.0, 6, st, y0, ys)
    ser = nv.serial_fine(nv.rhs_linear_scalar(-0.4), "euler", 0.0, 3.0, 6, 50, [3.5])
    assert abs(yT[0] - ser[0]) <= 1e-13 * abs(ser[0])
    assert abs(ys.item() - ser[0]) <= 1e-13 * abs(ser[0])


def test_serial_fine_cos_cubic_full_size():
    torch = need_gpu()
    w = workloads.scalar_cos_cubic()
    r = nvp.rhs("cos_cubic", 1)
    st = nvp.steps("euler", 0.0, w.steps_per_slice)
    y0 = torch.tensor([0.5], dtype=torch.float64, device="cuda")
    ys = torch.empty_like(y0)
    nvp.serial_fine(r, w.t0, w.T, w.S, st, y0, ys)
    ser = nv.serial_fine(nv.rhs_cos_cubic(), "euler", w.t0, w.T, w.S, w.steps_per_slice, [0.5])
    assert abs(ys.item() - ser[0]) <= 1e-11 * abs(ser[0])


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_vdp_bilinear_small(prec, tol):
    """Van der Pol, 9 x 9 grid on [-3,3]^2, RK4: table element by element and
    the bilinear composition, including evaluations that leave the square."""
    torch = need_gpu()
    mu, S, T, P = 1.7, 6, 3.0, 9
    r = nvp.rhs("vdp", 2, (mu,))
    smp = nvp.samples("bilinear2d", P, (-3.0, -3.0), (3.0, 3.0))
    st = nvp.steps("rk4", 1e-2, 0, prec)
    _, tab, yT, lam, oob = run_method(torch, r, 0.0, T, S, smp, st, [1.9, -2.5])
    m = nv.steps_per_slice(0.0, T, S, 1e-2)
    nodes = nv.uniform_nodes(-3.0, 3.0, P)
    otab = nv.build_table_2d(nv.rhs_vdp(mu), "rk4", 0.0, T, S, m, nodes, nodes)   # [j, p, q, c]
    gtab = tab.reshape(S, P, P, 2).transpose(0, 2, 1, 3)                            # [j, q, p] -> [j, p, q]
    assert rel_max(gtab, otab) <= tol
    olam, ooob = nv.compose_tables_2d(-3.0, 3.0, otab, [1.9, -2.5])
    assert rel_max(lam, olam) <= (tol if prec == "fp64" else 1e-4)
    assert oob == ooob


def test_maps_reuse_allocates_nothing_new():
    """A second build into the same maps object rewrites the same storage."""
    torch = need_gpu()
    r = nvp.rhs("cos_cubic", 1)
    smp = nvp.samples("pl1d", 16, (-2.0,), (2.0,))
    st = nvp.steps("euler", 0.0, 100)
    maps, tab1, _, _, _ = run_method(torch, r, 0.0, 1.0, 4, smp, st, [0.5])
    maps2, tab2, _, _, _ = run_method(torch, r, 0.0, 1.0, 4, smp, st, [0.5], maps=maps)
    assert maps2 is maps and np.array_equal(tab1, tab2)
    with pytest.raises(nvp.NvError):
        nvp.build_propagators(r, 0.0, 1.0, 5, smp, st, maps=maps)   # different S


@pytest.mark.parametrize("e,S,M", [(14, 32, 4), (16, 128, 7)])
def test_square_paper_table_shapes_fp32(e, S, M):
    """The shapes of the paper's GPU table (y' = y^2 on [0, 1/2], dt = 2^-e, N
    slices, M nodes) in float32 forward Euler with PL tables on [0, 2]: whole
    tables and every boundary state against the oracle."""
    torch = need_gpu()
    w = workloads.square_paper(e, S, M)
    tab, otab, lam, olam, oob, ooob = _pl_case(torch, "square", (), w.t0, w.T, S, M, 0.0, 2.0,
                                               "euler", w.dt, 0, 1.0, "fp32")
    assert rel_max(tab, otab) <= 1e-5
    assert rel_l2(lam, olam) <= 1e-5
    # the chords of this convex map lie above it, so with 4..7 nodes the last
    # lookup already lands above y = 2 in both (oracle: lambda_{S-1} = 2.03 / 2.005)
    assert oob == ooob == 1
