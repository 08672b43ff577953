"""GPU parity of the affine path (heat equation maps, chain composition)
against the FP64 oracle.

Tolerances: float64 <= 1e-11 relative L2 (maps: max-norm relative to the
largest entry), float32 <= 1e-5."""
import numpy as np
import pytest

import paper_1304_6514_gb300 as nvp
import workloads
from oracle import nievergelt as nv

from gpu_util import need_gpu, rel_l2, rel_max, run_method

pytestmark = pytest.mark.gpu


def _heat(torch, w, prec, rhs_name="heat1d"):
    r = nvp.rhs(rhs_name, w.dim, w.params if rhs_name == "heat1d" else ())
    smp = nvp.samples("affine")
    st = nvp.steps("rk4", w.dt, w.steps_per_slice, prec)
    maps, tab, yT, lam, oob = run_method(torch, r, w.t0, w.T, w.S, smp, st, w.y0)
    n = w.dim
    blocks = tab.reshape(w.S, n + 1, n)          # [j, col, row]
    b = blocks[:, 0, :]
    A = blocks[:, 1:, :].transpose(0, 2, 1)      # A[j][row, col]
    return maps, A, b, yT, lam


@pytest.mark.parametrize("n,S", [(40, 7), (64, 3), (1, 4), (97, 5), (40, 1), (256, 1)])
def test_heat_small_elementwise_fp64(n, S):
    """Every map entry and every boundary state; n = 40 and 97 leave padding
    rows in the last lanes, n = 1 is the degenerate single-unknown case, S = 1
    the single slice (a chain of one step)."""
    torch = need_gpu()
    dt = min(5e-5, 2.0 / (4.0 * (n + 1) ** 2))       # within RK4's stability limit
    w = workloads.heat1d(n=n, S=S, T=60 * dt, dt=dt)
    _, A, b, yT, lam = _heat(torch, w, "fp64")
    m = nv.workload_steps(w)
    fi, fh = nv.workload_rhs(w, True), nv.workload_rhs(w, False)
    oA, ob = nv.build_affine(fi, fh, "rk4", w.t0, w.T, w.S, m, n)
    assert rel_max(A, oA) <= 1e-11
    assert rel_max(b, ob) <= 1e-11
    olam = nv.compose_affine(oA, ob, w.y0)
    assert rel_l2(lam, olam) <= 1e-11
    assert rel_l2(yT, olam[-1]) <= 1e-11


@pytest.mark.parametrize("form", [1, 2, 3])
@pytest.mark.parametrize("n,S", [(128, 3), (200, 4), (256, 3), (512, 2)])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_heat_step_forms_elementwise(form, n, S, prec, tol):
    """Both forms of the homogeneous RK4 step (1: Horner stages, 2: the
    nine-point stencil with odd reflection at the Dirichlet ends) give the
    oracle's maps: n = 128 (four rows per lane), 200 (eight rows, lanes 25..31
    idle, right end inside the warp), 256, 512 (sixteen rows).  Step size at
    the RK4 stability edge, h cdx |lambda_max| = 2."""
    torch = need_gpu()
    dt = 2.0 / (4.0 * (n + 1) ** 2)
    w = workloads.heat1d(n=n, S=S, T=S * 3 * dt, dt=dt)
    nvp.tune_set(6, form)
    try:
        _, A, b, yT, lam = _heat(torch, w, prec)
    finally:
        nvp.tune_set(6, 0)
    m = nv.workload_steps(w)
    fi, fh = nv.workload_rhs(w, True), nv.workload_rhs(w, False)
    oA, ob = nv.build_affine(fi, fh, "rk4", w.t0, w.T, w.S, m, n)
    assert rel_max(A, oA) <= tol
    assert rel_max(b, ob) <= tol
    olam = nv.compose_affine(oA, ob, w.y0)
    assert rel_l2(lam, olam) <= (1e-11 if prec == "fp64" else 1e-4)


@pytest.mark.parametrize("n,S,steps,form", [
    (256, 1024, 10, 3), (256, 1024, 10, 4),      # the heat benchmark's build
    (256, 6, 3, 3), (100, 5, 5, 3), (128, 4, 15, 3), (512, 3, 21, 3), (512, 2, 31, 3), (200, 4, 10, 3),
    (256, 6, 8, 4), (100, 5, 6, 4), (128, 4, 15, 4), (176, 3, 12, 4), (200, 4, 10, 4),
    (256, 1024, 10, 5), (256, 6, 8, 5), (100, 5, 6, 5), (88, 3, 10, 5), (200, 4, 9, 5)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_heat_window_matches_full_width(n, S, steps, form, prec):
    """The windowed nine-point builds (each column integrated only over the
    rows its steps reach: form 3 one window of >= 8m+1 rows, form 4 a narrow
    window for the first steps and a wide one for the rest, form 5 three
    windows of 22, 44 and 88 rows) write the same
    maps as the full-width nine-point build, entry for entry (zeros compare
    equal whatever their sign).  n = 256, S = 1024, m = 10 is the heat
    benchmark's build; the others take every built window shape, windows
    against both Dirichlet ends, windows as wide as n (n = 128, m = 15;
    n = 88, m = 10) and n = 100, 176, 200 (not multiples of a window's rows
    per lane)."""
    torch = need_gpu()
    T = 0.1 if (n, S) == (256, 1024) else S * steps * 2.0 / (5.0 * (n + 1) ** 2)
    w = workloads.heat1d(n=n, S=S, T=T, dt=T / (S * steps))
    assert nv.workload_steps(w) == steps
    got = {}
    for f in (form, 2):
        nvp.tune_set(6, f)
        try:
            _, A, b, yT, lam = _heat(torch, w, prec)
        finally:
            nvp.tune_set(6, 0)
        got[f] = (A, b, lam)
    assert np.array_equal(got[form][0], got[2][0])
    assert np.array_equal(got[form][1], got[2][1])
    assert np.array_equal(got[form][2], got[2][2])
    # the zeros outside the reach are exact
    A = got[form][0]
    rows, cols = np.indices(A.shape[1:])
    outside = np.abs(rows - cols) > 4 * steps
    assert not np.any(A[:, outside])


@pytest.mark.parametrize("prec", ["fp32", "tf32_refine"])
@pytest.mark.parametrize("n,S,steps", [(256, 1024, 10), (256, 6, 8), (200, 4, 9), (88, 3, 10), (90, 5, 10),
                                       (256, 1, 10)])
def test_heat_f32_three_window_lane_shapes_agree(n, S, steps, prec):
    """The float32 three-window build runs its 22/44/88-row windows on 1/2/4
    lanes of 22 rows (key 17 = 1) or on 2/4/8 lanes of 11 rows (key 17 = 2,
    the float64 shape), each either one slice per register or two slices per
    packed f32x2 register (keys 3 and 4; an odd S leaves the last pair's high
    half unused, S = 1 takes the scalar kernel): every row is the same
    expression on the same values, so the maps and the composed states agree
    bit for bit, also with the TF32 rounding of the stored maps (the TF32
    scan's input).  n = 90 takes the row-by-row store (n not a multiple of
    four floats)."""
    torch = need_gpu()
    if prec == "tf32_refine" and n % 4:
        pytest.skip("the TF32 scan takes d a multiple of 4")
    T = 0.1 if (n, S) == (256, 1024) else S * steps * 2.0 / (5.0 * (n + 1) ** 2)
    w = workloads.heat1d(n=n, S=S, T=T, dt=T / (S * steps))
    got = {}
    for lanes in (1, 2, 3, 4):
        nvp.tune_set(6, 5)
        nvp.tune_set(17, lanes)
        try:
            maps, A, b, yT, lam = _heat(torch, w, prec)
            kernel = nvp.maps_info(maps).build_kernel.decode()
        finally:
            nvp.tune_set(6, 0)
            nvp.tune_set(17, 0)
        assert ("x2" in kernel) == (lanes >= 3 and S > 1), (lanes, kernel)
        got[lanes] = (A, b, lam)
    for lanes in (2, 3, 4):
        for k in range(3):
            assert np.array_equal(got[1][k], got[lanes][k]), (lanes, k)


@pytest.mark.parametrize("n,S,steps,rhs_name", [(256, 1024, 10, "heat1d"), (256, 7, 3, "heat1d"),
                                                (128, 5, 2, "heat1d"), (64, 3, 1, "heat1d"),
                                                (192, 6, 5, "heat1d"), (256, 4, 40, "heat1d"),
                                                (128, 5, 4, "heat1d_varcoef")])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_refine"])
def test_banded_chain_matches_dense(n, S, steps, rhs_name, prec):
    """The heat maps are zero off the band |r - c| <= 4m, and the cluster
    chain then reads only the columns of that band around each CTA's rows
    (rounded out to 16 so that every thread keeps its columns and their
    order): every boundary state equals the dense chain's (tunable 14 = 1)
    bit for bit, for the plain float64 / float32 compositions and the
    pipelined float64 refinement.  n = 256, S = 1024, m = 10 is the heat
    benchmark; m = 40 at n = 256 has a band wider than the matrix (dense);
    the variable-coefficient equation (time-dependent three-point operator)
    has the same band."""
    torch = need_gpu()
    T = 0.1 if (n, S) == (256, 1024) else S * steps * 2.0 / (5.0 * 1.25 * (n + 1) ** 2)
    if rhs_name == "heat1d":
        w = workloads.heat1d(n=n, S=S, T=T, dt=T / (S * steps))
    else:
        w = workloads.Workload("v", "heat1d_varcoef", n, 0.0, T, S, "rk4", T / (S * steps), 0, "affine",
                               y0=np.sin(np.pi * nv.heat1d_grid(n)))
    assert nv.workload_steps(w) == steps
    got = {}
    for dense in (0, 1):
        nvp.tune_set(14, dense)
        try:
            _, A, b, yT, lam = _heat(torch, w, prec, rhs_name)
        finally:
            nvp.tune_set(14, 0)
        got[dense] = (yT, lam)
    assert np.array_equal(got[0][0], got[1][0])
    assert np.array_equal(got[0][1], got[1][1])
    rows, cols = np.indices((n, n))
    assert not np.any(A[:, np.abs(rows - cols) > 4 * steps])   # the band the chain relies on


def test_build_reports_work_kernel_and_band():
    """nv_maps_info reports what the build ran: the point-steps integrated per
    slice (the forcing column at full width, each homogeneous column over its
    windows: 22·2 + 44·3 + 88·5 = 616 row-steps for m = 10), the kernel, and
    the band |r - c| <= 4m of the heat maps; the full-width form integrates
    all d rows; the advection-diffusion maps are dense, and their float32
    build integrates 3 steps on 32 x 32 windows and 7 on the 64 x 64 grid."""
    torch = need_gpu()
    n, S, steps = 256, 4, 10
    T = S * steps * 2.0 / (5.0 * (n + 1) ** 2)
    w = workloads.heat1d(n=n, S=S, T=T, dt=T / (S * steps))
    r = nvp.rhs("heat1d", n, w.params)
    for form, work, kernel in ((0, n * steps + n * 616, "heat_window3_kernel<double,2,11,0>"),
                               (2, (n + 1) * n * steps, "heat_poly9_kernel<double,8,0>")):
        nvp.tune_set(6, form)
        try:
            maps = nvp.build_propagators(r, w.t0, w.T, w.S, nvp.samples("affine"), nvp.steps("rk4", w.dt))
        finally:
            nvp.tune_set(6, 0)
        d = nvp.maps_info(maps)
        assert (d.work_per_slice, d.build_kernel.decode(), d.band) == (work, kernel, 4 * steps + 1)
        maps.destroy()
    wa = workloads.advdiff2d(S=2, T=2 * 10 * 2e-4, dt=2e-4)
    ra = nvp.rhs("advdiff2d", wa.dim, wa.params[:3])
    for form, work, kernel in ((0, 4097 * (3 * 1024 + 7 * 4096), "advdiff_window_kernel<float>"),
                               (1, 4097 * 4096 * 10, "advdiff_block_kernel<float>")):
        nvp.tune_set(15, form)
        try:
            maps = nvp.build_propagators(ra, wa.t0, wa.T, wa.S, nvp.samples("affine"),
                                         nvp.steps("rk4", wa.dt, 0, "fp32"))
        finally:
            nvp.tune_set(15, 0)
        d = nvp.maps_info(maps)
        assert (d.work_per_slice, d.build_kernel.decode(), d.band) == (work, kernel, 0)
        maps.destroy()


@pytest.mark.parametrize("form", [3, 4, 5])
def test_heat_window_refused_when_none_fits(form):
    """Forms 3, 4 and 5 with no built window holding 8m+1 rows within n are
    refused by the build with NV_ENOTSUP (n = 96, m = 11 needs 89 rows; the
    single windows are 32, 64, 88, 128, 176 and 256 rows, the two-phase ones
    end at 88 and 128, the three-phase one at 88)."""
    torch = need_gpu()
    n, S, steps = 96, 2, 11
    T = S * steps * 2.0 / (5.0 * (n + 1) ** 2)
    w = workloads.heat1d(n=n, S=S, T=T, dt=T / (S * steps))
    nvp.tune_set(6, form)
    try:
        with pytest.raises(nvp.NvError) as ei:
            _heat(torch, w, "fp64")
        assert ei.value.status == nvp.NV_ENOTSUP
    finally:
        nvp.tune_set(6, 0)


def test_heat_small_fp32():
    torch = need_gpu()
    w = workloads.heat1d(n=40, S=7, T=0.003, dt=1e-4)
    _, A, b, yT, lam = _heat(torch, w, "fp32")
    m = nv.workload_steps(w)
    oA, ob = nv.build_affine(nv.workload_rhs(w, True), nv.workload_rhs(w, False), "rk4",
                             w.t0, w.T, w.S, m, w.dim)
    assert rel_max(A, oA) <= 1e-5
    olam = nv.compose_affine(oA, ob, w.y0)
    assert rel_l2(yT, olam[-1]) <= 1e-5


def test_heat_varcoef_small():
    """Section 5's variable-coefficient heat equation: time-dependent operator,
    so every column takes the literal RK4 stages."""
    torch = need_gpu()
    n = 19
    w = workloads.Workload("v", "heat1d_varcoef", n, 0.0, 1.0, 5, "rk4", 1e-3, 0, "affine",
                           y0=np.sin(np.pi * nv.heat1d_grid(n)))
    _, A, b, yT, lam = _heat(torch, w, "fp64", "heat1d_varcoef")
    m = nv.workload_steps(w)
    fi, fh = nv.workload_rhs(w, True), nv.workload_rhs(w, False)
    oA, ob = nv.build_affine(fi, fh, "rk4", w.t0, w.T, w.S, m, n)
    assert rel_max(A, oA) <= 1e-11 and rel_max(b, ob) <= 1e-11
    assert rel_l2(yT, nv.compose_affine(oA, ob, w.y0)[-1]) <= 1e-11


_FULL = {}


def _full_oracle():
    """Heat equation at full size (n=256, S=1024, m=10): sampled slices of the
    oracle's maps and its serial fine solve (equal to the composed maps up to
    rounding, end of Section 4)."""
    if not _FULL:
        w = workloads.heat1d()
        m = nv.workload_steps(w)
        fi, fh = nv.workload_rhs(w, True), nv.workload_rhs(w, False)
        _FULL["w"] = w
        _FULL["slices"] = {j: nv.build_affine_slice(fi, fh, "rk4", w.t0, w.T, w.S, m, w.dim, j)
                           for j in (0, 517, 1023)}
        _FULL["serial"] = nv.serial_fine(fi, "rk4", w.t0, w.T, w.S, m, w.y0)
    return _FULL


@pytest.mark.parametrize("prec,tol,final_tol", [("fp64", 1e-11, 6e-14), ("fp32", 1e-5, 2e-4),
                                                ("fp32_refine", 1e-5, 1e-8)])
def test_heat_full_size(prec, tol, final_tol):
    """n=256, S=1024 slices, RK4 with m=10: three whole slice maps element by
    element, and the composed final state against the serial fine solve.

    float64 final state: 6e-14.  The nine-point form of the step maps smooth
    modes to themselves only if its weights satisfy c0 + 2 (c1 + .. + c4) = 1;
    with the weights merely rounded that sum is off by an ulp and the 10 240
    steps drift by 1.0e-13, which this bound rejects; with c4 absorbing the
    exact residual the drift is gone (2.4e-14 measured).

    float32 final state: the 1024 maps of this constant-coefficient problem
    are bitwise identical, so their float32 rounding composes coherently:
    rounding the exact maps to float32 alone gives 1.0e-5, computing them in
    float32 ~4e-5 (bound S * m * u32 * O(1) ~ 6e-4).  The bound here is 2e-4;
    the refined paths are the ones held to the method's target.  With one
    float64 correction pass (fp32_refine: defects from the float32 boundary
    states, the correction chained over the same float32 maps) the error
    contracts by about S times the maps' float32 rounding: 7.5e-10 measured,
    bound 1e-8."""
    torch = need_gpu()
    o = _full_oracle()
    w = o["w"]
    _, A, b, yT, lam = _heat(torch, w, prec)
    for j, (oA, ob) in o["slices"].items():
        assert rel_max(A[j], oA) <= tol, j
        assert rel_max(b[j], ob) <= tol, j
    print(prec, "final state relative error", rel_l2(yT, o["serial"]))
    assert rel_l2(yT, o["serial"]) <= final_tol
    assert rel_l2(lam[-1], yT) == 0.0


def test_heat_fp32_two_passes_reach_float64_error():
    """Full size: float32 maps + two float64 correction passes land at the
    float64 method's own error level against the serial fine solve (9.4e-15
    and 2.4e-14 measured; bound 5e-14), the equal-error point of the
    mixed-precision form."""
    torch = need_gpu()
    o = _full_oracle()
    w = o["w"]
    nvp.tune_set(5, 2)
    try:
        _, A, b, yT, lam = _heat(torch, w, "fp32_refine")
    finally:
        nvp.tune_set(5, 0)
    err = rel_l2(yT, o["serial"])
    print("fp32 + 2 passes final state relative error", err)
    assert err <= 5e-14


@pytest.mark.parametrize("n,S", [(40, 7), (256, 9), (100, 5)])
def test_heat_fp32_refined_small(n, S):
    """float32 maps + one float64 correction pass, every boundary state: the
    cluster chain (d = 256), and the fallback cluster chain (d = 40, 100)."""
    torch = need_gpu()
    dt = 2.0 / (4.0 * (n + 1) ** 2)
    w = workloads.heat1d(n=n, S=S, T=S * 3 * dt, dt=dt)
    _, A, b, yT, lam = _heat(torch, w, "fp32_refine")
    m = nv.workload_steps(w)
    fi, fh = nv.workload_rhs(w, True), nv.workload_rhs(w, False)
    oA, ob = nv.build_affine(fi, fh, "rk4", w.t0, w.T, w.S, m, n)
    assert rel_max(A, oA) <= 1e-5
    olam = nv.compose_affine(oA, ob, w.y0)
    assert rel_l2(lam, olam) <= 1e-9


def _refine_both_schedules(torch, w, passes, rhs_name="heat1d"):
    """Boundary states and final state of NV_FP32_REFINE with `passes` passes,
    pipelined (tunable 10 = 0) and one pass after another (10 = 1)."""
    r = nvp.rhs(rhs_name, w.dim, w.params if rhs_name == "heat1d" else ())
    maps = nvp.build_propagators(r, w.t0, w.T, w.S, nvp.samples("affine"),
                                 nvp.steps("rk4", w.dt, w.steps_per_slice, "fp32_refine"))
    y0 = torch.tensor(w.y0, dtype=torch.float64, device="cuda")
    out = {}
    try:
        nvp.tune_set(5, passes)
        for sched in (1, 0):
            nvp.tune_set(10, sched)
            yT = torch.empty_like(y0)
            lam = torch.full((w.S + 1, w.dim), float("nan"), dtype=torch.float64, device="cuda")
            nvp.compose(maps, y0, yT, lambdas=lam)
            nvp.maps_check(maps)
            out[sched] = (yT.cpu(), lam.cpu())
    finally:
        nvp.tune_set(5, 0)
        nvp.tune_set(10, 0)
        maps.destroy()
    return out


@pytest.mark.parametrize("passes", [1, 2, 3])
def test_heat_fp32_refine_pipelined_matches_sequential_full_size(passes):
    """n = 256, S = 1024: the pipelined schedule (approximate chain, defects
    and every correction chain concurrently in one cooperative launch) gives
    the sequential passes' boundary states and final state bit for bit, and
    two or more passes reach the float64 method's error level."""
    torch = need_gpu()
    o = _full_oracle()
    out = _refine_both_schedules(torch, o["w"], passes)
    assert torch.equal(out[0][0], out[1][0])
    assert torch.equal(out[0][1], out[1][1])
    err = rel_l2(out[0][0].numpy(), o["serial"])
    print(passes, "passes, pipelined, final state relative error", err)
    assert err <= (1e-8 if passes == 1 else 5e-14)


@pytest.mark.parametrize("n,S,passes,rhs_name", [(64, 7, 2, "heat1d"), (96, 2, 1, "heat1d"),
                                                 (128, 1, 3, "heat1d"), (256, 9, 2, "heat1d"),
                                                 (64, 33, 1, "heat1d_varcoef")])
def test_heat_fp32_refine_pipelined_small(n, S, passes, rhs_name):
    """Shapes of the pipelined schedule: two, four and eight rows per lane in
    the defect warps, chains shorter than the number of passes, the
    variable-coefficient equation.  Bit-identical to the sequential passes and
    within 1e-9 of the oracle's composition of its own maps."""
    torch = need_gpu()
    dt = 2.0 / (4.0 * 1.25 * (n + 1) ** 2)       # stable for diffusion coefficients up to 1.25
    if rhs_name == "heat1d":
        w = workloads.heat1d(n=n, S=S, T=S * 3 * dt, dt=dt)
    else:
        w = workloads.Workload("v", "heat1d_varcoef", n, 0.0, S * 3 * dt, S, "rk4", dt, 0, "affine",
                               y0=np.sin(np.pi * nv.heat1d_grid(n)))
    out = _refine_both_schedules(torch, w, passes, rhs_name)
    assert torch.equal(out[0][0], out[1][0])
    assert torch.equal(out[0][1], out[1][1])
    m = nv.workload_steps(w)
    fi, fh = nv.workload_rhs(w, True), nv.workload_rhs(w, False)
    oA, ob = nv.build_affine(fi, fh, "rk4", w.t0, w.T, w.S, m, n)
    olam = nv.compose_affine(oA, ob, w.y0)
    assert rel_l2(out[0][1].numpy(), olam) <= 1e-9


def test_pipelined_refinement_bounded_wait_reports_timeout_and_context_survives():
    """Failure detection of the pipelined refinement without a GPU fault: a
    test hook (tunable 12) keeps one defect's flag unset, so the correction
    chain's bounded wait for it runs out; the launch records NV_ETIMEOUT, which
    nv_maps_check reports, and every role gives up (the launch ends in about
    a second).  The next composition on the same maps and context matches the
    sequential passes bit for bit."""
    torch = need_gpu()
    import time
    n, S = 128, 40
    dt = 2.0 / (4.0 * 1.25 * (n + 1) ** 2)
    w = workloads.heat1d(n=n, S=S, T=S * 3 * dt, dt=dt)
    r = nvp.rhs("heat1d", w.dim, w.params)
    maps = nvp.build_propagators(r, w.t0, w.T, w.S, nvp.samples("affine"),
                                 nvp.steps("rk4", w.dt, w.steps_per_slice, "fp32_refine"))
    y0 = torch.tensor(w.y0, dtype=torch.float64, device="cuda")
    yT = torch.empty_like(y0)
    try:
        nvp.tune_set(5, 2)
        nvp.tune_set(12, 6)                       # withhold pass 1's defect of slice 5
        t0 = time.time()
        nvp.compose(maps, y0, yT)
        with pytest.raises(nvp.NvError) as exc:
            nvp.maps_check(maps)
        elapsed = time.time() - t0
        assert exc.value.status == nvp.NV_ETIMEOUT
        assert elapsed < 10.0
        nvp.tune_set(12, 0)
        out = {}
        for sched in (0, 1):
            nvp.tune_set(10, sched)
            y = torch.empty_like(y0)
            nvp.compose(maps, y0, y)
            nvp.maps_check(maps)
            out[sched] = y.cpu()
        assert torch.equal(out[0], out[1])
    finally:
        nvp.tune_set(12, 0)
        nvp.tune_set(10, 0)
        nvp.tune_set(5, 0)
        maps.destroy()


def test_heat_serial_fine_gpu():
    torch = need_gpu()
    w = workloads.heat1d(n=40, S=7, T=0.003, dt=1e-4)
    r = nvp.rhs("heat1d", w.dim, w.params)
    st = nvp.steps("rk4", w.dt)
    y0 = torch.tensor(w.y0, dtype=torch.float64, device="cuda")
    ys = torch.empty_like(y0)
    nvp.serial_fine(r, w.t0, w.T, w.S, st, y0, ys)
    ser = nv.serial_fine(nv.workload_rhs(w, True), "rk4", w.t0, w.T, w.S, nv.workload_steps(w), w.y0)
    assert rel_l2(ys.cpu().numpy(), ser) <= 1e-11


@pytest.mark.parametrize("cluster,rpc", [(2, 0), (4, 0), (8, 0), (16, 0), (-1, 1), (-1, 4), (-1, 32), (-1, 64)])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_chain_launch_shapes(cluster, rpc, prec, tol):
    """The composition does not depend on how the chain is laid out: one
    cluster of 2..16 CTAs exchanging lambda through distributed shared memory,
    or the grid-wide chain with 1..64 rows per CTA."""
    torch = need_gpu()
    w = workloads.heat1d(n=97, S=9, T=0.003, dt=5e-5)
    try:
        nvp.tune_set(3, cluster)
        nvp.tune_set(1, rpc)
        _, A, b, yT, lam = _heat(torch, w, prec)
    finally:
        nvp.tune_set(3, 0)
        nvp.tune_set(1, 0)
    m = nv.workload_steps(w)
    oA, ob = nv.build_affine(nv.workload_rhs(w, True), nv.workload_rhs(w, False), "rk4",
                             w.t0, w.T, w.S, m, w.dim)
    assert rel_l2(lam, nv.compose_affine(oA, ob, w.y0)) <= tol


def test_bounded_barrier_wait_reports_timeout_and_context_survives():
    """A grid barrier that nothing completes (test hook: one participant that
    never arrives) makes every CTA of the row chain give up at its bounded
    wait; the status word reports NV_ETIMEOUT, and the next composition on the
    same maps and context is correct."""
    torch = need_gpu()
    w = workloads.heat1d(n=40, S=7, T=0.003, dt=5e-5)
    r = nvp.rhs("heat1d", w.dim, w.params)
    maps = nvp.build_propagators(r, w.t0, w.T, w.S, nvp.samples("affine"), nvp.steps("rk4", w.dt))
    y0 = torch.tensor(w.y0, device="cuda")
    yT = torch.empty_like(y0)
    nvp.tune_set(3, -1)
    try:
        nvp.tune_set(7, 1)
        try:
            nvp.compose(maps, y0, yT)
            with pytest.raises(nvp.NvError) as ei:
                nvp.maps_check(maps)
            assert ei.value.status == nvp.NV_ETIMEOUT
        finally:
            nvp.tune_set(7, 0)
        nvp.compose(maps, y0, yT)
        nvp.maps_check(maps)
    finally:
        nvp.tune_set(3, 0)
    m = nv.workload_steps(w)
    fi, fh = nv.workload_rhs(w, True), nv.workload_rhs(w, False)
    oA, ob = nv.build_affine(fi, fh, "rk4", w.t0, w.T, w.S, m, w.dim)
    assert rel_l2(yT.cpu().numpy(), nv.compose_affine(oA, ob, w.y0)[-1]) <= 1e-11
    maps.destroy()
