"""GPU parity of the large linear system: periodic 2-D advection-diffusion on
a 64 x 64 grid (d = 4096), exact affine maps from 4097 basis solves, chain
composition over all SMs.  Sampled map columns against the oracle's basis
solves, composed state against the serial fine solve (end of Section 4)."""
import numpy as np
import pytest

import paper_1304_6514_gb300 as nvp
import workloads
from oracle import nievergelt as nv

from gpu_util import need_gpu, rel_l2, rel_max

pytestmark = pytest.mark.gpu

COLS = [0, 1, 63, 64, 2047, 4095, 4096]          # map columns: 0 is b_j, c >= 1 is A_j e_{c-1}


def _check(torch, w, prec, slices, tol_cols, tol_final):
    r = nvp.rhs("advdiff2d", w.dim, w.params[:3])
    maps = nvp.build_propagators(r, w.t0, w.T, w.S, nvp.samples("affine"),
                                 nvp.steps("rk4", w.dt, 0, prec))
    y0 = torch.tensor(w.y0, dtype=torch.float64, device="cuda")
    yT = torch.empty_like(y0)
    nvp.compose(maps, y0, yT)
    nvp.maps_check(maps)
    n = w.dim
    m = nv.workload_steps(w)
    fi, fh = nv.workload_rhs(w, True), nv.workload_rhs(w, False)
    for j in slices:
        blk = nvp.maps_slice(maps, j).double().cpu().numpy().reshape(n + 1, n)      # [col, row]
        assert np.all(blk[0] == 0.0)                                        # no forcing: b_j = 0
        Ac, _ = nv.build_affine_slice(fi, fh, "rk4", w.t0, w.T, w.S, m, n, j,
                                      columns=[c - 1 for c in COLS[1:]])
        assert rel_max(blk[COLS[1:]].T, Ac) <= tol_cols, j
    ser = nv.serial_fine(fi, "rk4", w.t0, w.T, w.S, m, w.y0)
    err = rel_l2(yT.cpu().numpy(), ser)
    print(prec, "final state relative error", err)
    assert err <= tol_final
    ys = torch.empty_like(y0)
    nvp.serial_fine(r, w.t0, w.T, w.S, nvp.steps("rk4", w.dt), y0, ys)
    assert rel_l2(ys.cpu().numpy(), ser) <= 1e-11
    maps.destroy()


def test_advdiff_small_fp64():
    torch = need_gpu()
    w = workloads.advdiff2d(S=3, T=3 * 2e-3)
    _check(torch, w, "fp64", [0, 1, 2], 1e-11, 1e-11)


def test_advdiff_full_size_fp32():
    """S = 512 slices (t in [0,1]), float32 maps (34.4 GB).  The 512 maps of
    this constant-coefficient problem are identical, so float32 rounding adds
    up coherently (as for the heat equation): 8.6e-5 measured.  Plain float32
    maps therefore miss the float32 target (1e-5 on the final state); the
    bound 2e-4 here is that documented floor, and the float32 target is held
    by the refined path (test_advdiff_fp32_refined_full_size, 1e-7)."""
    torch = need_gpu()
    _check(torch, workloads.advdiff2d(), "fp32", [0, 255, 511], 1e-5, 2e-4)


def test_advdiff_full_size_fp64():
    """S = 512 slices, float64 maps (68.7 GB)."""
    torch = need_gpu()
    _check(torch, workloads.advdiff2d(), "fp64", [0, 511], 1e-11, 1e-11)


def test_advdiff_bf16_refined_small():
    """bfloat16 maps (entries within 2^-9 of the float32 solves) composed over
    3 slices, then the float64 correction passes: the refined state meets the
    1e-4 target for refined reduced precision, and refinement beats the
    unrefined bfloat16 chain."""
    torch = need_gpu()
    w = workloads.advdiff2d(S=3, T=3 * 2e-3)
    nvp.tune_set(5, -1)
    try:
        r = nvp.rhs("advdiff2d", w.dim, w.params[:3])
        maps = nvp.build_propagators(r, w.t0, w.T, w.S, nvp.samples("affine"),
                                     nvp.steps("rk4", w.dt, 0, "bf16_refine"))
        y0 = torch.tensor(w.y0, dtype=torch.float64, device="cuda")
        y_raw = torch.empty_like(y0)
        nvp.compose(maps, y0, y_raw)
        nvp.maps_check(maps)
        maps.destroy()
    finally:
        nvp.tune_set(5, 0)
    _check(torch, w, "bf16_refine", [0, 2], 4e-3, 1e-4)
    m = nv.workload_steps(w)
    ser = nv.serial_fine(nv.workload_rhs(w, True), "rk4", w.t0, w.T, w.S, m, w.y0)
    print("unrefined bfloat16 chain relative error", rel_l2(y_raw.cpu().numpy(), ser))
    assert rel_l2(y_raw.cpu().numpy(), ser) > 1e-4


def test_advdiff_bf16_refined_32_slices():
    """32 slices: the bfloat16 rounding compounds along the chain (the slowly
    decaying modes, the mean among them, keep it), but the two correction
    passes of the default still converge."""
    torch = need_gpu()
    _check(torch, workloads.advdiff2d(S=32, T=32 * 2e-3), "bf16_refine", [0, 31], 4e-3, 1e-4)


def test_advdiff_bf16_refined_full_size():
    """S = 512, bfloat16 maps (17.2 GB) composed by the float32-accumulating
    chain, then the default float64 correction passes for this S (six: each
    pass contracts the error by roughly S / 1500 here, measured 3.4e-2 after
    two passes): the refined final state meets the 1e-4 target for refined
    reduced precision against the oracle's serial fine solve."""
    torch = need_gpu()
    _check(torch, workloads.advdiff2d(), "bf16_refine", [0, 511], 4e-3, 1e-4)


def test_advdiff_fp32_refined_full_size():
    """S = 512, float32 maps (34.4 GB) and chain, one float64 correction pass:
    from the float32 method's 8.8e-5 to float64-level agreement with the serial
    fine solve."""
    torch = need_gpu()
    _check(torch, workloads.advdiff2d(), "fp32_refine", [0, 511], 1e-5, 1e-7)


@pytest.mark.parametrize("S,m", [(3, 10), (2, 1), (2, 2), (4, 3), (3, 4), (5, 7)])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16_refine"])
def test_advdiff_window_build_matches_whole_grid(prec, S, m):
    """The float64 / float32 / bfloat16 build integrates the first min(m, 3) steps of
    each column on a 32 x 32 window around its unit point (the points those
    steps cannot reach are exactly zero) and the rest on the whole periodic
    grid: every map entry equals the whole-grid build's (tunable 15 = 1) bit
    for bit, for every column of every slice (windows across the periodic
    seams included), with m = 10 as in the benchmark, m <= 3 (the windows
    only) and m = 4, 7; and the entries farther than 4m points (periodic
    Manhattan distance) from a column's unit point are exactly zero."""
    torch = need_gpu()
    w = workloads.advdiff2d(S=S, T=S * m * 2e-4, dt=2e-4)
    assert nv.workload_steps(w) == m
    r = nvp.rhs("advdiff2d", w.dim, w.params[:3])
    got = {}
    for form in (0, 1):
        nvp.tune_set(15, form)
        try:
            maps = nvp.build_propagators(r, w.t0, w.T, w.S, nvp.samples("affine"),
                                         nvp.steps("rk4", w.dt, 0, prec))
            nvp.maps_check(maps)
            got[form] = nvp.maps_slice(maps, 0, w.S).cpu()
            maps.destroy()
        finally:
            nvp.tune_set(15, 0)
    assert torch.equal(got[0], got[1])
    n = w.dim
    blocks = got[0].double().numpy().reshape(w.S, n + 1, n)    # [slice, column, point]
    assert not np.any(blocks[:, 0])                            # b_j = 0: no forcing
    pts = np.arange(n)
    px, py = pts % 64, pts // 64
    for c in (1, 13, 64, 65, 2080, 4033, 4096):
        cx, cy = (c - 1) % 64, (c - 1) // 64
        dx = np.minimum((px - cx) % 64, (cx - px) % 64)
        dy = np.minimum((py - cy) % 64, (cy - py) % 64)
        assert not np.any(blocks[:, c, dx + dy > 4 * m])


@pytest.mark.parametrize("S", [1, 2, 5])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16_refine"])
def test_tiled_chain_ring_and_register_kernels_agree(prec, S):
    """The d > 512 chain has two kernels with the same arithmetic in the same
    order: loads into registers in batches (tunable 9 = 1) and the
    shared-memory ring fed by bulk copies (9 = 2, the default).  Their boundary
    states agree bit for bit, over column blocks whose last stage is ragged
    (4097 columns over 76 or 38 blocks), for chains shorter than, equal to and
    longer than the ring kernel's three rotating exchange buffers, and the final
    state is the serial fine solve's within the precision's bound."""
    torch = need_gpu()
    w = workloads.advdiff2d(S=S, T=S * 2e-3)
    r = nvp.rhs("advdiff2d", w.dim, w.params[:3])
    maps = nvp.build_propagators(r, w.t0, w.T, w.S, nvp.samples("affine"),
                                 nvp.steps("rk4", w.dt, 0, prec))
    y0 = torch.tensor(w.y0, dtype=torch.float64, device="cuda")
    out = {}
    try:
        for form in (1, 2):
            nvp.tune_set(9, form)
            yT = torch.empty_like(y0)
            lam = torch.full((w.S + 1, w.dim), float("nan"), dtype=torch.float64, device="cuda")
            nvp.compose(maps, y0, yT, lambdas=lam)
            nvp.maps_check(maps)
            out[form] = (yT.cpu(), lam.cpu())
    finally:
        nvp.tune_set(9, 0)
        maps.destroy()
    assert torch.equal(out[1][0], out[2][0])
    assert torch.equal(out[1][1], out[2][1])
    assert torch.equal(out[2][1][-1], out[2][0])
    m = nv.workload_steps(w)
    ser = nv.serial_fine(nv.workload_rhs(w, True), "rk4", w.t0, w.T, w.S, m, w.y0)
    tol = {"fp64": 1e-11, "fp32": 1e-5, "bf16_refine": 1e-4}[prec]
    assert rel_l2(out[2][0].numpy(), ser) <= tol


def test_ring_chain_bounded_wait_reports_timeout_and_context_survives():
    """Failure detection of the d > 512 ring chain (tagged exchange, no grid
    barrier) without a GPU fault: a test hook (tunable 13) keeps the first
    CTA from storing its partials of step 1, so the CTAs that need them give
    up after their bounded wait; NV_ETIMEOUT is reported and the launch ends
    within seconds.  The next composition on the same maps and context matches
    the register kernel bit for bit."""
    torch = need_gpu()
    import time
    w = workloads.advdiff2d(S=3, T=3 * 2e-3)
    r = nvp.rhs("advdiff2d", w.dim, w.params[:3])
    maps = nvp.build_propagators(r, w.t0, w.T, w.S, nvp.samples("affine"),
                                 nvp.steps("rk4", w.dt, 0, "fp64"))
    y0 = torch.tensor(w.y0, dtype=torch.float64, device="cuda")
    yT = torch.empty_like(y0)
    try:
        nvp.tune_set(9, 2)                        # the ring kernel
        nvp.tune_set(13, 2)                       # CTA 0 skips step 1's partials
        t0 = time.time()
        nvp.compose(maps, y0, yT)
        with pytest.raises(nvp.NvError) as exc:
            nvp.maps_check(maps)
        assert exc.value.status == nvp.NV_ETIMEOUT
        assert time.time() - t0 < 10.0
        nvp.tune_set(13, 0)
        out = {}
        for form in (2, 1):
            nvp.tune_set(9, form)
            y = torch.empty_like(y0)
            nvp.compose(maps, y0, y)
            nvp.maps_check(maps)
            out[form] = y.cpu()
        assert torch.equal(out[1], out[2])
    finally:
        nvp.tune_set(13, 0)
        nvp.tune_set(9, 0)
        maps.destroy()


@pytest.mark.parametrize("S,m", [(3, 10), (2, 2), (2, 4), (3, 5), (2, 6), (2, 7)])
def test_advdiff_fp64_window_strip_heights_agree(S, m):
    """The float64 window build with 8-, 16- and 32-row strips (key 16; 512,
    256 and 128 threads per CTA), with the ladder of row windows after the
    first three steps (key 15 = 0: 40, 48, 56 rows for steps 4-6 at 8-row
    strips, 48 rows for steps 4-5 at 16) and without it (key 15 = 2), computes
    every point with the same expression as the whole-grid kernel (key 15 = 1):
    the maps agree bit for bit, for m covering partial and whole ladders."""
    torch = need_gpu()
    w = workloads.advdiff2d(S=S, T=S * m * 2e-4, dt=2e-4)
    r = nvp.rhs("advdiff2d", w.dim, w.params[:3])
    got = {}
    for rows, form in ((16, 1), (8, 0), (16, 0), (32, 0), (8, 2), (16, 2)):
        nvp.tune_set(16, rows)
        nvp.tune_set(15, form)
        try:
            maps = nvp.build_propagators(r, w.t0, w.T, w.S, nvp.samples("affine"), nvp.steps("rk4", w.dt))
            nvp.maps_check(maps)
            name = nvp.maps_info(maps).build_kernel.decode()
            assert name == (f"advdiff_window64_kernel<{rows}>" if form != 1 else "advdiff_affine_kernel<double>")
            got[(rows, form)] = nvp.maps_slice(maps, 0, w.S).cpu()
            maps.destroy()
        finally:
            nvp.tune_set(16, 0)
            nvp.tune_set(15, 0)
    ref = got[(16, 1)]
    for key, val in got.items():
        assert torch.equal(val, ref), key
