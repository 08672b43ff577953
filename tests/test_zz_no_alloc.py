"""The allocation-free affine composition (nv_compose_affine_noalloc).

It exists for callers that cannot allocate device memory when they compose
(an application whose memory pool already owns the GPU, a real-time loop that
must not pay for cudaMalloc/cudaFree, a plug-in limited to the buffers it is
lent).  Its scratch is a fixed static device array shared by every call, so
these checks make two calls in a row on one stream and compare each with the
regular nv_compose on the same maps, within the float64 tolerance the parity
tests use (1e-11), and at the size limit (d = 4096) every boundary state
with the oracle's serial fine solve.  The file sorts last so that a run
stopping at the first failure has run every other test before it."""
import numpy as np
import pytest

import paper_1304_6514_gb300 as nvp
import workloads
from oracle import nievergelt as nv

from gpu_util import need_gpu, rel_l2


def test_noalloc_rejects_oversized_dim_on_host():
    """dim beyond the static scratch is refused before anything is launched."""
    from paper_1304_6514_gb300 import _build
    _build.build()
    lib = nvp.load_library()
    st = lib.nv_compose_affine_noalloc(1, 0, 4097, 4, 1, 1, None, None, None)
    assert st == nvp.NV_EINVAL
    assert "4096" in nvp.last_error()


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_noalloc_matches_compose_twice(prec, tol):
    """float32 maps: nv_compose may compose them in float32 arithmetic, this
    entry point accumulates in float64, so they agree to the float32
    tolerance of the other tests."""
    torch = need_gpu()
    w = workloads.heat1d(n=97, S=9, T=0.003, dt=5e-5)
    maps = nvp.build_propagators(nvp.rhs("heat1d", w.dim, w.params), w.t0, w.T, w.S,
                                 nvp.samples("affine"), nvp.steps("rk4", w.dt, 0, prec))
    y0 = torch.tensor(w.y0, dtype=torch.float64, device="cuda")
    yT_ref = torch.empty_like(y0)
    lam_ref = torch.empty((w.S + 1, w.dim), dtype=torch.float64, device="cuda")
    nvp.compose(maps, y0, yT_ref, lam_ref)
    nvp.maps_check(maps)
    maps_dev = nvp.maps_data(maps)              # caller-owned copy of the map data
    torch.cuda.synchronize()

    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for call in range(2):
        yT = torch.full_like(y0, float("nan"))
        lam = torch.full_like(lam_ref, float("nan"))
        status.fill_(-1)
        nvp.compose_affine_noalloc(maps_dev, prec, w.dim, w.S, y0, yT, lam, status)
        torch.cuda.synchronize()
        assert int(status.item()) == nvp.NV_OK, call
        assert rel_l2(yT.cpu().numpy(), yT_ref.cpu().numpy()) <= tol, call
        assert rel_l2(lam.cpu().numpy(), lam_ref.cpu().numpy()) <= tol, call
    maps.destroy()


@pytest.mark.gpu
def test_noalloc_full_size_heat():
    """The benchmark's heat maps (n = 256, S = 1024): same final state as
    nv_compose, twice in a row."""
    torch = need_gpu()
    w = workloads.heat1d()
    maps = nvp.build_propagators(nvp.rhs("heat1d", w.dim, w.params), w.t0, w.T, w.S,
                                 nvp.samples("affine"), nvp.steps("rk4", w.dt))
    y0 = torch.tensor(w.y0, dtype=torch.float64, device="cuda")
    yT_ref = torch.empty_like(y0)
    nvp.compose(maps, y0, yT_ref)
    maps_dev = nvp.maps_data(maps)
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for call in range(2):
        yT = torch.full_like(y0, float("nan"))
        status.fill_(-1)
        nvp.compose_affine_noalloc(maps_dev, "fp64", w.dim, w.S, y0, yT, None, status)
        torch.cuda.synchronize()
        assert int(status.item()) == nvp.NV_OK, call
        assert np.all(np.isfinite(yT.cpu().numpy()))
        assert rel_l2(yT.cpu().numpy(), yT_ref.cpu().numpy()) <= 1e-11, call
    maps.destroy()


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_noalloc_at_size_limit_against_oracle(prec, tol):
    """At the documented limit d = 4096 (the 64 x 64 advection-diffusion maps,
    S = 3 slices, RK4 m = 10): the static scratch is full and the cooperative
    chain runs 256 CTAs.  Two calls in a row on one stream; every boundary
    state against the oracle's float64 serial fine solve at the slice ends
    (the composed affine maps equal it to rounding, end of Section 4) and
    against nv_compose on the same maps; the status word reads NV_OK.
    float32 maps: the float32 rounding of their entries over three slices
    stays within the float32 tolerance."""
    torch = need_gpu()
    w = workloads.advdiff2d(S=3, T=3 / 512)
    assert w.dim == 4096                     # NVPIT_NOALLOC_MAX_DIM
    m = nv.workload_steps(w)
    h = nv.step_size(w.t0, w.T, w.S, m)
    f = nv.workload_rhs(w, True)
    Tj = nv.slice_times(w.t0, w.T, w.S)
    ref = [np.asarray(w.y0, dtype=np.float64)]
    for j in range(w.S):
        ref.append(nv.integrate(f, "rk4", Tj[j], ref[-1][:, None], h, m)[:, 0])
    ref = np.array(ref)

    maps = nvp.build_propagators(nvp.rhs("advdiff2d", w.dim, w.params[:3]), w.t0, w.T, w.S,
                                 nvp.samples("affine"), nvp.steps("rk4", w.dt, 0, prec))
    y0 = torch.tensor(w.y0, dtype=torch.float64, device="cuda")
    yT_c = torch.empty_like(y0)
    lam_c = torch.empty((w.S + 1, w.dim), dtype=torch.float64, device="cuda")
    nvp.compose(maps, y0, yT_c, lam_c)
    nvp.maps_check(maps)
    maps_dev = nvp.maps_data(maps)
    torch.cuda.synchronize()
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for call in range(2):
        yT = torch.full_like(y0, float("nan"))
        lam = torch.full_like(lam_c, float("nan"))
        status.fill_(-1)
        nvp.compose_affine_noalloc(maps_dev, prec, w.dim, w.S, y0, yT, lam, status)
        torch.cuda.synchronize()
        assert int(status.item()) == nvp.NV_OK, call
        lam_h = lam.cpu().numpy()
        for j in range(w.S + 1):
            assert rel_l2(lam_h[j], ref[j]) <= tol, (call, j, rel_l2(lam_h[j], ref[j]))
        assert rel_l2(yT.cpu().numpy(), ref[-1]) <= tol, call
        assert rel_l2(lam_h, lam_c.cpu().numpy()) <= tol, call
    maps.destroy()
