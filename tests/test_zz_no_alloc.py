"""The allocation-free affine composition (nv_compose_affine_noalloc).

It exists for callers that cannot allocate device memory when they compose
(an application whose memory pool already owns the GPU, a real-time loop that
must not pay for cudaMalloc/cudaFree, a plug-in limited to the buffers it is
lent).  Its scratch is a fixed static device array shared by every call, so
these checks make two calls in a row on one stream and compare each with the
regular nv_compose on the same maps, within the float64 tolerance the parity
tests use (1e-11).  The file sorts last so that a run stopping at the first
failure has run every other test before it."""
import numpy as np
import pytest

import paper_1304_6514_gb300 as nvp
import workloads

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
    for call in range(2):
        yT = torch.full_like(y0, float("nan"))
        nvp.compose_affine_noalloc(maps_dev, "fp64", w.dim, w.S, y0, yT)
        torch.cuda.synchronize()
        assert np.all(np.isfinite(yT.cpu().numpy()))
        assert rel_l2(yT.cpu().numpy(), yT_ref.cpu().numpy()) <= 1e-11, call
    maps.destroy()
