"""GPU parity of the refined tensor-core composition (NV_TF32_REFINE):
float32 maps, block totals as tcgen05 TF32 products, batched cluster chains,
then float64 residual-correction passes (three by default).  Target after refinement: relative
L2 error of the boundary states <= 1e-4 against the FP64 oracle."""
import numpy as np
import pytest

import paper_1304_6514_gb300 as nvp
import workloads
from oracle import nievergelt as nv

from gpu_util import need_gpu, rel_l2

pytestmark = pytest.mark.gpu


def _run(torch, w, block=0):
    try:
        nvp.tune_set(4, block)
        r = nvp.rhs("heat1d", w.dim, w.params)
        maps = nvp.build_propagators(r, w.t0, w.T, w.S, nvp.samples("affine"),
                                     nvp.steps("rk4", w.dt, 0, "tf32_refine"))
        y0 = torch.tensor(w.y0, dtype=torch.float64, device="cuda")
        yT = torch.empty_like(y0)
        lam = torch.empty((w.S + 1, w.dim), dtype=torch.float64, device="cuda")
        nvp.compose(maps, y0, yT, lam)
        nvp.maps_check(maps)
        return yT.cpu().numpy(), lam.cpu().numpy()
    finally:
        nvp.tune_set(4, 0)


def _oracle_states(w):
    m = nv.workload_steps(w)
    A, b = nv.build_affine(nv.workload_rhs(w, True), nv.workload_rhs(w, False), "rk4",
                           w.t0, w.T, w.S, m, w.dim)
    return nv.compose_affine(A, b, w.y0)


@pytest.mark.parametrize("n,S,block", [(64, 37, 0), (100, 12, 5), (200, 9, 0), (128, 16, 1),
                                       (256, 8, 8), (32, 5, 2), (4, 3, 0)])
def test_refined_scan_small(n, S, block):
    """Ragged slab counts (d = 100, 200), one and two row halves, the last
    block shorter than the others, one block (L = S) and one slice per block."""
    torch = need_gpu()
    w = workloads.heat1d(n=n, S=S, T=S * 4e-4, dt=2.0 / (4.0 * (n + 1) ** 2))
    yT, lam = _run(torch, w, block)
    olam = _oracle_states(w)
    assert rel_l2(lam, olam) <= 1e-4
    assert rel_l2(yT, olam[-1]) <= 1e-4


def test_refined_scan_full_size():
    """n = 256, S = 1024 (the benchmark workload) against the serial fine
    solve; the refined error is far below the float32 maps' own 5e-5."""
    torch = need_gpu()
    w = workloads.heat1d()
    m = nv.workload_steps(w)
    ser = nv.serial_fine(nv.workload_rhs(w, True), "rk4", w.t0, w.T, w.S, m, w.y0)
    yT, lam = _run(torch, w)
    err = rel_l2(yT, ser)
    print("refined relative error", err)
    assert err <= 1e-4
    assert rel_l2(lam[-1], yT) == 0.0


def test_refined_scan_rejects_unsupported_sizes():
    torch = need_gpu()
    for n in (97, 300):
        w = workloads.heat1d(n=n, S=4, T=1e-4, dt=1e-6)
        with pytest.raises(nvp.NvError) as e:
            _run(torch, w)
        assert e.value.status == nvp.NV_ENOTSUP
