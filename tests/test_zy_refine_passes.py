"""Error of the tensor-core composition of the full heat-equation workload
(n = 256, S = 1024) against the serial fine solve, before refinement and after
1, 2 and 3 float64 correction passes.  Each pass must contract the error."""
import pytest

import paper_1304_6514_gb300 as nvp
import workloads
from oracle import nievergelt as nv

from gpu_util import need_gpu, rel_l2

pytestmark = pytest.mark.gpu


def test_refinement_passes_contract_full_size():
    torch = need_gpu()
    w = workloads.heat1d()
    m = nv.workload_steps(w)
    ser = nv.serial_fine(nv.workload_rhs(w, True), "rk4", w.t0, w.T, w.S, m, w.y0)
    maps = nvp.build_propagators(nvp.rhs("heat1d", w.dim, w.params), w.t0, w.T, w.S,
                                 nvp.samples("affine"), nvp.steps("rk4", w.dt, 0, "tf32_refine"))
    y0 = torch.tensor(w.y0, dtype=torch.float64, device="cuda")
    errs = []
    try:
        for passes in (-1, 1, 2, 3):
            nvp.tune_set(5, passes)
            yT = torch.empty_like(y0)
            nvp.compose(maps, y0, yT)
            nvp.maps_check(maps)
            errs.append(rel_l2(yT.cpu().numpy(), ser))
    finally:
        nvp.tune_set(5, 0)
    print("errors before / after 1, 2, 3 passes:", errs)
    for i in range(3):
        assert errs[i + 1] < 0.5 * errs[i] or errs[i + 1] < 1e-9, errs
