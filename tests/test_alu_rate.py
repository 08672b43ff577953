"""The measured FMA rate the ALU-bound builds are reported against
(nv_alu_rate): a GB300's float64 and float32 pipes land near their nominal
rates (152 SMs x 2 FP64 / 128 FP32 FMA lanes x 2 FLOP x ~2 GHz)."""
import pytest

import paper_1304_6514_gb300 as nvp

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,nominal", [("fp64", 1.26e12), ("fp32", 80.5e12)])
def test_alu_rate_is_near_the_nominal_rate(prec, nominal):
    need_gpu()
    rate = nvp.alu_rate(prec)
    assert 0.6 * nominal < rate < 1.2 * nominal, rate
