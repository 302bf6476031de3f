"""The pipe-throughput probe behind the ALU roofline's peak returns issue
rates in the range a Blackwell SM can have (at most four warp instructions per
clock: one per scheduler)."""
import pytest

import paper_1708_09746_gb300 as G

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def test_probe_pipes_plausible():
    need_gpu()
    r = G.gf2x_probe_pipes()
    assert r["sms"] > 0
    for k in ("shfl_per_clk_sm", "xor_per_clk_sm", "lds_per_clk_sm"):
        assert 0.05 < r[k] <= 4.0, (k, r)
