"""The autotuner on the GPU: it returns parameters in range and a time, and a
product made with any parameters (tuned or forced) is still bit-exact."""
import numpy as np
import pytest

import paper_1708_09746_gb300 as G
from oracle import product as P
import workloads as W

from gpu_util import gpu_mul, need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def test_autotune_picks_valid_parameters_and_keeps_parity():
    na, nb = 1 << 22, (1 << 22) - 77
    best = G.gf2x_autotune(na, nb, reps=2)
    assert 4 <= best["fft_depth"] <= 7
    assert best["fft_buffers"] in (1, 2)
    assert best["bcvt_tile_log"] in (10, 11, 12, 13)
    assert best["bcvt_threads"] in (128, 256, 512)
    assert best["ms"] > 0
    assert G.gf2x_tune_get(na, nb) == best
    a, b = W.operand_pair(31, na, nb)
    assert np.array_equal(gpu_mul(a, na, b, nb), P.mul(a, na, b, nb))


@pytest.mark.parametrize("params", [(4, 1, 10, 128), (5, 2, 13, 512), (6, 1, 4, 32),
                                    (1, 1, 14, 64), (7, 1, 11, 256)])
def test_forced_parameters_keep_parity(params):
    # 2^24-bit operands: 7 FFT layers above the 4096-point tile, so the fusion
    # depth changes the number and split of the strided passes
    na, nb = (1 << 24) - 5, (1 << 23) + 9
    G.gf2x_tune_set(na, nb, *params)
    a, b = W.operand_pair(32 + params[0], na, nb)
    got = gpu_mul(a, na, b, nb)
    G.gf2x_tune_set(na, nb, 7, 2, 11, 256)
    assert np.array_equal(got, P.mul(a, na, b, nb))
