"""Argument checks of the other forms' entry points (F~_{2^256}, simple,
Frobenius): host pointers, an output overlapping an operand and sizes past
each form's limit are refused with GF2X_EINVAL before any launch; zero-length
operands give the empty product; afterwards a product is still exact."""
import numpy as np
import pytest
import torch

import paper_1708_09746_gb300 as G
from oracle import product as P
import workloads as W

from gpu_util import empty_dev, from_dev, need_gpu, to_dev

pytestmark = pytest.mark.gpu

FORMS = {
    "tower256": (G.gf2x_mul_tower256, G.gf2x_mul_tower256_async),
    "simple": (G.gf2x_mul_simple, G.gf2x_mul_simple_async),
    "frobenius": (G.gf2x_mul_frobenius, G.gf2x_mul_frobenius_async),
}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("form", sorted(FORMS))
def test_refused_arguments(form):
    sync, asyn = FORMS[form]
    n = 5000
    a, b = W.operand_pair(3, n, n)
    da, db = to_dev(a), to_dev(b)
    ow = G.gf2x_out_words(n, n)
    out = empty_dev(ow)
    host = torch.from_numpy(a.view(np.int64).copy())
    for args in [(host, n, db, n, out), (da, n, db, n, torch.zeros(ow, dtype=torch.int64)),
                 (da, n, db, n, da),                     # output overlaps an operand
                 (da, (1 << 33) + 1, db, n, out)]:       # longer than 2^33 bits
        with pytest.raises(G.GF2XError) as e:
            sync(*args)
        assert e.value.status == G.GF2X_EINVAL, (form, e.value.status)
    s = torch.cuda.Stream()
    with pytest.raises(G.GF2XError) as e:
        asyn(da, n, host, n, out, s)
    assert e.value.status == G.GF2X_EINVAL
    sync(da, 0, db, n, out)   # the empty product: nothing to do
    sync(da, n, db, 0, out)
    G.gf2x_stream_status(s)   # nothing was launched on it
    sync(da, n, db, n, out)
    assert np.array_equal(from_dev(out, ow), P.mul(a, n, b, n))


def test_points_helpers():
    assert G.gf2x_tower256_fft_points(1 << 28, 1 << 28) == 1 << 22
    assert G.gf2x_tower256_fft_points(128, 128) == 2
    assert G.gf2x_tower256_fft_points(0, 5) == 0
    assert G.gf2x_frobenius_points(1 << 28, 1 << 28) == 22
    assert G.gf2x_frobenius_points(64, 65) == 0   # 128 bits: one point
    assert G.gf2x_frobenius_points(0, 3) == -1
