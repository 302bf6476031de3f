"""The allocation-free product gf2x_mul_noalloc against gf2x_mul.

gf2x_mul_noalloc is for callers that cannot allocate device memory while
they multiply (their device memory all belongs to their own pool, or an
allocation there would synchronise the device): its scratch is a static
device array of the library.  This file is named so that pytest collects it
last; it must pass both alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest
import torch

import paper_1708_09746_gb300 as G
import workloads as W

from gpu_util import empty_dev, from_dev, need_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _both(na, nb, seed, stream=None):
    a, b = W.operand_pair(seed, na, nb)
    da, db = to_dev(a), to_dev(b)
    ow = G.gf2x_out_words(na, nb)
    ref = empty_dev(ow)
    G.gf2x_mul(da, na, db, nb, ref)
    got = torch.full((ow,), -1, dtype=torch.int64, device="cuda")
    G.gf2x_mul_noalloc(da, na, db, nb, got, stream)
    torch.cuda.synchronize()
    return from_dev(got, ow), from_dev(ref, ow)


def test_noalloc_matches_gf2x_mul_two_calls_in_a_row():
    # two calls in a row share the static scratch: the second must not see
    # anything left over from the first (different sizes, then the same size)
    for na, nb, seed in [(1 << 20, 1 << 20, 0), (70001, 5000, 1), (70001, 5000, 2)]:
        got, ref = _both(na, nb, seed)
        assert np.array_equal(got, ref), (na, nb)


def test_noalloc_largest_size_and_limit():
    # the largest accepted transform: 2^18 points (two 2^23-bit operands)
    got, ref = _both(1 << 23, 1 << 23, 3, torch.cuda.Stream())
    assert np.array_equal(got, ref)
    # two words more need 2^19 points: rejected with GF2X_EINVAL
    na = (1 << 23) + 128
    da = to_dev(W.uniform_poly(4, na))
    out = empty_dev(G.gf2x_out_words(na, 1 << 23))
    with pytest.raises(G.GF2XError) as e:
        G.gf2x_mul_noalloc(da, na, da, 1 << 23, out)
    assert e.value.status == G.GF2X_EINVAL


def test_noalloc_small_and_ragged():
    for na, nb in [(1, 1), (64, 65), (1000, 3), (4097, 8191)]:
        got, ref = _both(na, nb, na + nb)
        assert np.array_equal(got, ref), (na, nb)
