"""The allocation-free product gf2x_mul_noalloc against the oracle and gf2x_mul.

gf2x_mul_noalloc is for callers that cannot allocate device memory while
they multiply (their device memory all belongs to their own pool, or an
allocation there would synchronise the device): its scratch is a static
device array of the library.  Its results are checked word for word against
the CPU oracle's product and against gf2x_mul on the same inputs, and a call
after the first must leave the device's free memory unchanged.  This file is
named so that pytest collects it last; it must pass both alone in a fresh
process and after the other tests.
"""
import numpy as np
import pytest
import torch

import paper_1708_09746_gb300 as G
from oracle import product as P
import workloads as W

from gpu_util import empty_dev, from_dev, need_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _check(na, nb, seed, stream=None):
    """gf2x_mul_noalloc, gf2x_mul and the oracle on one seeded pair."""
    a, b = W.operand_pair(seed, na, nb)
    da, db = to_dev(a), to_dev(b)
    ow = G.gf2x_out_words(na, nb)
    ref = empty_dev(ow)
    G.gf2x_mul(da, na, db, nb, ref)
    got = torch.full((ow,), -1, dtype=torch.int64, device="cuda")
    G.gf2x_mul_noalloc(da, na, db, nb, got, stream)
    torch.cuda.synchronize()
    got, ref = from_dev(got, ow), from_dev(ref, ow)
    want = P.mul(a, na, b, nb)
    assert np.array_equal(got, want), (na, nb, "noalloc vs oracle")
    assert np.array_equal(ref, want), (na, nb, "gf2x_mul vs oracle")


def test_noalloc_matches_oracle_two_calls_in_a_row():
    # two calls in a row share the static scratch: the second must not see
    # anything left over from the first (different sizes, then the same size)
    for na, nb, seed in [(1 << 20, 1 << 20, 0), (70001, 5000, 1), (70001, 5000, 2)]:
        _check(na, nb, seed)


def test_noalloc_leaves_free_memory_unchanged():
    na, nb = (1 << 21) + 77, (1 << 20) - 3
    a, b = W.operand_pair(5, na, nb)
    da, db = to_dev(a), to_dev(b)
    ow = G.gf2x_out_words(na, nb)
    out = empty_dev(ow)
    G.gf2x_mul_noalloc(da, na, db, nb, out)  # first call: per-device set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        G.gf2x_mul_noalloc(da, na, db, nb, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, "free device memory changed by %d bytes" % (free0 - free1)
    assert np.array_equal(from_dev(out, ow), P.mul(a, na, b, nb))


def test_noalloc_largest_sizes_and_limit():
    # the largest accepted transform: 2^18 points, as two 2^23-bit operands
    # and as the most uneven shape (2^18 - 1 words times one word pads the
    # long operand to the whole 2^18 points)
    _check(1 << 23, 1 << 23, 3, torch.cuda.Stream())
    _check((1 << 24) - 64, 64, 6)
    _check(64, (1 << 24) - 64, 7)
    # two words more need 2^19 points: rejected with GF2X_EINVAL
    na = (1 << 23) + 128
    da = to_dev(W.uniform_poly(4, na))
    out = empty_dev(G.gf2x_out_words(na, 1 << 23))
    with pytest.raises(G.GF2XError) as e:
        G.gf2x_mul_noalloc(da, na, da, 1 << 23, out)
    assert e.value.status == G.GF2X_EINVAL


def test_noalloc_rejects_host_pointers():
    # host memory is refused before any launch (the entry point takes device
    # pointers only)
    na = 4096
    a = torch.from_numpy(W.uniform_poly(8, na).view(np.int64).copy())
    out = torch.zeros(G.gf2x_out_words(na, na), dtype=torch.int64)
    with pytest.raises(G.GF2XError) as e:
        G.gf2x_mul_noalloc(a, na, a, na, out)
    assert e.value.status == G.GF2X_EINVAL


def test_noalloc_small_and_ragged():
    for na, nb in [(1, 1), (64, 65), (1000, 3), (4097, 8191)]:
        _check(na, nb, na + nb)
