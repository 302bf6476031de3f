"""The F~_{2^256} (w = 128) form of Alg. 5 on the GPU against the oracle.

Stage by stage (changeRepr into F~_{2^256}, the generic F~_{2^256} pointmul,
changeRepr^-1 with the 128-bit recombination) against oracle/tower256.py on
the same seeded inputs, element by element; whole products against the plain
carry-less product of oracle/product.py, word for word, from one bit to the
2^28-bit workload (ragged lengths, unbalanced shapes, transforms with strided
passes).  Every comparison is bit-exact.
"""
import numpy as np
import pytest
import torch

import paper_1708_09746_gb300 as G
from oracle import product as P
from oracle import tower256 as T
import workloads as W

from gpu_util import empty_dev, from_dev, need_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _ints(words, width_words):
    w = np.asarray(words, dtype=np.uint64)
    out = []
    for i in range(len(w) // width_words):
        v = 0
        for k in range(width_words):
            v |= int(w[width_words * i + k]) << (64 * k)
        out.append(v)
    return out


def _words(vals, width_words):
    out = np.zeros(len(vals) * width_words, dtype=np.uint64)
    for i, v in enumerate(vals):
        for k in range(width_words):
            out[width_words * i + k] = (v >> (64 * k)) & (2**64 - 1)
    return out


def _halves(vals):
    """F~_{2^256} elements -> the device layout: lo halves, then hi halves."""
    return np.concatenate([_words([v & T.M128 for v in vals], 2), _words([v >> 128 for v in vals], 2)])


def _unhalves(words, n2):
    lo = _ints(words[: 2 * n2], 2)
    hi = _ints(words[2 * n2: 4 * n2], 2)
    return [l | (h << 128) for l, h in zip(lo, hi)]


def test_chrepr256_stage():
    Pn, N2 = 256, 1024
    blocks = W.random_words(40, 2 * Pn)
    F = empty_dev(4 * N2)
    G.gf2x_stage_chrepr256(to_dev(blocks), Pn, F, N2)
    torch.cuda.synchronize()
    got = _unhalves(from_dev(F), N2)
    blk = _ints(blocks, 2)
    want = [T.chrepr256(blk[i % Pn]) for i in range(N2)]
    assert got == want


def test_pointmul256_stage():
    N2 = 2048
    A = W.random_words(41, 4 * N2)
    B = W.random_words(42, 4 * N2)
    dB = to_dev(B)
    G.gf2x_stage_pointmul256(to_dev(A), dB, N2)
    torch.cuda.synchronize()
    got = _unhalves(from_dev(dB), N2)
    a, b = _unhalves(A, N2), _unhalves(B, N2)
    for i in range(N2):
        assert got[i] == T.tmul256(a[i], b[i]), i


@pytest.mark.parametrize("out_words,total_bits", [(1024, 1024 * 64), (1023, 1023 * 64 - 5),
                                                  (1, 3), (700, 700 * 64 - 63)])
def test_ichrepr256_combine_stage(out_words, total_bits):
    N2 = 512
    E = W.random_words(43 + out_words, 4 * N2)
    out = torch.full((out_words + 2,), -1, dtype=torch.int64, device="cuda")
    G.gf2x_stage_ichrepr256_combine(to_dev(E), N2, out, out_words, total_bits)
    torch.cuda.synchronize()
    res = from_dev(out)
    cc = [T.ichrepr256(e) for e in _unhalves(E, N2)]
    want = np.array(T.combine256(cc, out_words), dtype=np.uint64)
    if total_bits % 64:
        want[-1] &= np.uint64((1 << (total_bits % 64)) - 1)
    assert np.array_equal(res[:out_words], want)
    assert all(int(x) == 2**64 - 1 for x in res[out_words:]), "wrote past the output"


SIZES = [(1, 1), (64, 64), (127, 129), (128, 128), (129, 1), (1000, 3), (4096, 4096),
         (65536 + 77, 40000), (1 << 20, 1 << 20), ((1 << 20) + 5, (1 << 19) - 3),
         (1 << 22, 1 << 21), (1 << 22, 64), (1 << 24, 1 << 24), (3 * (1 << 22) + 1, 1 << 23)]


@pytest.mark.parametrize("na,nb", SIZES)
def test_products_against_oracle(na, nb):
    a, b = W.operand_pair(na % 1009 + nb % 101, na, nb)
    ow = G.gf2x_out_words(na, nb)
    out = torch.full((ow + 2,), -0x5A5A5A5A5A5A5A5B, dtype=torch.int64, device="cuda")
    G.gf2x_mul_tower256(to_dev(a), na, to_dev(b), nb, out)
    res = from_dev(out)
    assert all(int(x) == 0xA5A5A5A5A5A5A5A5 for x in res[ow:]), "wrote past the product"
    assert np.array_equal(res[:ow], P.mul(a, na, b, nb))


def test_async_on_a_side_stream_and_edge_inputs():
    na, nb = (1 << 21) + 333, (1 << 21) - 9
    a, b = W.operand_pair(77, na, nb)
    a[-1] |= np.uint64(0xFFFF000000000000)  # bits past the length are ignored
    ow = G.gf2x_out_words(na, nb)
    out = empty_dev(ow)
    s = torch.cuda.Stream()
    G.gf2x_mul_tower256_async(to_dev(a), na, to_dev(b), nb, out, s)
    G.gf2x_stream_status(s)
    assert np.array_equal(from_dev(out, ow), P.mul(a, na, b, nb))
    # all-ones squared: every even bit up to 2n - 2
    n = (1 << 20) + 64
    ones = W.all_ones(n)
    out = empty_dev(G.gf2x_out_words(n, n))
    G.gf2x_mul_tower256(to_dev(ones), n, to_dev(ones), n, out)
    want = P.mul(ones, n, ones, n)
    assert np.array_equal(from_dev(out, len(want)), want)
    # zero-length operand: nothing written
    z = empty_dev(1)
    G.gf2x_mul_tower256(z, 0, to_dev(a), na, z)


def test_fullsize_2_28_against_oracle():
    a, na, b, nb = W.make_workload("c1_2^28")
    assert G.gf2x_tower256_fft_points(na, nb) == 1 << 22
    ow = G.gf2x_out_words(na, nb)
    out = empty_dev(ow)
    G.gf2x_mul_tower256(to_dev(a), na, to_dev(b), nb, out)
    got = from_dev(out, ow)
    del out
    torch.cuda.empty_cache()
    want = P.mul(a, na, b, nb)
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, "first differing word %d" % int(bad[0])
