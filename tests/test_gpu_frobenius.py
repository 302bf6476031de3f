"""The Frobenius-partition form (Appendix C) on the GPU against the oracle.

BasisCvt of one-bit coefficients (tile passes and streaming passes), the
encoding and its inverse, and the FFT at beta_{m+64} + V_m against
oracle/frobenius.py and oracle/stages.py element by element; whole products
against the plain carry-less product word for word, from one bit to the
2^28-bit workload (products of fewer than 32 points take the atomic scatter of
the inverse encoding, the others the warp-ballot one).  Bit-exact throughout.
"""
import numpy as np
import pytest
import torch

import paper_1708_09746_gb300 as G
from oracle import frobenius as FR
from oracle import product as P
from oracle import simple as SM
from oracle import stages as S
import workloads as W

from gpu_util import empty_dev, from_dev, ints_to_pairs, need_gpu, pairs_to_ints, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _bits(words, L):
    w = np.asarray(words, dtype=np.uint64)
    return [(int(w[i >> 6]) >> (i & 63)) & 1 for i in range(1 << L)]


def _words(bits):
    nw = max(1, (len(bits) + 63) // 64)
    out = np.zeros(nw, dtype=np.uint64)
    for i, b in enumerate(bits):
        if b:
            out[i >> 6] |= np.uint64(1 << (i & 63))
    return out


@pytest.mark.parametrize("L", [0, 1, 2, 5, 6, 7, 10, 13, 18, 19, 20])
def test_bit_basis_cvt(L):
    nw = max(1, (1 << L) // 64)
    x = W.random_words(100 + L, nw)
    if L < 6:
        x[0] &= np.uint64((1 << (1 << L)) - 1)
    d = to_dev(x)
    G.gf2x_stage_bit_basis_cvt(d, L, 0)
    torch.cuda.synchronize()
    got = from_dev(d, nw)
    want = _words(S.basis_cvt(_bits(x, L)))
    assert np.array_equal(got, want)
    G.gf2x_stage_bit_basis_cvt(d, L, 1)
    torch.cuda.synchronize()
    assert np.array_equal(from_dev(d, nw), x)


@pytest.mark.parametrize("m,log_bits", [(0, 7), (2, 8), (4, 10), (5, 11), (5, 12), (8, 14),
                                        (10, 17)])
def test_encoding_and_inverse(m, log_bits):
    n = 1 << m
    nw = max(1, (1 << log_bits) // 64)
    g = W.random_words(200 + m, nw)
    if log_bits < 6:
        g[0] &= np.uint64((1 << (1 << log_bits)) - 1)
    E = empty_dev(2 * n)
    G.gf2x_stage_frobenius_encode(to_dev(g), log_bits, m, E, 0)
    torch.cuda.synchronize()
    got = pairs_to_ints(from_dev(E))
    bits = _bits(g, log_bits)
    for i in range(n):
        col = 0
        for j in range(128):
            pos = i + j * n
            if pos < len(bits) and bits[pos]:
                col |= 1 << j
        assert got[i] == FR.encode(col), i
    # the inverse: random elements back to 128 n bits
    vals = pairs_to_ints(W.random_words(300 + m, 2 * n))
    c = torch.full((2 * n,), -1, dtype=torch.int64, device="cuda")
    G.gf2x_stage_frobenius_encode(c, m + 7, m, to_dev(ints_to_pairs(vals)), 1)
    torch.cuda.synchronize()
    cb = _bits(from_dev(c), m + 7)
    for i in range(n):
        col = FR.decode(vals[i])
        assert all(cb[i + j * n] == (col >> j) & 1 for j in range(128)), i


@pytest.mark.parametrize("m", [0, 1, 4, 8, 11, 12])
def test_fft_at_frobenius_points(m):
    n = 1 << m
    g = pairs_to_ints(W.random_words(400 + m, 2 * n))
    F = to_dev(ints_to_pairs(g))
    G.gf2x_stage_fft_frobenius(F, m, 0)
    torch.cuda.synchronize()
    got = pairs_to_ints(from_dev(F))
    if m <= 8:
        assert got == SM.fft_simple(g, FR.alpha_index(m))
    else:
        alpha = FR.alpha_index(m)
        for i in [0, 1, n - 1, n // 3]:
            assert got[i] == SM.eval_novelpoly_simple(g, SM.phi_beta(alpha | i)), i
    G.gf2x_stage_fft_frobenius(F, m, 1)
    torch.cuda.synchronize()
    assert pairs_to_ints(from_dev(F)) == g


SIZES = [(1, 1), (64, 64), (100, 29), (128, 128), (1000, 3), (2048, 2047), (4096, 4096),
         (65536 + 77, 40000), (1 << 20, 1 << 20), ((1 << 20) + 5, (1 << 19) - 3), (1 << 22, 64),
         (1 << 24, 1 << 24), (3 * (1 << 22) + 1, 1 << 23)]


@pytest.mark.parametrize("na,nb", SIZES)
def test_products_against_oracle(na, nb):
    a, b = W.operand_pair(na % 991 + nb % 83, na, nb)
    ow = G.gf2x_out_words(na, nb)
    out = torch.full((ow + 2,), -0x5A5A5A5A5A5A5A5B, dtype=torch.int64, device="cuda")
    G.gf2x_mul_frobenius(to_dev(a), na, to_dev(b), nb, out)
    res = from_dev(out)
    assert all(int(x) == 0xA5A5A5A5A5A5A5A5 for x in res[ow:]), "wrote past the product"
    assert np.array_equal(res[:ow], P.mul(a, na, b, nb))


def test_fullsize_2_28_against_oracle():
    a, na, b, nb = W.make_workload("c1_2^28")
    assert G.gf2x_frobenius_points(na, nb) == 22
    ow = G.gf2x_out_words(na, nb)
    out = empty_dev(ow)
    s = torch.cuda.Stream()
    G.gf2x_mul_frobenius_async(to_dev(a), na, to_dev(b), nb, out, s)
    s.synchronize()
    got = from_dev(out, ow)
    del out
    torch.cuda.empty_cache()
    want = P.mul(a, na, b, nb)
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, "first differing word %d" % int(bad[0])
