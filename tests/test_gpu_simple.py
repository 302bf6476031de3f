"""The simple polynomial-basis form (Alg. 4) on the GPU against the oracle.

The general GF(2^128) product and the FFT stages against oracle/simple.py
element by element (the Cantor basis of the library and of the oracle is the
same one: each beta_i is the root with coefficient 0 at z^0), whole products
against the plain carry-less product word for word from one bit to the 2^28-bit
workload.  Bit-exact throughout.
"""
import numpy as np
import pytest
import torch

import paper_1708_09746_gb300 as G
from oracle import product as P
from oracle import simple as SM
import workloads as W

from gpu_util import empty_dev, from_dev, ints_to_pairs, need_gpu, pairs_to_ints, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def test_general_product_stage():
    n = 4096
    A = W.random_words(51, 2 * n)
    B = W.random_words(52, 2 * n)
    # edge values: 0, 1, z^127 (the reduction of its square), all ones
    A[:8] = np.array([0, 0, 1, 0, 0, 1 << 63, 2**64 - 1, 2**64 - 1], dtype=np.uint64)
    B[:8] = np.array([5, 7, 0, 1 << 63, 0, 1 << 63, 2**64 - 1, 2**64 - 1], dtype=np.uint64)
    dB = to_dev(B)
    G.gf2x_stage_gfmul_simple(to_dev(A), dB, n)
    torch.cuda.synchronize()
    got = pairs_to_ints(from_dev(dB))
    a, b = pairs_to_ints(A), pairs_to_ints(B)
    for i in range(n):
        assert got[i] == SM.gmul(a[i], b[i]), i


@pytest.mark.parametrize("log_n,layers", [(1, 1), (4, 4), (8, 5), (11, 11), (12, 12), (13, 12),
                                          (15, 10), (16, 13)])
def test_fft_stage_forward_and_inverse(log_n, layers):
    n = 1 << log_n
    P_ = 1 << layers
    coeffs = pairs_to_ints(W.random_words(60 + log_n, 2 * P_))
    periodic = [coeffs[i % P_] for i in range(n)]
    F = to_dev(ints_to_pairs(periodic))
    G.gf2x_stage_fft_simple(F, log_n, layers, 0)
    torch.cuda.synchronize()
    got = pairs_to_ints(from_dev(F))
    if log_n <= 12:
        want = SM.fft_simple(coeffs + [0] * (n - P_))
        assert got == want
    else:
        # sampled points by direct evaluation
        rng = np.random.default_rng(log_n)
        for i in [0, 1, n - 1] + [int(x) for x in rng.integers(0, n, 3)]:
            assert got[i] == SM.eval_novelpoly_simple(coeffs, SM.phi_beta(i)), i
    # the inverse of the whole transform returns the zero-padded coefficients
    G.gf2x_stage_fft_simple(F, log_n, log_n, 1)
    torch.cuda.synchronize()
    back = pairs_to_ints(from_dev(F))
    assert back == coeffs + [0] * (n - P_)


SIZES = [(1, 1), (64, 64), (65, 63), (1000, 3), (4096, 4096), (65536 + 77, 40000),
         (1 << 20, 1 << 20), ((1 << 20) + 5, (1 << 19) - 3), (1 << 22, 64), (1 << 23, 1 << 23)]


@pytest.mark.parametrize("na,nb", SIZES)
def test_products_against_oracle(na, nb):
    a, b = W.operand_pair(na % 997 + nb % 89, na, nb)
    ow = G.gf2x_out_words(na, nb)
    out = torch.full((ow + 2,), -0x5A5A5A5A5A5A5A5B, dtype=torch.int64, device="cuda")
    G.gf2x_mul_simple(to_dev(a), na, to_dev(b), nb, out)
    res = from_dev(out)
    assert all(int(x) == 0xA5A5A5A5A5A5A5A5 for x in res[ow:]), "wrote past the product"
    assert np.array_equal(res[:ow], P.mul(a, na, b, nb))


def test_fullsize_2_28_against_oracle():
    a, na, b, nb = W.make_workload("c1_2^28")
    ow = G.gf2x_out_words(na, nb)
    out = empty_dev(ow)
    s = torch.cuda.Stream()
    G.gf2x_mul_simple_async(to_dev(a), na, to_dev(b), nb, out, s)
    s.synchronize()
    got = from_dev(out, ow)
    del out
    torch.cuda.empty_cache()
    want = P.mul(a, na, b, nb)
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, "first differing word %d" % int(bad[0])
