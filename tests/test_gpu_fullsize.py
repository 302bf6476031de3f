"""Parity at the full workload sizes (2^28 ... 2^33-bit operands), in the
launch configuration the benchmark times: gf2x_mul_async on a side stream.

The headline 2^28-bit product is compared word for word with the whole
oracle product.  At the larger sizes a full oracle product takes minutes, so
the CUDA result is checked against (i) product words the oracle computes one by one from the
definition c_k = sum_{i+j=k} a_i b_j (word 0, the top words, the words around
the operands' lengths and seeded random words), (ii) modular fingerprints:
c mod r = (a mod r)(b mod r) mod r for random irreducible r of degree 64, which
a wrong product passes with probability below 2^-50 each, and (iii) where the
operands have a closed-form product (all-ones squared, a times 1 + x^k), the
whole output.  Bits past the product and words past the output buffer are
checked too.
"""
import numpy as np
import pytest
import torch

import paper_1708_09746_gb300 as G
from oracle import product as P
import workloads as W

from gpu_util import need_gpu, to_dev

pytestmark = pytest.mark.gpu

SENTINEL = -0x5A5A5A5A5A5A5A5B  # 0xA5A5A5A5A5A5A5A5 as int64


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _gpu_product(a, na, b, nb):
    """The product through gf2x_mul_async on a side stream, as the bench
    launches it, into a buffer with a sentinel tail."""
    ow = G.gf2x_out_words(na, nb)
    da, db = to_dev(a), to_dev(b)
    out = torch.full((ow + 4,), SENTINEL, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        G.gf2x_mul_async(da, na, db, nb, out, s)
    s.synchronize()
    del da, db
    res = out.cpu().numpy().view(np.uint64)
    del out
    torch.cuda.empty_cache()
    assert all(int(x) == 0xA5A5A5A5A5A5A5A5 for x in res[ow:]), "wrote past the product"
    return res[:ow]


def _sample_positions(na, nb, ow, seed, n_random):
    na_w, nb_w = (na + 63) // 64, (nb + 63) // 64
    pos = {0, 1, ow - 1, ow - 2, ow // 2, na_w - 1, na_w, nb_w - 1, nb_w}
    rng = np.random.default_rng(seed)
    pos.update(int(x) for x in rng.integers(0, ow, n_random))
    return sorted(p for p in pos if 0 <= p < ow)


def _check_sampled(c, a, na, b, nb, seed, n_random=8, n_fp=2):
    ow = len(c)
    rem = (na + nb - 1) % 64
    top_mask = (1 << rem) - 1 if rem else 2**64 - 1
    for j in _sample_positions(na, nb, ow, seed, n_random):
        want = P.product_word(a, na, b, nb, j)
        if j == ow - 1:
            want &= top_mask
        assert int(c[j]) == want, "word %d" % j
    assert int(c[-1]) & ~top_mask & (2**64 - 1) == 0, "bits past the product"
    rng = np.random.default_rng(seed + 1)
    for _ in range(n_fp):
        r = P.random_irreducible64(rng)
        assert P.fingerprint_ok(a, na, b, nb, c, r), "fingerprint mod x^64+%#x" % r


def test_fullsize_2_28_whole_product_against_oracle():
    # The headline workload compared word for word with the whole oracle
    # product (Karatsuba over the host's fastest carry-less word product,
    # PMULL on an aarch64 host, on all host cores).
    a, na, b, nb = W.make_workload("c1_2^28")
    c = _gpu_product(a, na, b, nb)
    want = P.mul(a, na, b, nb)
    assert len(c) == len(want)
    bad = np.flatnonzero(c != want)
    assert bad.size == 0, "first differing word %d of %d (oracle clmul: %s)" % (
        int(bad[0]), len(c), P.clmul_kind())


@pytest.mark.parametrize("name,n_fp", [
    ("c1_2^28", 4),          # the headline workload
    ("c1_2^29", 2),
    ("c1_2^28_sparse", 2),   # 1 %-dense bits
    ("c1_2^29_sparse", 2),
    ("c1_2^28x2^16", 4),     # unequal lengths: Pb << N
    ("c2_2^30", 2),
    ("c2_2^32", 1),
])
def test_fullsize_sampled(name, n_fp):
    a, na, b, nb = W.make_workload(name)
    c = _gpu_product(a, na, b, nb)
    _check_sampled(c, a, na, b, nb, seed=na % 9973 + nb % 997, n_fp=n_fp)


@pytest.mark.parametrize("name", ["c1_2^28_ones", "c1_2^29_ones"])
def test_fullsize_all_ones_closed_form(name):
    # (sum_{i<n} x^i)^2 = sum_{i<n} x^(2i) over GF(2): every even bit up to
    # 2n-2, i.e. words 0x5555...; the last word holds the bits below 2n-1.
    a, na, b, nb = W.make_workload(name)
    c = _gpu_product(a, na, b, nb)
    want = np.full(len(c), 0x5555555555555555, dtype=np.uint64)
    rem = (na + nb - 1) % 64
    if rem:
        want[-1] &= np.uint64((1 << rem) - 1)
    assert np.array_equal(c, want)


def _shift_xor(a, na, k):
    """a + x^k a as words (the product a * (1 + x^k)), from the definition of
    the shift."""
    ow = P.out_words(na, k + 1)
    out = np.zeros(ow, dtype=np.uint64)
    aw = a[: (na + 63) // 64]
    out[: len(aw)] ^= aw
    q, s = divmod(k, 64)
    if s == 0:
        out[q: q + len(aw)] ^= aw
    else:
        out[q: q + len(aw)] ^= aw << np.uint64(s)
        hi = aw >> np.uint64(64 - s)
        n = min(len(aw), ow - q - 1)
        out[q + 1: q + 1 + n] ^= hi[:n]
    return out


def test_maximum_size_shift_closed_form():
    # The largest operands the library accepts (2^33 bits, N = 2^28 points):
    # a random a times b = 1 + x^k, whose product a + x^k a is known word for
    # word at any size; k is not a multiple of 64 so that every word mixes
    # two shifted words.
    na = 1 << 33
    k = (1 << 33) - 12345
    nb = k + 1
    a = W.uniform_poly(9, na)
    b = np.zeros((nb + 63) // 64, dtype=np.uint64)
    b[0] = np.uint64(1)
    b[k // 64] |= np.uint64(1 << (k % 64))
    assert G.gf2x_fft_points(na, nb) == 1 << 28
    c = _gpu_product(a, na, b, nb)
    want = _shift_xor(a, na, k)
    assert np.array_equal(c, want)


def test_beyond_maximum_rejected():
    z = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(G.GF2XError):
        G.gf2x_mul(z, (1 << 33) + 1, z, 1, z)
