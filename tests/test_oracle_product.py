"""Pins for the end-to-end oracle (oracle/product.py, oracle/gf2x_oracle.c).

The oracle is the plain definition of the method's output, c = a * b in
GF(2)[x] (Sec. 2.1, Alg. 5).  It is pinned here against things other than
itself: the bit-by-bit definition on exhaustive tiny inputs, closed forms
(shifts, (1+x) * sum x^i, squaring spreads bits), and ring invariants
(degree, commutativity, distributivity, associativity), so that a dropped
term, a wrong shift or a transposed operand fails a test.
"""
import numpy as np
import pytest

from oracle import product as P
import workloads as W


def _int_to_words(v, nw):
    return np.array([(v >> (64 * i)) & (2**64 - 1) for i in range(nw)],
                    dtype=np.uint64)


def _words_to_int(w):
    return sum(int(x) << (64 * i) for i, x in enumerate(w))


def _ref_int_mul(a, b):
    """Carry-less product of Python ints from the definition, set-of-exponents
    form: the coefficient of x^k is the parity of #{(i, j): i + j = k}."""
    ea = [i for i in range(a.bit_length()) if (a >> i) & 1]
    eb = [j for j in range(b.bit_length()) if (b >> j) & 1]
    r = 0
    for i in ea:
        for j in eb:
            r ^= 1 << (i + j)
    return r


def test_clmul64_definition():
    rng = np.random.default_rng(11)
    vals = [0, 1, 2, 3, 2**63, 2**64 - 1, 0x8000000000000001]
    vals += [int(x) for x in rng.integers(0, 2**63, size=20, dtype=np.uint64) * 2 + 1]
    for x in vals:
        for y in vals[:12]:
            lo, hi = P.clmul64(x, y)
            assert lo | (hi << 64) == _ref_int_mul(x, y)


def test_clmul64_fast_forms_match_definition():
    # The 4-bit window form and the form the product routines use (PMULL on
    # an aarch64 host that has it) against the bit-by-bit definition: every
    # single-bit pair, structured words, and random pairs.
    rng = np.random.default_rng(12)
    vals = [0, 1, 2**64 - 1, 0x5555555555555555, 0xAAAAAAAAAAAAAAAA,
            0x8000000000000001, 0x0F0F0F0F0F0F0F0F]
    vals += [1 << i for i in range(64)]
    pairs = [(x, y) for x in vals for y in vals]
    r = rng.integers(0, 2**64 - 1, size=(4000, 2), dtype=np.uint64, endpoint=True)
    pairs += [(int(x), int(y)) for x, y in r]
    for x, y in pairs:
        want = P.clmul64(x, y)
        assert P.clmul64_win4(x, y) == want, (hex(x), hex(y))
        assert P.clmul64_fast(x, y) == want, (hex(x), hex(y), P.clmul_kind())
    assert P.clmul_kind() in ("pmull", "win4")


def test_exhaustive_8x8_bits():
    # every pair of polynomials with at most 8 bits
    for a in range(256):
        A = np.array([a], dtype=np.uint64)
        for b in range(0, 256, 3):
            B = np.array([b], dtype=np.uint64)
            want = _ref_int_mul(a, b)
            got = P.mul_bits(A, 8, B, 8)
            assert _words_to_int(got) == want
    # and the word-level paths agree on the same pairs
    for a in range(0, 256, 7):
        for b in range(256):
            A = np.array([a], dtype=np.uint64)
            B = np.array([b], dtype=np.uint64)
            assert _words_to_int(P.mul_schoolbook(A, 8, B, 8)) == _ref_int_mul(a, b)


@pytest.mark.parametrize("na,nb", [(1, 1), (63, 64), (64, 65), (129, 7), (1000, 999),
                                   (4096, 4096), (4095, 1), (3000, 4096)])
def test_random_against_bits(na, nb):
    a, b = W.operand_pair(na * 7 + nb, na, nb)
    want = P.mul_bits(a, na, b, nb)
    assert np.array_equal(P.mul_schoolbook(a, na, b, nb), want)
    assert np.array_equal(P.mul_karatsuba(a, na, b, nb), want)
    assert np.array_equal(P.mul(a, na, b, nb), want)
    # cross-check against the Python-int definition too
    assert _words_to_int(want) == _ref_int_mul(_words_to_int(a), _words_to_int(b))


def test_karatsuba_large_vs_schoolbook():
    na = nb = 64 * 300 + 17
    a, b = W.operand_pair(5, na, nb)
    assert np.array_equal(P.mul_karatsuba(a, na, b, nb, par_depth=2),
                          P.mul_schoolbook(a, na, b, nb))


def test_closed_forms():
    n = 5000
    # x^k * b is a shift by k
    b = W.uniform_poly(3, n)
    for k in (0, 1, 63, 64, 65, 1000):
        a = _int_to_words(1 << k, (k + 64) // 64)
        got = _words_to_int(P.mul(a, k + 1, b, n))
        assert got == _words_to_int(b) << k
    # (1 + x^k) * b = b + (b << k)
    k = 77
    a = _int_to_words(1 | (1 << k), 2)
    assert _words_to_int(P.mul(a, k + 1, b, n)) == _words_to_int(b) ^ (_words_to_int(b) << k)
    # (1 + x) * sum_{i<n} x^i = 1 + x^n
    ones = W.all_ones(n)
    one_x = np.array([3], dtype=np.uint64)
    assert _words_to_int(P.mul(one_x, 2, ones, n)) == 1 | (1 << n)
    # squaring spreads bits: a^2 = sum a_i x^(2i)
    a = W.uniform_poly(9, 3000)
    ai = _words_to_int(a)
    spread = sum(1 << (2 * i) for i in range(3000) if (ai >> i) & 1)
    assert _words_to_int(P.mul(a, 3000, a, 3000)) == spread
    # all-ones times all-ones: coefficient k is the parity of the number of
    # (i, j) with i + j = k, i.e. of min(k, 2n-2-k) + 1
    m = 700
    o = W.all_ones(m)
    got = _words_to_int(P.mul(o, m, o, m))
    want = sum(1 << k for k in range(2 * m - 1) if (min(k, 2 * m - 2 - k) + 1) & 1)
    assert got == want


def test_ring_invariants():
    na, nb, nc = 20000, 13000, 9000
    a = W.uniform_poly(21, na)
    b = W.uniform_poly(22, nb)
    c = W.uniform_poly(23, nc)
    ab = P.mul(a, na, b, nb)
    # degree: deg(ab) = deg a + deg b (top bits forced)
    top = na + nb - 2
    ai = _words_to_int(ab)
    assert ai.bit_length() - 1 == top
    # commutativity
    assert np.array_equal(P.mul(b, nb, a, na), ab)
    # associativity (a b) c = a (b c)
    bc = P.mul(b, nb, c, nc)
    assert np.array_equal(P.mul(ab, na + nb - 1, c, nc), P.mul(a, na, bc, nb + nc - 1))
    # distributivity a (b + c) = ab + ac
    bpc = np.zeros(max(len(b), len(c)), dtype=np.uint64)
    bpc[:len(b)] ^= b
    bpc[:len(c)] ^= c
    lhs = P.mul(a, na, bpc, max(nb, nc))
    ac = P.mul(a, na, c, nc)
    rhs = np.zeros(len(lhs), dtype=np.uint64)
    rhs[:len(ab)] ^= ab
    rhs[:len(ac)] ^= ac
    assert np.array_equal(lhs, rhs)


def test_empty_operands():
    a = W.uniform_poly(1, 100)
    assert P.mul(a, 100, a, 0).size == 0
    assert P.out_words(0, 5) == 0
    assert P.out_words(64, 1) == 1
    assert P.out_words(64, 2) == 2


def test_fingerprint_detects_errors():
    rng = np.random.default_rng(5)
    r = P.random_irreducible64(rng)
    assert P.is_irreducible64(r)
    # x^64 + x^4 + x^3 + x + 1 is a known irreducible pentanomial;
    # x^64 + 1 = (x + 1)^64 is not.
    assert P.is_irreducible64(0x1B)
    assert not P.is_irreducible64(1)
    na = nb = 6000
    a, b = W.operand_pair(8, na, nb)
    c = P.mul(a, na, b, nb)
    assert P.fingerprint_ok(a, na, b, nb, c, r)
    bad = c.copy()
    bad[17] ^= np.uint64(1 << 5)
    assert not P.fingerprint_ok(a, na, b, nb, bad, r)


def test_product_word_matches_full_product():
    na, nb = 64 * 50 + 3, 64 * 31 + 60
    a, b = W.operand_pair(31, na, nb)
    full = P.mul_bits(a, na, b, nb)
    for j in range(len(full)):
        w = P.product_word(a, na, b, nb, j)
        if j == len(full) - 1 and (na + nb - 1) % 64:
            w &= (1 << ((na + nb - 1) % 64)) - 1
        assert w == int(full[j])
