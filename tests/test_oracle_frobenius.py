"""Pins for the Frobenius-partition form (oracle/frobenius.py, Appendix C).

Proposition C.1 (E is a bijection) by the rank of E over GF(2) for small m;
the truncated FFT against direct evaluation of the polynomial at every point
alpha + phi_beta(i), alpha = beta_{m+64}; the encoding against its inverse;
whole products against the bit-by-bit definition.
"""
import numpy as np
import pytest

from oracle import frobenius as FR
from oracle import product as P
from oracle import simple as SM
import workloads as W


def _rank(vectors):
    rows, rank = list(vectors), 0
    nbits = max(v.bit_length() for v in rows) if rows else 0
    for bit in range(nbits):
        piv = next((i for i in range(rank, len(rows)) if (rows[i] >> bit) & 1), None)
        if piv is None:
            continue
        rows[rank], rows[piv] = rows[piv], rows[rank]
        for i in range(len(rows)):
            if i != rank and (rows[i] >> bit) & 1:
                rows[i] ^= rows[rank]
        rank += 1
    return rank


@pytest.mark.parametrize("m", [0, 1, 2])
def test_E_is_a_bijection(m):
    # the images of the monomials x^t, t < 128 n, as 128 n-bit vectors: the
    # evaluations at the n points concatenated
    n = 1 << m
    alpha = FR.alpha_index(m)
    pts = [SM.phi_beta(alpha | i) for i in range(n)]
    vecs = []
    for t in range(128 * n):
        v = 0
        for i, x in enumerate(pts):
            v |= SM.gpow(x, t) << (128 * i)
        vecs.append(v)
    assert _rank(vecs) == 128 * n


@pytest.mark.parametrize("m,nbits", [(0, 128), (1, 200), (2, 512), (3, 1000)])
def test_E_against_direct_evaluation(m, nbits):
    a = W.uniform_poly(90 + m, nbits)
    vals, _ = FR.E_map(a, nbits, m)
    alpha = FR.alpha_index(m)
    for i in range(1 << m):
        assert vals[i] == FR.eval_bits_at(a, nbits, SM.phi_beta(alpha | i)), i


def test_encoding_inverse():
    rng = np.random.default_rng(8)
    for _ in range(20):
        col = int.from_bytes(rng.bytes(16), "little")
        assert FR.decode(FR.encode(col)) == col
    # the encoding multipliers: w_0 = 1, w_(2^l) = beta_(64 - l)
    beta = SM.cantor_basis()
    w = FR.enc_multipliers()
    assert w[0] == 1 and all(w[1 << l] == beta[64 - l] for l in range(7))


@pytest.mark.parametrize("na,nb", [(1, 1), (64, 64), (100, 29), (128, 128), (300, 700),
                                    (1000, 1000), (2048, 2047), (5000, 3)])
def test_whole_product_against_bit_definition(na, nb):
    a, b = W.operand_pair(na * 5 + nb, na, nb)
    got, _ = FR.binpolymul_frobenius(a, na, b, nb)
    assert np.array_equal(np.array(got, dtype=np.uint64), P.mul_bits(a, na, b, nb))
