"""Pins for the simple polynomial-basis form (oracle/simple.py, Alg. 4).

The field product is checked against the modulus it is defined by and the
field axioms; the Cantor basis against its defining relations and the shift
property s_k(phi_beta(j)) = phi_beta(j >> k) with s_k computed by iteration of
s_1(x) = x^2 + x; the FFT against direct evaluation at every point; whole
products against the bit-by-bit definition of the product.
"""
import numpy as np
import pytest

from oracle import product as P
from oracle import simple as SM
import workloads as W


def _rand(rng, bits=128):
    return int.from_bytes(rng.bytes(bits // 8), "little")


def test_modulus_and_field_axioms():
    z = 2
    # z^128 = z^7 + z^2 + z + 1
    assert SM.gpow(z, 128) == 0x87
    rng = np.random.default_rng(5)
    for _ in range(10):
        a, b, c = _rand(rng), _rand(rng), _rand(rng)
        assert SM.gmul(a, b) == SM.gmul(b, a)
        assert SM.gmul(a, b ^ c) == SM.gmul(a, b) ^ SM.gmul(a, c)
        assert SM.gmul(SM.gmul(a, b), c) == SM.gmul(a, SM.gmul(b, c))
    a = _rand(rng) | 1
    assert SM.gpow(a, 2**128) == a                       # Frobenius
    assert SM.gmul(a, SM.gpow(a, 2**128 - 2)) == 1        # inverse
    # products of two blocks of degree < 64 never wrap
    x, y = _rand(rng, 64), _rand(rng, 64)
    assert SM.gmul(x, y) == SM.S.gf2_polmul(x, y)


def test_cantor_basis_relations_and_shift_property():
    beta = SM.cantor_basis()
    assert beta[0] == 1
    for i in range(1, 128):
        assert SM.gmul(beta[i], beta[i]) ^ beta[i] == beta[i - 1]
        assert beta[i] & 1 == 0
    # the basis spans the field: rank 128 over GF(2)
    rows, rank = list(beta), 0
    for bit in range(128):
        piv = next((i for i in range(rank, 128) if (rows[i] >> bit) & 1), None)
        if piv is None:
            continue
        rows[rank], rows[piv] = rows[piv], rows[rank]
        for i in range(128):
            if i != rank and (rows[i] >> bit) & 1:
                rows[i] ^= rows[rank]
        rank += 1
    assert rank == 128
    rng = np.random.default_rng(6)
    for _ in range(12):
        j = int(rng.integers(0, 2**40))
        k = int(rng.integers(0, 24))
        assert SM.s_k_iter(k, SM.phi_beta(j)) == SM.phi_beta(j >> k)


def test_fft_simple_against_direct_evaluation():
    rng = np.random.default_rng(7)
    for n in (1, 2, 4, 8, 32):
        g = [_rand(rng) for _ in range(n)]
        out = SM.fft_simple(g)
        for i in range(n):
            assert out[i] == SM.eval_novelpoly_simple(g, SM.phi_beta(i)), (n, i)
        assert SM.ifft_simple(out) == g


@pytest.mark.parametrize("na,nb", [(1, 1), (64, 64), (65, 63), (300, 700), (1000, 1000),
                                    (2048, 2048), (4096, 1234), (5000, 3)])
def test_whole_product_against_bit_definition(na, nb):
    a, b = W.operand_pair(na * 3 + nb, na, nb)
    got, _ = SM.binpolymul_simple(a, na, b, nb)
    assert np.array_equal(np.array(got, dtype=np.uint64), P.mul_bits(a, na, b, nb))
