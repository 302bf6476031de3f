"""Pins for the F~_{2^256} (w = 128) stage reference (oracle/tower256.py).

Each function is checked against something other than itself: the field
axioms and the defining relation of x_8 (Sec. 3.2), the subfield F~_{2^128}
(the existing, separately pinned tower product), the ring homomorphism and
inverse of changeRepr, direct evaluation of the FFT at every point, and whole
products against the bit-by-bit definition c_k = XOR_{i+j=k} a_i b_j.
"""
import numpy as np
import pytest

from oracle import product as P
from oracle import stages as S
from oracle import tower256 as T
import workloads as W


def _rand(rng, bits):
    return int.from_bytes(rng.bytes(bits // 8), "little")


def test_defining_relation_and_subfield():
    x8 = T.R256
    # x_8^2 = x_8 + v_127
    assert T.tmul256(x8, x8) == x8 ^ T.V127
    rng = np.random.default_rng(1)
    for _ in range(20):
        a, b = _rand(rng, 128), _rand(rng, 128)
        assert T.tmul256(a, b) == S.tmul(a, b)  # F~_{2^128} is the low half


def test_field_axioms():
    rng = np.random.default_rng(2)
    for _ in range(6):
        a, b, c = _rand(rng, 256), _rand(rng, 256), _rand(rng, 256)
        assert T.tmul256(a, b) == T.tmul256(b, a)
        assert T.tmul256(a, b ^ c) == T.tmul256(a, b) ^ T.tmul256(a, c)
        assert T.tmul256(T.tmul256(a, b), c) == T.tmul256(a, T.tmul256(b, c))
    # Frobenius: a^(2^256) = a, and a nonzero a has an inverse a^(2^256 - 2)
    a = _rand(rng, 256) | 1
    x = a
    for _ in range(256):
        x = T.tmul256(x, x)
    assert x == a
    assert T.tmul256(a, T.tpow256(a, 2**256 - 2)) == 1


def test_fft256_against_direct_evaluation():
    rng = np.random.default_rng(3)
    for n in (1, 2, 4, 16):
        g = [_rand(rng, 256) for _ in range(n)]
        out = T.fft256(g)
        for i in range(n):
            assert out[i] == T.eval_novelpoly256(g, i), (n, i)
        assert T.ifft256(out) == g


def test_chrepr256_homomorphism_and_inverse():
    rng = np.random.default_rng(4)
    for _ in range(8):
        p, q = _rand(rng, 128), _rand(rng, 128)
        pq = S.gf2_polmul(p, q)  # degree <= 254: no wrap-around
        assert T.tmul256(T.chrepr256(p), T.chrepr256(q)) == T.chrepr256(pq)
        assert T.ichrepr256(T.chrepr256(pq)) == pq
        assert T.ichrepr256(T.chrepr256(p)) == p


@pytest.mark.parametrize("na,nb", [(1, 1), (64, 64), (128, 128), (129, 100), (300, 700),
                                    (1000, 1000), (2048, 2048), (4096, 1234), (5000, 3)])
def test_whole_product_against_bit_definition(na, nb):
    a, b = W.operand_pair(na * 7 + nb, na, nb)
    got, _ = T.binpolymul256(a, na, b, nb)
    want = P.mul_bits(a, na, b, nb)
    assert np.array_equal(np.array(got, dtype=np.uint64), want)
