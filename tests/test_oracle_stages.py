"""Pins for the stage reference (oracle/stages.py).

Each stage of Alg. 5 is checked against something other than itself: the
paper's worked examples (Table 1, Fig. 2, Appendix B, stored under
tests/golden/ with citations), its propositions (Prop. 3.1, 3.3), field
axioms, brute-force triangular solves and direct evaluation.
"""
import os

import numpy as np
import pytest

from oracle import product as P
from oracle import stages as S
import workloads as W

RNG = np.random.default_rng(1234)


def _rand128(n):
    return [int(x) | (int(y) << 64) for x, y in
            zip(RNG.integers(0, 2**64, n, dtype=np.uint64),
                RNG.integers(0, 2**64, n, dtype=np.uint64))]


def _golden(golden_dir, name):
    rows = []
    with open(os.path.join(golden_dir, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_gf4_gf16_from_definition():
    # GF(4): x_1^2 = x_1 + 1  -> 0x2 * 0x2 = 0x3
    assert S.tmul(2, 2) == 3
    assert S.tmul(3, 3) == 2
    # GF(16): x_2^2 = x_2 + x_1 -> 0x4 * 0x4 = 0x6
    assert S.tmul(4, 4) == 6
    # x_3^2 = x_3 + x_2 x_1 -> 0x10 * 0x10 = 0x18
    assert S.tmul(16, 16) == 0x18
    # x_7^2 = x_7 + x_1 ... x_6 = v_64 + v_63
    assert S.tmul(1 << 64, 1 << 64) == (1 << 64) | (1 << 63)
    # products of distinct generators are single basis vectors (Def. 3.1)
    assert S.tmul(1 << 4, 1 << 64) == 1 << 68


def test_field_axioms():
    xs = _rand128(6)
    for a in xs:
        for b in xs[:3]:
            assert S.tmul(a, b) == S.tmul(b, a)
            for c in xs[:2]:
                assert S.tmul(S.tmul(a, b), c) == S.tmul(a, S.tmul(b, c))
                assert S.tmul(a, b ^ c) == S.tmul(a, b) ^ S.tmul(a, c)
        assert S.tmul(a, 1) == a
    a = xs[0]
    assert S.tmul(a, S.tinv(a)) == 1
    # Frobenius: a^(2^128) = a
    y = a
    for _ in range(128):
        y = S.tmul(y, y)
    assert y == a


def test_subfield_closure():
    # the low 2^k bits form the subfield \tilde F_{2^(2^k)} (Sec. 3.2)
    for k in (1, 2, 3, 4, 5, 6):
        w = 1 << k
        for _ in range(20):
            a = int(RNG.integers(0, 2**w if w < 64 else 2**63))
            b = int(RNG.integers(0, 2**w if w < 64 else 2**63))
            assert S.tmul(a, b) < (1 << w)


def test_prop_3_1_and_3_3():
    T = S.S_table(128, 128)
    for k in range(128):
        # Prop. 3.1: s_k(v_k) = 1
        assert T[k][k] == 1
        # s_k vanishes on V_k
        for t in range(k):
            assert T[k][t] == 0
    for i in range(1, 128):
        v = 1 << i
        # Prop. 3.3: v_i^2 + v_i in V_i, and s_1 removes exactly one top bit
        u = S.s1(v)
        assert u < (1 << i)
        assert u >> (i - 1) == 1
    # s_k(alpha) is k bits shorter than alpha and ignores alpha's low k bits
    for k in range(0, 30):
        for t in range(k, 40):
            assert T[k][t].bit_length() == t - k + 1


def test_table1_vanishing_polynomials(golden_dir):
    for row in _golden(golden_dir, "table1_si.txt"):
        i = int(row[0])
        want = sum(1 << int(e) for e in row[1:])
        assert S.s_poly(i) == want
    # closed form s_k = sum_{j subset of k} x^(2^j) over a wider range
    for k in range(0, 12):
        want = sum(1 << (1 << j) for j in range(k + 1) if (j & k) == j)
        assert S.s_poly(k) == want


def test_fig2_multipliers(golden_dir):
    for row in _golden(golden_dir, "fig2_multipliers.txt"):
        k = int(row[0])
        for pair in row[1:]:
            alpha, mult = (int(x, 16) for x in pair.split(":"))
            assert S.s_k(k, alpha) == mult
    # the fan-out top layer: s_3(0) = 0
    assert S.s_k(3, 0) == 0


def test_appendix_b_schedule(golden_dir):
    want = [(int(r[1]), int(r[2])) for r in _golden(golden_dir, "appB_basiscvt.txt")]
    trace = []
    S.basis_cvt(list(range(16)), trace)
    assert trace == want


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64, 128])
def test_basis_cvt_vs_triangular_solve(n):
    f = [int(x) for x in W.random_words(n, n)]
    g = S.basis_cvt(f)
    assert g == S.basis_cvt_bruteforce(f)
    assert S.ibasis_cvt(g) == f


def test_basis_cvt_128bit_coefficients():
    f = _rand128(64)
    assert S.basis_cvt(f) == S.basis_cvt_bruteforce(f)


def test_novelpoly_degrees():
    for k in range(64):
        assert S.X_poly(k).bit_length() - 1 == k


@pytest.mark.parametrize("n,alpha", [(2, 0), (8, 0), (16, 0), (32, 0), (16, 0x40), (8, 0x1234 << 3)])
def test_fft_vs_direct_evaluation(n, alpha):
    g = _rand128(n)
    F = S.fft_lch(g, alpha)
    for i in range(n):
        assert F[i] == S.eval_novelpoly(g, i ^ alpha)
    assert S.ifft_lch(F, alpha) == g


def test_vectorised_novelpoly_evaluation():
    # the vectorised sum agrees with the term-by-term one, and X_j vanishes
    # on V_b whenever bit b of j is set (s_b has the roots V_b)
    g = _rand128(32)
    glo, ghi = S._split128(g)
    for x in [0, 1, 5, 31, 0x1234, (1 << 70) + 3]:
        assert S.eval_novelpoly_np(glo, ghi, x) == S.eval_novelpoly(g, x)
    lo, hi = S.novel_basis_at(64, 5)
    assert all(int(lo[j]) == 0 and int(hi[j]) == 0 for j in range(8, 64))
    assert any(int(lo[j]) or int(hi[j]) for j in range(8))
    lo, hi = S.novel_basis_at(8, 0x99)
    for i in range(3):
        assert int(lo[1 << i]) | (int(hi[1 << i]) << 64) == S.s_k(i, 0x99)


def test_chrepr_homomorphism_and_inverse():
    xs = [int(x) for x in W.random_words(77, 8)]
    for p in xs[:4]:
        for q in xs[4:]:
            lo, hi = P.clmul64(p, q)
            pq = lo | (hi << 64)
            assert S.tmul(S.chrepr(p), S.chrepr(q)) == S.chrepr(pq)
            assert S.ichrepr(S.chrepr(pq)) == pq
    for e in _rand128(5):
        assert S.chrepr(S.ichrepr(e)) == e


@pytest.mark.parametrize("na,nb", [(1, 1), (64, 64), (65, 64), (200, 3000), (1024, 1024),
                                   (4096, 128), (64 * 33, 64 * 31 + 5)])
def test_stage_pipeline_equals_product(na, nb):
    a, b = W.operand_pair(na + 3 * nb, na, nb)
    out, _ = S.binpolymul(a, na, b, nb)
    assert np.array_equal(np.array(out, dtype=np.uint64), P.mul_bits(a, na, b, nb))
