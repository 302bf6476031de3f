"""Stage-by-stage parity of the GPU kernels with the stage reference
(oracle/stages.py), through the C ABI's stage entry points."""
import numpy as np
import pytest
import torch

import paper_1708_09746_gb300 as G
from oracle import stages as S
import workloads as W

from gpu_util import empty_dev, from_dev, ints_to_pairs, need_gpu, pairs_to_ints, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _rand128(seed, n):
    w = W.random_words(seed, 2 * n)
    return pairs_to_ints(w)


@pytest.mark.parametrize("log_n", [0, 1, 2, 4, 7, 11, 12, 13, 14, 16, 18, 20])
def test_basis_cvt64(log_n):
    n = 1 << log_n
    f = W.random_words(100 + log_n, n)
    want = S.basis_cvt([int(x) for x in f])
    d = to_dev(f)
    G.gf2x_stage_basis_cvt64(d, log_n, 0)
    got = from_dev(d, n)
    assert [int(x) for x in got] == want
    G.gf2x_stage_basis_cvt64(d, log_n, 1)
    assert np.array_equal(from_dev(d, n), f)


@pytest.mark.parametrize("log_n", [1, 3, 10, 11, 12, 13, 15, 17, 19])
def test_basis_cvt128(log_n):
    n = 1 << log_n
    f = _rand128(200 + log_n, n)
    g = S.basis_cvt(f)
    d = to_dev(ints_to_pairs(f))
    G.gf2x_stage_basis_cvt128(d, log_n, 0)
    assert pairs_to_ints(from_dev(d, 2 * n)) == g
    # iBasisCvt: the inverse returns the monomial coefficients
    d2 = to_dev(ints_to_pairs(g))
    G.gf2x_stage_basis_cvt128(d2, log_n, 1)
    assert pairs_to_ints(from_dev(d2, 2 * n)) == f


def test_ibasis_cvt_definition_small():
    n = 64
    g = _rand128(5, n)
    d = to_dev(ints_to_pairs(g))
    G.gf2x_stage_basis_cvt128(d, 6, 1)
    assert pairs_to_ints(from_dev(d, 2 * n)) == S.ibasis_cvt(g)


@pytest.mark.parametrize("p,n", [(1, 1), (1, 8), (4, 16), (1024, 1024), (4096, 16384)])
def test_chrepr(p, n):
    g = W.random_words(300 + n, p)
    dg = to_dev(g)
    F = empty_dev(2 * n)
    G.gf2x_stage_chrepr(dg, p, F, n)
    got = pairs_to_ints(from_dev(F, 2 * n))
    phi = [S.chrepr(int(w)) for w in g]
    assert got == [phi[i % p] for i in range(n)]


# bottom tiles of 2^8 .. 2^12 points run rows 0-2 in registers with per-lane
# tables, smaller ones on the product table: both sides of the switch
@pytest.mark.parametrize("log_n,log_p", [(1, 1), (1, 0), (4, 3), (6, 6), (7, 7), (8, 8), (9, 4),
                                         (10, 9), (11, 11), (12, 12), (12, 7)])
def test_fft_forward(log_n, log_p):
    n, p = 1 << log_n, 1 << log_p
    g = _rand128(400 + log_n, p)
    # the fan-out: the input holds the p coefficients repeated n/p times
    d = to_dev(ints_to_pairs([g[i % p] for i in range(n)]))
    G.gf2x_stage_fft(d, log_n, log_p, 0)
    got = pairs_to_ints(from_dev(d, 2 * n))
    want = S.fft_lch(g + [0] * (n - p), 0)
    assert got == want


@pytest.mark.parametrize("log_n", [1, 5, 7, 8, 9, 10, 11, 12])
def test_fft_inverse(log_n):
    n = 1 << log_n
    vals = _rand128(500 + log_n, n)
    d = to_dev(ints_to_pairs(vals))
    G.gf2x_stage_fft(d, log_n, log_n, 1)
    assert pairs_to_ints(from_dev(d, 2 * n)) == S.ifft_lch(vals, 0)


@pytest.mark.parametrize("log_n,log_p,points", [(13, 13, 4), (16, 16, 3), (18, 18, 2), (19, 19, 2),
                                                (20, 20, 2), (20, 14, 2)])
def test_fft_strided_passes(log_n, log_p, points):
    # Sizes with layers above the 4096-point tile run strided passes (one
    # to three); outputs are checked at sampled points against the direct
    # evaluation f(i) = sum_j g_j X_j(i), and the inverse must undo the
    # forward transform exactly.
    n, p = 1 << log_n, 1 << log_p
    w = W.random_words(450 + log_n + log_p, 2 * p)
    g = np.zeros(2 * n, dtype=np.uint64)
    for r in range(n // p):
        g[2 * p * r: 2 * p * (r + 1)] = w
    d = to_dev(g)
    G.gf2x_stage_fft(d, log_n, log_p, 0)
    got = from_dev(d, 2 * n).copy()
    rng = np.random.default_rng(log_n * 31 + log_p)
    idx = [n - 1] + [int(x) for x in rng.integers(0, n, points - 1)]
    glo, ghi = w[0::2].copy(), w[1::2].copy()
    for i in idx:
        want = S.eval_novelpoly_np(glo, ghi, i)
        assert int(got[2 * i]) | (int(got[2 * i + 1]) << 64) == want, i
    G.gf2x_stage_fft(d, log_n, log_n, 1)
    back = from_dev(d, 2 * n)
    want_back = np.zeros(2 * n, dtype=np.uint64)
    want_back[: 2 * p] = w
    assert np.array_equal(back, want_back)


def test_fft_horner_spot_check():
    log_n = 11
    n = 1 << log_n
    g = _rand128(600, n // 2)
    d = to_dev(ints_to_pairs(g + g))
    G.gf2x_stage_fft(d, log_n, log_n - 1, 0)
    got = pairs_to_ints(from_dev(d, 2 * n))
    for i in [0, 1, 2, 777, n // 2, n - 1]:
        assert got[i] == S.eval_novelpoly(g, i)


def test_pointmul():
    n = 1 << 14
    A = W.random_words(700, 2 * n)
    B = W.random_words(701, 2 * n)
    dA, dB = to_dev(A), to_dev(B)
    dC = empty_dev(2 * n)
    G.gf2x_stage_pointmul(dA, dB, dC, n)
    lo, hi = S.tmul_vec(A[0::2], A[1::2], B[0::2], B[1::2])
    got = from_dev(dC, 2 * n)
    assert np.array_equal(got[0::2], lo) and np.array_equal(got[1::2], hi)
    # in place into B
    G.gf2x_stage_pointmul(dA, dB, dB, n)
    got = from_dev(dB, 2 * n)
    assert np.array_equal(got[0::2], lo) and np.array_equal(got[1::2], hi)


def test_ichrepr_combine():
    n = 512
    # products of chunk polynomials have degree <= 126: build such elements
    polys = [(int(x) & ((1 << 127) - 1)) for x in _rand128(800, n)]
    F = [S.chrepr(q) for q in polys]
    d = to_dev(ints_to_pairs(F))
    for total_bits in (64 * n + 64, 64 * n + 63, 64 * n - 5, 100):
        ow = (total_bits + 63) // 64
        out = empty_dev(ow)
        G.gf2x_stage_ichrepr_combine(d, n, out, total_bits)
        got = [int(x) for x in from_dev(out, ow)]
        want = S.interleaved_combine(polys, ow)
        if total_bits % 64:
            want[-1] &= (1 << (total_bits % 64)) - 1
        assert got == want
