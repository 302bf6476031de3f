"""Products by a short operand (no transform) and the tail split of products
just above a power-of-two length, against the oracle.

gf2x_mul multiplies directly when the shorter operand has at most 16 words,
and, when cutting at most 16 words off the operands halves the transform,
computes a0 b0 with the half-length transform and adds the tail products
directly (a b = a0 b0 + x^(64 A) a1 b + x^(64 B) a0 b1, distributivity).
Every product here is compared word for word with the oracle's, or at the
full 2^28 + 64-bit size with sampled words from the definition and modular
fingerprints; gf2x_product_path confirms which way each product went.
"""
import numpy as np
import pytest
import torch

import paper_1708_09746_gb300 as G
from oracle import product as P
import workloads as W

from gpu_util import gpu_mul, need_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


SHORT = [1, 2, 63, 64, 65, 127, 200, 640, 1023, 1024]          # at most 16 words
LONG = [1, 70, 1000, 4096, 65536 + 13, (1 << 20) + 3, (1 << 22) + 777]


@pytest.mark.parametrize("ns", SHORT)
def test_direct_short_operand(ns):
    for i, nl in enumerate(LONG):
        for na, nb in ((nl, ns), (ns, nl)):
            a, b = W.operand_pair(ns * 31 + i, na, nb)
            assert G.gf2x_product_path(na, nb)[0] == 2
            got = gpu_mul(a, na, b, nb)
            assert np.array_equal(got, P.mul(a, na, b, nb)), (na, nb)


@pytest.mark.parametrize("aw,bw,extra_bits", [
    ((1 << 14) + 1, (1 << 14) + 1, 0),    # one word past half the transform
    ((1 << 14) + 1, (1 << 14) + 1, -17),  # ragged last word
    ((1 << 14) + 8, (1 << 14) + 9, -5),   # 16 words past: still split
    (49152 + 2, (1 << 14) + 1, 0),        # unbalanced (not chunked): two words past
    ((1 << 13) + 20, (1 << 13) - 4, -1),
])
def test_tail_split(aw, bw, extra_bits):
    na, nb = 64 * aw + extra_bits, 64 * bw
    path, A, B = G.gf2x_product_path(na, nb)
    assert path == 3, (na, nb, path)
    assert A + B - 1 <= G.gf2x_fft_points(na, nb) // 2
    a, b = W.operand_pair(aw + bw, na, nb)
    got = gpu_mul(a, na, b, nb)
    assert np.array_equal(got, P.mul(a, na, b, nb))


def test_no_split_past_sixteen_words():
    aw = bw = (1 << 14) + 9  # 17 words past half the transform
    assert G.gf2x_product_path(64 * aw, 64 * bw)[0] == 0
    a, b = W.operand_pair(5, 64 * aw, 64 * bw)
    assert np.array_equal(gpu_mul(a, 64 * aw, b, 64 * bw), P.mul(a, 64 * aw, b, 64 * bw))


@pytest.mark.parametrize("name", ["c1_2^28+64", "c1_2^28x64"])
def test_fullsize_split_and_direct(name):
    a, na, b, nb = W.make_workload(name)
    assert G.gf2x_product_path(na, nb)[0] == (3 if name == "c1_2^28+64" else 2)
    ow = G.gf2x_out_words(na, nb)
    out = torch.full((ow + 2,), -0x5A5A5A5A5A5A5A5B, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    G.gf2x_mul_async(to_dev(a), na, to_dev(b), nb, out, s)
    s.synchronize()
    res = out.cpu().numpy().view(np.uint64)
    assert all(int(x) == 0xA5A5A5A5A5A5A5A5 for x in res[ow:])
    c = res[:ow]
    rng = np.random.default_rng(na % 1000)
    rem = (na + nb - 1) % 64
    top = (1 << rem) - 1 if rem else 2**64 - 1
    pos = {0, 1, ow - 1, ow - 2, (1 << 22) - 1, 1 << 22, (1 << 22) + 1, ow // 2}
    pos.update(int(x) for x in rng.integers(0, ow, 8))
    for j in sorted(p for p in pos if 0 <= p < ow):
        want = P.product_word(a, na, b, nb, j)
        if j == ow - 1:
            want &= top
        assert int(c[j]) == want, j
    for _ in range(3):
        r = P.random_irreducible64(rng)
        assert P.fingerprint_ok(a, na, b, nb, c, r)


def test_host_call_with_pinned_buffers():
    # page-locked and pageable host buffers (staged copies on the library's
    # streams either way)
    for na, nb in [((1 << 20) + 77, (1 << 19) + 5), (1 << 22, 1 << 22)]:
        a, b = W.operand_pair(na % 97, na, nb)
        ow = G.gf2x_out_words(na, nb)
        ha = torch.from_numpy(a.view(np.int64).copy()).pin_memory()
        hb = torch.from_numpy(b.view(np.int64).copy()).pin_memory()
        ho = torch.full((ow,), -1, dtype=torch.int64).pin_memory()
        G.gf2x_mul_host(ha, na, hb, nb, ho)
        want = P.mul(a, na, b, nb)
        assert np.array_equal(ho.numpy().view(np.uint64), want)
        ho2 = np.full(ow, 7, dtype=np.uint64)   # pageable output
        G.gf2x_mul_host(ha, na, hb, nb, ho2)
        assert np.array_equal(ho2, want)
