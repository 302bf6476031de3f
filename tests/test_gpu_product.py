"""Parity of the whole product path (gf2x_mul through the C ABI) with the
CPU oracle, bit-exact, on seeded inputs."""
import numpy as np
import pytest
import torch

import paper_1708_09746_gb300 as G
from oracle import product as P
import workloads as W

from gpu_util import empty_dev, from_dev, gpu_mul, need_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def test_c0_2pow20_seed0():
    # 2^20 x 2^20 bits, seed 0, top bits forced: a 2^21-1-bit product.
    a, na, b, nb = W.make_workload("c0_2^20")
    got = gpu_mul(a, na, b, nb)
    want = P.mul(a, na, b, nb)
    assert np.array_equal(got, want)


SMALL = [(1, 1), (1, 64), (64, 1), (64, 64), (65, 63), (127, 129), (128, 128),
         (200, 3000), (3000, 200), (4096, 4096), (4097, 1), (1, 4097), (640, 700),
         (64 * 33, 64 * 31 + 5), (8191, 8193), (65536, 65536), (65536, 65535),
         (100000, 3), (131072 + 64, 131072 - 64),
         # b of 9 .. 16 words: its forward transform stops at layer 3
         (64 * 100, 64 * 16), (64 * 100, 64 * 9), (64 * 300, 64 * 32),
         # b of 2 .. 4 words under a bottom tile of 2^9 points: forward rows
         # below 3 only, on the product table; the inverse rows 0-2 in registers
         (64 * 300, 64 * 4), (64 * 300, 64 * 2), (64 * 200, 64 * 3 + 1)]


@pytest.mark.parametrize("na,nb", SMALL)
def test_small_and_ragged(na, nb):
    a, b = W.operand_pair(na * 31 + nb, na, nb)
    got = gpu_mul(a, na, b, nb)
    assert np.array_equal(got, P.mul(a, na, b, nb))


# Unbalanced operands (the long one at least four chunks of the short one's
# power-of-two size, 512 words or more) take the chunked product: chunks of
# the long operand times one transform of the short one, XORed into the
# output at their offsets; the last chunk may be one word
UNBALANCED = [(64 * 2048, 64 * 100), (64 * 100 + 5, 64 * 2048 + 1), (64 * 5000 + 3, 1),
              (64 * 4096 * 4 + 17, 64 * 600 + 3), (64 * 2049, 64 * 512), (64 * 2048, 64 * 513),
              (64 * 512 * 7 + 1, 64 * 512 - 7)]


@pytest.mark.parametrize("na,nb", UNBALANCED)
def test_unbalanced_chunked(na, nb):
    a, b = W.operand_pair(na * 3 + nb, na, nb)
    got = gpu_mul(a, na, b, nb)
    assert np.array_equal(got, P.mul(a, na, b, nb))


def test_unbalanced_chunked_async_stream():
    na, nb = 64 * 3000 + 9, 64 * 200 + 1
    a, b = W.operand_pair(4242, na, nb)
    want = P.mul(a, na, b, nb)
    da, db = to_dev(a), to_dev(b)
    out = empty_dev(len(want))
    s = torch.cuda.Stream()
    G.gf2x_mul_async(da, na, db, nb, out, s)
    s.synchronize()
    assert np.array_equal(from_dev(out, len(want)), want)


def test_random_sizes_sweep():
    rng = np.random.default_rng(77)
    for it in range(40):
        na = int(rng.integers(1, 1 << int(rng.integers(1, 17))))
        nb = int(rng.integers(1, 1 << int(rng.integers(1, 17))))
        a, b = W.operand_pair(1000 + it, na, nb, top_bit=bool(it % 2))
        assert np.array_equal(gpu_mul(a, na, b, nb), P.mul(a, na, b, nb)), (na, nb)


def test_bits_past_length_ignored():
    na, nb = 1000, 777
    a, b = W.operand_pair(5, na, nb)
    a_dirty, b_dirty = a.copy(), b.copy()
    a_dirty[-1] |= np.uint64(~((1 << (na % 64)) - 1) & (2**64 - 1))
    b_dirty[-1] |= np.uint64(~((1 << (nb % 64)) - 1) & (2**64 - 1))
    assert np.array_equal(gpu_mul(a_dirty, na, b_dirty, nb), P.mul(a, na, b, nb))


def _dirty(x, n):
    """x with every bit past its length n set in the last word (and one word
    more), which the product must ignore."""
    y = np.concatenate([x.copy(), np.array([~np.uint64(0)], dtype=np.uint64)])
    if n % 64:
        y[(n - 1) // 64] |= np.uint64(~((1 << (n % 64)) - 1) & (2**64 - 1))
    return y


# Operands of 2^17 words and more (their BasisCvt starts with the top VarSubs
# pass), with every bit past their lengths set: Split must pad with zeros and
# mask the last word; lengths past a power of two, 2^17- to 2^19-block
# conversions
SPLIT_LARGE = [((1 << 23) + 77, (1 << 23) - 5), ((1 << 24) + 1, (1 << 23) + 3),
             ((1 << 23) + 64, (1 << 22) + 7)]


@pytest.mark.parametrize("na,nb", SPLIT_LARGE)
def test_split_large_dirty(na, nb):
    a, b = W.operand_pair(na % 1009 + nb, na, nb)
    got = gpu_mul(_dirty(a, na), na, _dirty(b, nb), nb)
    assert np.array_equal(got, P.mul(a, na, b, nb))


def test_split_large_dirty_batched():
    # two products of one shape in one grouped launch: Split reads each
    # product's operand through its descriptor
    na, nb = (1 << 23) + 77, (1 << 23) - 5
    prods = [W.operand_pair(300 + i, na, nb) for i in range(2)]
    batch = G.gf2x_batch_create([na, na], [nb, nb], 1 << 30)
    try:
        da = [to_dev(_dirty(a, na)) for a, _ in prods]
        db = [to_dev(_dirty(b, nb)) for _, b in prods]
        outs = [empty_dev(G.gf2x_out_words(na, nb)) for _ in prods]
        G.gf2x_batch_execute(batch, da, db, outs)
        torch.cuda.synchronize()
        for (a, b), o in zip(prods, outs):
            want = P.mul(a, na, b, nb)
            assert np.array_equal(from_dev(o, len(want)), want)
    finally:
        G.gf2x_batch_destroy(batch)


def test_all_ones_and_sparse():
    n = 1 << 18
    o = W.all_ones(n)
    assert np.array_equal(gpu_mul(o, n, o, n), P.mul(o, n, o, n))
    s1 = W.sparse_poly(3, n)
    s2 = W.sparse_poly(1003, n)
    assert np.array_equal(gpu_mul(s1, n, s2, n), P.mul(s1, n, s2, n))


def test_zero_length_operand_writes_nothing():
    a = to_dev(W.uniform_poly(1, 100))
    out = torch.full((4,), 7, dtype=torch.int64, device="cuda")
    G.gf2x_mul(a, 100, a, 0, out)
    torch.cuda.synchronize()
    assert from_dev(out).tolist() == [7, 7, 7, 7]


def test_invalid_arguments():
    a = to_dev(W.uniform_poly(1, 640))
    out = empty_dev(32)
    # host pointer
    host = np.zeros(32, dtype=np.uint64)
    with pytest.raises(G.GF2XError) as e:
        G.gf2x_mul(host, 640, a, 640, out)
    assert e.value.status == -1
    # overlapping output
    with pytest.raises(G.GF2XError):
        G.gf2x_mul(a, 640, a, 640, a)
    # too large
    with pytest.raises(G.GF2XError):
        G.gf2x_mul(a, 1 << 40, a, 640, out)


def test_plan_api_and_host_api():
    na, nb = 50000, 70001
    a, b = W.operand_pair(9, na, nb)
    want = P.mul(a, na, b, nb)
    plan = G.gf2x_plan_create(na, nb)
    try:
        ws_bytes = G.gf2x_plan_workspace_bytes(plan)
        ws = torch.empty(ws_bytes // 8 + 32, dtype=torch.int64, device="cuda")
        da, db = to_dev(a), to_dev(b)
        out = empty_dev(len(want))
        s = torch.cuda.Stream()
        G.gf2x_plan_execute(plan, da, db, out, ws, s)
        s.synchronize()
        assert np.array_equal(from_dev(out, len(want)), want)
        out2 = empty_dev(len(want))
        G.gf2x_plan_execute(plan, da, db, out2, None, None)
        torch.cuda.synchronize()
        assert np.array_equal(from_dev(out2, len(want)), want)
    finally:
        G.gf2x_plan_destroy(plan)
    host_out = np.zeros(len(want), dtype=np.uint64)
    G.gf2x_mul_host(a, na, b, nb, host_out)
    assert np.array_equal(host_out, want)


@pytest.mark.parametrize("na,nb", [(1, 1), (64, 64), (65, 64), (129, 70), (190, 3),
                                   (1000, 777), (64 * 37 + 5, 64 * 11), (1 << 18, (1 << 18) - 3)])
def test_host_buffers_pieces(na, nb):
    # gf2x_mul_host writes its output in four pieces, each copied back while
    # the next is computed: outputs of 1 .. 3 words leave pieces empty
    a, b = W.operand_pair(na * 7 + nb, na, nb)
    want = P.mul(a, na, b, nb)
    host_out = np.full(len(want) + 2, 0xA5A5A5A5A5A5A5A5, dtype=np.uint64)
    pinned = torch.from_numpy(host_out.view(np.int64)).pin_memory()
    G.gf2x_mul_host(a, na, b, nb, pinned)
    got = pinned.numpy().view(np.uint64)
    assert np.array_equal(got[:len(want)], want)
    assert all(int(x) == 0xA5A5A5A5A5A5A5A5 for x in got[len(want):])


def test_batched_uneven():
    lens = W.log_uniform_lengths(7, 24, 6, 16)
    pairs = []
    for i in range(0, 24, 2):
        na, nb = int(lens[i]), int(lens[i + 1])
        a, b = W.operand_pair(500 + i, na, nb)
        pairs.append((a, na, b, nb))
    da = [to_dev(p[0]) for p in pairs]
    db = [to_dev(p[2]) for p in pairs]
    outs = [empty_dev(G.gf2x_out_words(p[1], p[3])) for p in pairs]
    G.gf2x_mul_batched(da, [p[1] for p in pairs], db, [p[3] for p in pairs], outs)
    torch.cuda.synchronize()
    for p, o in zip(pairs, outs):
        want = P.mul(p[0], p[1], p[2], p[3])
        assert np.array_equal(from_dev(o, len(want)), want)


@pytest.mark.parametrize("log_bits", [20, 24, 28])
def test_basis_cvt_takes_grouped_passes(log_bits):
    # Before launching, the BasisCvt schedule (register nodes, runs, class and
    # top passes) is expanded and compared with the level list of Alg. 3; a
    # mismatch falls back to one launch per division, which is correct but
    # slow.  The product must take the grouped passes: a handful of launches
    # per conversion, against 35 .. 231 divisions.
    n = 1 << log_bits
    a, b = W.operand_pair(log_bits, n, n)
    G.gf2x_profile_reset()
    G.gf2x_profile_enable(1)
    try:
        got = gpu_mul(a, n, b, n)
    finally:
        G.gf2x_profile_enable(0)
    st = G.profile_all()
    assert st["basis_cvt"][1] <= 2 * 8, st["basis_cvt"]
    assert st["ibasis_cvt"][1] <= 8, st["ibasis_cvt"]
    if log_bits <= 20:
        assert np.array_equal(got, P.mul(a, n, b, n))


def test_plain_launches_without_programmatic_dependence():
    # the product path's kernels are launched with programmatic dependent
    # launch; GF2X_PDL=0 launches them in plain stream order: the same product
    import os
    import subprocess
    import sys
    na, nb = (1 << 20) + 3, (1 << 19) - 5
    code = (
        "import numpy as np, paper_1708_09746_gb300 as G, workloads as W\n"
        "from oracle import product as P\n"
        "import sys; sys.path.insert(0, 'tests')\n"
        "from gpu_util import gpu_mul\n"
        "a, b = W.operand_pair(99, %d, %d)\n"
        "assert np.array_equal(gpu_mul(a, %d, b, %d), P.mul(a, %d, b, %d))\n"
        "print('ok')\n" % (na, nb, na, nb, na, nb))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, GF2X_PDL="0")
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stderr[-2000:]
