"""Batched products (grouped launches, CUDA-graph replay) and the serving
loop (memory admission, continuous batching, bounded waits): every result is
bit-exact against the CPU oracle and identical to the same product alone."""
import numpy as np
import pytest
import torch

import paper_1708_09746_gb300 as G
from oracle import product as P
import workloads as W

from gpu_util import empty_dev, from_dev, need_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()


def _pairs(seed, n, lo, hi, dup_every=3):
    lens = W.log_uniform_lengths(seed, 2 * n, lo, hi)
    out = []
    for i in range(n):
        na, nb = int(lens[2 * i]), int(lens[2 * i + 1])
        if dup_every and i % dup_every == 2:  # same shape as the previous product
            na, nb = out[-1][1], out[-1][3]
        a, b = W.operand_pair(seed * 1000 + i, na, nb)
        out.append((a, na, b, nb))
    return out


def _alone(a, na, b, nb):
    ow = G.gf2x_out_words(na, nb)
    o = empty_dev(ow)
    G.gf2x_mul(to_dev(a), na, to_dev(b), nb, o)
    torch.cuda.synchronize()
    return from_dev(o, ow)


def test_batch_plan_graph_replay():
    prods = _pairs(11, 40, 6, 16)
    prods.append((W.uniform_poly(1, 64), 64, W.uniform_poly(2, 1), 0))  # empty product
    na = [p[1] for p in prods]
    nb = [p[3] for p in prods]
    batch = G.gf2x_batch_create(na, nb, 64 << 20)
    try:
        assert G.gf2x_batch_workspace_bytes(batch) > 0
        for rep in range(2):  # capture on the first execution, replay on the second
            if rep == 1:
                prods = [(W.uniform_poly(500 + i, p[1]), p[1], W.uniform_poly(900 + i, p[3]), p[3])
                         for i, p in enumerate(prods)]
            da = [to_dev(p[0]) for p in prods]
            db = [to_dev(p[2]) for p in prods]
            outs = [empty_dev(G.gf2x_out_words(p[1], p[3])) for p in prods]
            s = torch.cuda.Stream()
            G.gf2x_batch_execute(batch, da, db, outs, s)
            s.synchronize()
            for p, o in zip(prods, outs):
                if p[3] == 0:
                    continue
                want = P.mul(p[0], p[1], p[2], p[3])
                assert np.array_equal(from_dev(o, len(want)), want), (p[1], p[3])
    finally:
        G.gf2x_batch_destroy(batch)


def test_batch_chunks_under_small_budget():
    # a budget of one product's workspace forces one product per launch
    prods = _pairs(12, 9, 10, 14, dup_every=1)
    na = [p[1] for p in prods]
    nb = [p[3] for p in prods]
    batch = G.gf2x_batch_create(na, nb, 1)
    try:
        da = [to_dev(p[0]) for p in prods]
        db = [to_dev(p[2]) for p in prods]
        outs = [empty_dev(G.gf2x_out_words(p[1], p[3])) for p in prods]
        G.gf2x_batch_execute(batch, da, db, outs)
        torch.cuda.synchronize()
        for p, o in zip(prods, outs):
            want = P.mul(p[0], p[1], p[2], p[3])
            assert np.array_equal(from_dev(o, len(want)), want)
    finally:
        G.gf2x_batch_destroy(batch)


def test_server_mix_equals_alone():
    prods = _pairs(13, 60, 6, 18)
    # a few highly unequal pairs, as in the serving workload: a short operand
    # of 16 words (direct products) and operands of 2^14 x 512 words (by
    # chunks of the longer one), in both orders
    for i in range(4):
        a, b = W.operand_pair(77 + i, 1 << 18, 1 << 10)
        prods.append((a, 1 << 18, b, 1 << 10))
    for i in range(2):
        a, b = W.operand_pair(90 + i, 1 << 20, (1 << 15) - 3)
        prods.append((a, 1 << 20, b, (1 << 15) - 3) if i == 0 else (b, (1 << 15) - 3, a, 1 << 20))
    assert G.gf2x_product_path(1 << 20, (1 << 15) - 3)[0] == 1
    sv = G.gf2x_server_create(256 << 20, 4)
    try:
        da = [to_dev(p[0]) for p in prods]
        db = [to_dev(p[2]) for p in prods]
        outs = [empty_dev(G.gf2x_out_words(p[1], p[3])) for p in prods]
        torch.cuda.synchronize()
        tickets = [G.gf2x_server_submit(sv, da[i], p[1], db[i], p[3], outs[i])
                   for i, p in enumerate(prods)]
        for t in tickets:
            G.gf2x_server_wait(sv, t, 30_000_000)
        for i, p in enumerate(prods):
            got = from_dev(outs[i], G.gf2x_out_words(p[1], p[3]))
            assert np.array_equal(got, _alone(*p)), i
            if i % 7 == 0:
                assert np.array_equal(got, P.mul(p[0], p[1], p[2], p[3]))
        p50, p99, thr, done = G.gf2x_server_stats(sv)
        assert done == len(prods)
        assert 0 < p50 <= p99 and thr > 0
    finally:
        G.gf2x_server_destroy(sv)


def test_server_memory_admission_and_limits():
    n = 1 << 20
    plan = G.gf2x_plan_create(n, n)
    ws = G.gf2x_plan_workspace_bytes(plan)
    G.gf2x_plan_destroy(plan)
    # room for one such product at a time: the others wait for memory
    sv = G.gf2x_server_create(ws + (ws // 2), 4)
    try:
        prods = [W.operand_pair(300 + i, n, n) for i in range(4)]
        da = [to_dev(a) for a, _ in prods]
        db = [to_dev(b) for _, b in prods]
        outs = [empty_dev(G.gf2x_out_words(n, n)) for _ in prods]
        torch.cuda.synchronize()
        tickets = [G.gf2x_server_submit(sv, da[i], n, db[i], n, outs[i]) for i in range(4)]
        # a wait that runs out reports the timeout and leaves the ticket valid
        with pytest.raises(G.GF2XError) as e:
            G.gf2x_server_wait(sv, tickets[-1], 0)
        assert e.value.status == G.GF2X_ETIMEOUT
        for t in tickets:
            G.gf2x_server_wait(sv, t, 60_000_000)
        for i, (a, b) in enumerate(prods):
            want = P.mul(a, n, b, n)
            assert np.array_equal(from_dev(outs[i], len(want)), want)
        # a product whose workspace can never fit the arena is refused
        big = to_dev(W.uniform_poly(5, 1 << 22))
        out = empty_dev(G.gf2x_out_words(1 << 22, 1 << 22))
        with pytest.raises(G.GF2XError) as e:
            G.gf2x_server_submit(sv, big, 1 << 22, big, 1 << 22, out)
        assert e.value.status == G.GF2X_EINVAL
    finally:
        G.gf2x_server_destroy(sv)


def test_batch_tuned_in_batch_context():
    prods = _pairs(14, 48, 10, 18)
    na = [p[1] for p in prods]
    nb = [p[3] for p in prods]
    batch = G.gf2x_batch_create(na, nb, 256 << 20)
    try:
        da = [to_dev(p[0]) for p in prods]
        db = [to_dev(p[2]) for p in prods]
        outs = [empty_dev(G.gf2x_out_words(p[1], p[3])) for p in prods]
        s = torch.cuda.Stream()
        with pytest.raises(G.GF2XError):  # nothing to tune on before an execution
            G.gf2x_batch_tune(batch, 1)
        G.gf2x_batch_execute(batch, da, db, outs, s)
        before, after = G.gf2x_batch_tune(batch, 1)
        assert 0 < after <= before
        for o in outs:
            o.zero_()
        G.gf2x_batch_execute(batch, da, db, outs, s)  # the tuned plans, captured again
        G.gf2x_batch_status(batch)
        for p, o in zip(prods, outs):
            want = P.mul(p[0], p[1], p[2], p[3])
            assert np.array_equal(from_dev(o, len(want)), want), (p[1], p[3])
    finally:
        G.gf2x_batch_destroy(batch)
