"""Device-side failures reach the call that caused them.

Every wait inside the FFT pass kernel is bounded; a wait that runs out ends the
kernel early (after the copies it started have landed) and records
GF2X_ETIMEOUT in the status word of the launching call.  The tests make the
waits run out on purpose with gf2x_debug_set_wait_spins(0) (every wait gives
up at once, without waiting: nothing faults and nothing hangs) and check that
the timeout is reported to that call, stream, batch or server request only,
and that the next product with the default bound is exact.

The products are 2^20 x 2^20 bits: N = 2^15 points, so the first FFT pass of
each operand is a strided pass whose tiles arrive by bulk copies on an
mbarrier (the waits that are made to run out).
"""
import numpy as np
import pytest
import torch

import paper_1708_09746_gb300 as G
from oracle import product as P
import workloads as W

from gpu_util import empty_dev, from_dev, need_gpu, to_dev

pytestmark = pytest.mark.gpu

NA = NB = 1 << 20


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()
    yield
    G.gf2x_debug_set_wait_spins(-1)


@pytest.fixture(scope="module")
def pair():
    a, b = W.operand_pair(31, NA, NB)
    return a, b, P.mul(a, NA, b, NB)


class _short_waits:
    def __enter__(self):
        G.gf2x_debug_set_wait_spins(0)

    def __exit__(self, *exc):
        G.gf2x_debug_set_wait_spins(-1)


def _exact(da, db, want):
    ow = len(want)
    out = empty_dev(ow)
    G.gf2x_mul(da, NA, db, NB, out)
    assert np.array_equal(from_dev(out, ow), want)


def test_async_timeout_goes_to_its_stream(pair):
    a, b, want = pair
    da, db = to_dev(a), to_dev(b)
    out = empty_dev(len(want))
    s = torch.cuda.Stream()
    with _short_waits():
        G.gf2x_mul_async(da, NA, db, NB, out, s)
    s.synchronize()
    # a synchronous product after it is not charged with the other stream's
    # timeout, and is exact
    _exact(da, db, want)
    with pytest.raises(G.GF2XError) as e:
        G.gf2x_stream_status(s)
    assert e.value.status == G.GF2X_ETIMEOUT
    G.gf2x_stream_status(s)  # read once, then cleared
    # an untouched stream reports nothing
    G.gf2x_stream_status(torch.cuda.Stream())


def test_sync_call_reports_its_own_timeout(pair):
    a, b, want = pair
    da, db = to_dev(a), to_dev(b)
    out = empty_dev(len(want))
    with _short_waits():
        with pytest.raises(G.GF2XError) as e:
            G.gf2x_mul(da, NA, db, NB, out)
    assert e.value.status == G.GF2X_ETIMEOUT
    _exact(da, db, want)
    with _short_waits():
        with pytest.raises(G.GF2XError) as e:
            G.gf2x_mul_host(a, NA, b, NB, np.zeros(len(want), dtype=np.uint64))
    assert e.value.status == G.GF2X_ETIMEOUT
    host_out = np.zeros(len(want), dtype=np.uint64)
    G.gf2x_mul_host(a, NA, b, NB, host_out)
    assert np.array_equal(host_out, want)


def test_batch_timeout_goes_to_its_batch(pair):
    a, b, want = pair
    da, db = to_dev(a), to_dev(b)
    ow = len(want)
    s = torch.cuda.Stream()
    # a batch captured (at its first execution) while the waits give up at
    # once keeps that bound in its graph; it reports the timeout through
    # gf2x_batch_status
    bad = G.gf2x_batch_create([NA, NA], [NB, NB], 64 << 20)
    try:
        outs = [empty_dev(ow), empty_dev(ow)]
        with _short_waits():
            G.gf2x_batch_execute(bad, [da, da], [db, db], outs, s)
        with pytest.raises(G.GF2XError) as e:
            G.gf2x_batch_status(bad)
        assert e.value.status == G.GF2X_ETIMEOUT
    finally:
        G.gf2x_batch_destroy(bad)
    good = G.gf2x_batch_create([NA, NA], [NB, NB], 64 << 20)
    try:
        outs = [empty_dev(ow), empty_dev(ow)]
        G.gf2x_batch_execute(good, [da, da], [db, db], outs, s)
        G.gf2x_batch_status(good)
        for o in outs:
            assert np.array_equal(from_dev(o, ow), want)
    finally:
        G.gf2x_batch_destroy(good)
    G.gf2x_stream_status(s)  # the batches used their own words, not the stream's


def test_server_timeout_goes_to_its_request(pair):
    a, b, want = pair
    da, db = to_dev(a), to_dev(b)
    ow = len(want)
    sv = G.gf2x_server_create(256 << 20, 2, 8)
    try:
        out = empty_dev(ow)
        with _short_waits():
            t = G.gf2x_server_submit(sv, da, NA, db, NB, out)
            with pytest.raises(G.GF2XError) as e:
                G.gf2x_server_wait(sv, t, 30_000_000)
        assert e.value.status == G.GF2X_ETIMEOUT
        out2 = empty_dev(ow)
        t2 = G.gf2x_server_submit(sv, da, NA, db, NB, out2)
        G.gf2x_server_wait(sv, t2, 30_000_000)
        assert np.array_equal(from_dev(out2, ow), want)
    finally:
        G.gf2x_server_destroy(sv)
