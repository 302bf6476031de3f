"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds random-number generation and input shapes only: none of the
method's arithmetic.  The paper measures products of random polynomials of
power-of-two sizes (Table 2: 2^21 .. 2^29 bits per operand) with no stated
distribution; these generators stand in for its workloads at its sizes.

Generator (one definition, used everywhere):
  * splitmix64 seeds 2^16 independent xoshiro256** streams: stream s of seed
    S starts from four successive splitmix64 outputs of the state
    S * 2^32 + s.
  * Word i of a sequence is output number (i div 2^16) of stream (i mod 2^16).
A polynomial of n bits is the first ceil(n/64) words, bit i of word j being
the coefficient of x^(64 j + i), with bits >= n cleared.
"""
import math

import numpy as np

LANES = 1 << 16
_M64 = (1 << 64) - 1


def _splitmix64_next(state):
    """Vectorised splitmix64: returns (new_state, output)."""
    state = state + np.uint64(0x9E3779B97F4A7C15)
    z = state
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    z = z ^ (z >> np.uint64(31))
    return state, z


def _rotl(x, k):
    return (x << np.uint64(k)) | (x >> np.uint64(64 - k))


class WordStream:
    """The documented xoshiro256** sequence for one seed, read in order."""

    def __init__(self, seed, lanes=LANES):
        self.lanes = lanes
        with np.errstate(over="ignore"):
            st = (np.uint64(seed & 0xFFFFFFFF) << np.uint64(32)) + np.arange(lanes, dtype=np.uint64)
            s = []
            for _ in range(4):
                st, z = _splitmix64_next(st)
                s.append(z)
        self.s = s

    def steps(self, nsteps):
        """The next nsteps * lanes words (step-major, lane-minor)."""
        s0, s1, s2, s3 = self.s
        out = np.empty((nsteps, self.lanes), dtype=np.uint64)
        with np.errstate(over="ignore"):
            for t in range(nsteps):
                out[t] = _rotl(s1 * np.uint64(5), 7) * np.uint64(9)
                tt = s1 << np.uint64(17)
                s2 ^= s0
                s3 ^= s1
                s1 ^= s2
                s0 ^= s3
                s2 ^= tt
                s3 = _rotl(s3, 45)
        self.s = [s0, s1, s2, s3]
        return out.reshape(-1)


def random_words(seed, n):
    """n uint64 words of the documented xoshiro256** sequence for `seed`."""
    n = int(n)
    if n <= 0:
        return np.zeros(0, dtype=np.uint64)
    ws = WordStream(seed)
    return ws.steps((n + LANES - 1) // LANES)[:n].copy()


def _mask_top(words, nbits, top_bit):
    nw = (nbits + 63) // 64
    w = words[:nw]
    if nbits % 64:
        w[-1] &= np.uint64((1 << (nbits % 64)) - 1)
    if top_bit and nbits > 0:
        w[(nbits - 1) // 64] |= np.uint64(1 << ((nbits - 1) % 64))
    return w


def uniform_poly(seed, nbits, top_bit=True, offset_words=0):
    """Uniformly random polynomial of exactly nbits bits (top bit forced)."""
    nw = (nbits + 63) // 64
    w = random_words(seed, offset_words + nw)[offset_words:]
    return _mask_top(w, nbits, top_bit)


def operand_pair(seed, na_bits, nb_bits, top_bit=True):
    """Operands a then b drawn from one sequence: a takes the first
    ceil(na/64) words and b the next ceil(nb/64)."""
    nwa = (na_bits + 63) // 64
    nwb = (nb_bits + 63) // 64
    w = random_words(seed, nwa + nwb)
    a = _mask_top(w[:nwa].copy(), na_bits, top_bit)
    b = _mask_top(w[nwa:nwa + nwb].copy(), nb_bits, top_bit)
    return a, b


def all_ones(nbits):
    nw = (nbits + 63) // 64
    w = np.full(nw, np.uint64(_M64), dtype=np.uint64)
    return _mask_top(w, nbits, False)


def sparse_poly(seed, nbits, density=0.01, top_bit=True):
    """Each bit is 1 with probability `density`: bit k is set iff word k of
    the sequence is below density * 2^64.  Top bit forced."""
    nw = (nbits + 63) // 64
    thr = np.uint64(min(_M64, int(density * 2.0**64)))
    out = np.zeros(nw, dtype=np.uint64)
    weights = np.uint64(1) << np.arange(64, dtype=np.uint64)
    ws = WordStream(seed)
    w0 = 0
    step_chunk = 32  # 32 * 2^16 draws = 2^15 output words per chunk
    while w0 < nw:
        draws = ws.steps(step_chunk)
        nwc = min(nw - w0, draws.size // 64)
        bits = (draws[:64 * nwc] < thr).reshape(nwc, 64)
        out[w0:w0 + nwc] = np.bitwise_or.reduce(
            np.where(bits, weights, np.uint64(0)), axis=1)
        w0 += nwc
    return _mask_top(out, nbits, top_bit)


def log_uniform_lengths(seed, count, lo_log2, hi_log2):
    """count lengths floor(2^U), U ~ Uniform[lo, hi], from the sequence."""
    w = random_words(seed, count)
    u = (w >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    return np.floor(np.exp2(lo_log2 + (hi_log2 - lo_log2) * u)).astype(np.int64)


def poisson_arrivals(seed, rate_per_s, duration_s):
    """Arrival times (s) of a Poisson stream: exponential gaps from the
    sequence by inversion, -ln(1-u)/rate."""
    est = int(rate_per_s * duration_s * 1.5) + 64
    w = random_words(seed, est)
    u = (w >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    t = np.cumsum(-np.log1p(-u) / rate_per_s)
    return t[t < duration_s]


# Named workloads (sizes of the paper's Table 2 and of the benchmark configs).
WORKLOADS = {
    "c0_2^20": dict(na_bits=1 << 20, nb_bits=1 << 20, seed=0, kind="uniform"),
    "c1_2^28": dict(na_bits=1 << 28, nb_bits=1 << 28, seed=1, kind="uniform"),
    "c1_2^29": dict(na_bits=1 << 29, nb_bits=1 << 29, seed=2, kind="uniform"),
    "c1_2^28_ones": dict(na_bits=1 << 28, nb_bits=1 << 28, seed=None, kind="ones"),
    "c1_2^28_sparse": dict(na_bits=1 << 28, nb_bits=1 << 28, seed=3, kind="sparse"),
    "c1_2^29_ones": dict(na_bits=1 << 29, nb_bits=1 << 29, seed=None, kind="ones"),
    "c1_2^29_sparse": dict(na_bits=1 << 29, nb_bits=1 << 29, seed=3, kind="sparse"),
    "c1_2^28x2^16": dict(na_bits=1 << 28, nb_bits=1 << 16, seed=4, kind="uniform"),
    "c1_2^28+64": dict(na_bits=(1 << 28) + 64, nb_bits=(1 << 28) + 64, seed=12, kind="uniform"),
    "c1_2^28x64": dict(na_bits=1 << 28, nb_bits=64, seed=13, kind="uniform"),
    "c2_2^30": dict(na_bits=1 << 30, nb_bits=1 << 30, seed=5, kind="uniform"),
    "c2_2^32": dict(na_bits=1 << 32, nb_bits=1 << 32, seed=6, kind="uniform"),
}


def make_workload(name):
    spec = WORKLOADS[name]
    na, nb = spec["na_bits"], spec["nb_bits"]
    if spec["kind"] == "uniform":
        a, b = operand_pair(spec["seed"], na, nb)
    elif spec["kind"] == "ones":
        a, b = all_ones(na), all_ones(nb)
    elif spec["kind"] == "sparse":
        a = sparse_poly(spec["seed"], na)
        b = sparse_poly(spec["seed"] + 1000, nb)
    else:
        raise ValueError(spec["kind"])
    return a, na, b, nb


def log2_ceil(n):
    return 0 if n <= 1 else math.ceil(math.log2(n))
