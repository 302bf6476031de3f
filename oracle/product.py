"""ctypes wrapper over the C oracle (gf2x_oracle.c).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

All polynomials are numpy uint64 arrays, bit i of word j = coefficient of
x^(64 j + i) (the packing reading of Sec. 2.1).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        L.gf2o_clmul64.argtypes = [ctypes.c_uint64, ctypes.c_uint64, u64p, u64p]
        L.gf2o_mul_schoolbook.argtypes = [u64p, ctypes.c_int64, u64p,
                                          ctypes.c_int64, u64p]
        L.gf2o_mul_karatsuba.argtypes = [u64p, ctypes.c_int64, u64p,
                                         ctypes.c_int64, u64p, ctypes.c_int]
        L.gf2o_mul_karatsuba.restype = ctypes.c_int
        L.gf2o_mul_bits.argtypes = [u64p, ctypes.c_int64, u64p, ctypes.c_int64,
                                    u64p, ctypes.c_int64]
        L.gf2o_poly_mod64.argtypes = [u64p, ctypes.c_int64, ctypes.c_uint64]
        L.gf2o_poly_mod64.restype = ctypes.c_uint64
        L.gf2o_mulmod64.argtypes = [ctypes.c_uint64, ctypes.c_uint64,
                                    ctypes.c_uint64]
        L.gf2o_mulmod64.restype = ctypes.c_uint64
        L.gf2o_num_threads.restype = ctypes.c_int
        L.gf2o_product_word.argtypes = [u64p, ctypes.c_int64, u64p, ctypes.c_int64,
                                        ctypes.c_int64]
        L.gf2o_product_word.restype = ctypes.c_uint64
        L.gf2o_clmul64_win4.argtypes = [ctypes.c_uint64, ctypes.c_uint64, u64p, u64p]
        L.gf2o_clmul64_fast.argtypes = [ctypes.c_uint64, ctypes.c_uint64, u64p, u64p]
        L.gf2o_clmul_kind.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(arr):
    return arr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _words(x, nbits):
    """Copy of the first ceil(nbits/64) words with bits >= nbits cleared."""
    nw = (nbits + 63) // 64
    a = np.ascontiguousarray(np.asarray(x, dtype=np.uint64)[:nw]).copy()
    if nbits % 64 and nw:
        a[-1] &= np.uint64((1 << (nbits % 64)) - 1)
    return a


def out_words(na_bits, nb_bits):
    """Words of the product of an na-bit and an nb-bit polynomial."""
    if na_bits == 0 or nb_bits == 0:
        return 0
    return (na_bits + nb_bits - 1 + 63) // 64


def clmul64(x, y):
    lo = ctypes.c_uint64()
    hi = ctypes.c_uint64()
    lib().gf2o_clmul64(int(x), int(y), ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def clmul64_win4(x, y):
    lo = ctypes.c_uint64()
    hi = ctypes.c_uint64()
    lib().gf2o_clmul64_win4(int(x), int(y), ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def clmul64_fast(x, y):
    """The form the product routines use (PMULL where the host has it)."""
    lo = ctypes.c_uint64()
    hi = ctypes.c_uint64()
    lib().gf2o_clmul64_fast(int(x), int(y), ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def clmul_kind():
    """'pmull' or 'win4': the carry-less multiply the product routines use."""
    return "pmull" if lib().gf2o_clmul_kind() == 1 else "win4"


def mul_schoolbook(a, na_bits, b, nb_bits):
    A, B = _words(a, na_bits), _words(b, nb_bits)
    ow = out_words(na_bits, nb_bits)
    if ow == 0:
        return np.zeros(0, dtype=np.uint64)
    out = np.zeros(len(A) + len(B), dtype=np.uint64)
    lib().gf2o_mul_schoolbook(_p(A), len(A), _p(B), len(B), _p(out))
    return out[:ow]


def mul_karatsuba(a, na_bits, b, nb_bits, par_depth=0):
    A, B = _words(a, na_bits), _words(b, nb_bits)
    ow = out_words(na_bits, nb_bits)
    if ow == 0:
        return np.zeros(0, dtype=np.uint64)
    out = np.zeros(len(A) + len(B), dtype=np.uint64)
    rc = lib().gf2o_mul_karatsuba(_p(A), len(A), _p(B), len(B), _p(out),
                                   int(par_depth))
    if rc != 0:
        raise MemoryError("oracle Karatsuba allocation failed")
    return out[:ow]


def mul_bits(a, na_bits, b, nb_bits):
    A, B = _words(a, na_bits), _words(b, nb_bits)
    ow = out_words(na_bits, nb_bits)
    if ow == 0:
        return np.zeros(0, dtype=np.uint64)
    out = np.zeros(ow, dtype=np.uint64)
    lib().gf2o_mul_bits(_p(A), na_bits, _p(B), nb_bits, _p(out), ow)
    return out


def mul(a, na_bits, b, nb_bits, threads=None):
    """The oracle product: schoolbook for short operands, Karatsuba above."""
    nw = max((na_bits + 63) // 64, (nb_bits + 63) // 64)
    if nw <= 64:
        return mul_schoolbook(a, na_bits, b, nb_bits)
    depth = 0
    if threads is None:
        threads = lib().gf2o_num_threads()
    if threads > 1 and nw >= 4096:
        # enough tasks (3^depth) to keep every thread busy, and no deeper than
        # the recursion itself (halving down to the 32-word base case)
        depth = 1
        while 3 ** depth < 4 * threads and (nw >> (depth + 1)) >= 64:
            depth += 1
    return mul_karatsuba(a, na_bits, b, nb_bits, par_depth=depth)


def product_word(a, na_bits, b, nb_bits, j):
    """Word j of a*b from the definition (for sampled checks of long
    products).  The caller masks bits >= total length in the last word."""
    A, B = _words(a, na_bits), _words(b, nb_bits)
    return int(lib().gf2o_product_word(_p(A), len(A), _p(B), len(B), int(j)))


def poly_mod64(a, nbits, r_low):
    """a(x) mod (x^64 + r_low(x))."""
    A = _words(a, nbits)
    return lib().gf2o_poly_mod64(_p(A), len(A), int(r_low))


def mulmod64(x, y, r_low):
    return lib().gf2o_mulmod64(int(x), int(y), int(r_low))


def num_threads():
    return lib().gf2o_num_threads()


# ---------------------------------------------------------------------------
# Degree-64 irreducible moduli for the fingerprint check.


def _pmod(a, m):
    """Remainder of Python-int GF(2) polynomials."""
    dm = m.bit_length() - 1
    while a and a.bit_length() - 1 >= dm:
        a ^= m << (a.bit_length() - 1 - dm)
    return a


def _pgcd(a, b):
    while b:
        a, b = b, _pmod(a, b)
    return a


def is_irreducible64(r_low):
    """Rabin's test for r = x^64 + r_low: x^(2^64) = x mod r and
    gcd(x^(2^32) - x, r) = 1 (64 has the single prime divisor 2)."""
    r = (1 << 64) | int(r_low)
    v = 2  # the polynomial x
    for i in range(64):
        v = mulmod64(v, v, r_low)
        if i == 31:
            if _pgcd(r, v ^ 2) != 1:
                return False
    return v == 2


def random_irreducible64(rng):
    """A random degree-64 irreducible polynomial (returned without x^64)."""
    while True:
        r_low = int(rng.integers(0, 2**63, dtype=np.uint64)) * 2 + 1
        if is_irreducible64(r_low):
            return r_low


def fingerprint_ok(a, na_bits, b, nb_bits, c, r_low):
    """(a mod r)(b mod r) mod r == c mod r; a wrong c passes with probability
    about deg(c)/2^64 for a random irreducible r."""
    ow = out_words(na_bits, nb_bits)
    ra = poly_mod64(a, na_bits, r_low)
    rb = poly_mod64(b, nb_bits, r_low)
    rc = poly_mod64(np.asarray(c, dtype=np.uint64)[:ow], 64 * ow, r_low) if ow else 0
    return mulmod64(ra, rb, r_low) == rc
