"""Step-by-step restatement of the paper's stages, slow and plain.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Used to check each GPU
stage on its own; the end-to-end oracle is oracle.product (the plain
carry-less product).

Field elements of the tower \\tilde F_{2^128} (Sec. 3.2) are Python ints (or
pairs of numpy uint64 arrays lo/hi in the vectorised helpers): bit i is the
coefficient of the tower basis vector v_i (Def. 3.1), so the integer i is the
representative \\bar{i} (Def. 3.2) and the subfield \\tilde F_{2^(2^k)} is
the low 2^k bits.

Readings of the paper used here:
  * changeRepr (Alg. 5, Sec. 4.3): a 64-bit block p(z) is sent to p(r) with
    r = x_7 = v_64, whose minimal polynomial has degree 128, so the map is a
    ring homomorphism on products of degree <= 126 (Sec. 2.1 allows any
    irreducible g(z) of degree 2w); changeRepr^-1 is the inverse of the
    128x128 matrix [r^0 .. r^127].
  * BasisCvt (Alg. 3): k is the largest power of two K with 2^K <= deg f,
    i.e. for 2^m coefficients K = the largest power of two <= m-1.
  * FFT_LCH output order is natural: entry i is f(\\bar{i} + alpha).
"""
from functools import lru_cache

import numpy as np

# ---------------------------------------------------------------------------
# Tower field (Sec. 3.2): x_1^2 + x_1 + 1 over GF(2), and
# x_{k+1}^2 + x_{k+1} + prod_{i<=k} x_i over the previous field.  An element
# of width 2W = 2^(k+1) is lo + hi * x_{k+1} with lo, hi of width W, and
# prod_{i<=k} x_i = v_{W-1} is the single bit W-1 of the half field.


def tmul_scalar(a, b, width=128):
    """Generic tower multiplication by the defining relations (Karatsuba)."""
    if width == 1:
        return a & b
    if width <= 8:
        return _gf256_table()[a][b] if width == 8 else _tmul_small(a, b, width)
    h = width // 2
    m = (1 << h) - 1
    a0, a1, b0, b1 = a & m, a >> h, b & m, b >> h
    p0 = tmul_scalar(a0, b0, h)
    p1 = tmul_scalar(a1, b1, h)
    p2 = tmul_scalar(a0 ^ a1, b0 ^ b1, h)
    lo = p0 ^ tmul_scalar(p1, 1 << (h - 1), h)  # x^2 = x + v_{h-1}
    hi = p2 ^ p0
    return lo | (hi << h)


@lru_cache(maxsize=None)
def _tmul_small(a, b, width):
    if width == 1:
        return a & b
    h = width // 2
    m = (1 << h) - 1
    a0, a1, b0, b1 = a & m, a >> h, b & m, b >> h
    p0 = _tmul_small(a0, b0, h)
    p1 = _tmul_small(a1, b1, h)
    p2 = _tmul_small(a0 ^ a1, b0 ^ b1, h)
    lo = p0 ^ _tmul_small(p1, 1 << (h - 1), h)
    hi = p2 ^ p0
    return lo | (hi << h)


@lru_cache(maxsize=None)
def _gf256_table():
    return [[_tmul_small(a, b, 8) for b in range(256)] for a in range(256)]


@lru_cache(maxsize=None)
def gf256_np():
    return np.array(_gf256_table(), dtype=np.uint8)


def _tmul_vec_w(a, b, width):
    """Vectorised tower product of uint64 arrays holding width-bit elements."""
    if width == 8:
        t = gf256_np()
        return t[a.astype(np.intp), b.astype(np.intp)].astype(np.uint64)
    h = width // 2
    m = np.uint64((1 << h) - 1)
    sh = np.uint64(h)
    a0, a1, b0, b1 = a & m, a >> sh, b & m, b >> sh
    p0 = _tmul_vec_w(a0, b0, h)
    p1 = _tmul_vec_w(a1, b1, h)
    p2 = _tmul_vec_w(a0 ^ a1, b0 ^ b1, h)
    P = np.full_like(p1, np.uint64(1 << (h - 1)))
    lo = p0 ^ _tmul_vec_w(p1, P, h)
    hi = p2 ^ p0
    return lo | (hi << sh)


def tmul_vec(alo, ahi, blo, bhi):
    """Vectorised product in \\tilde F_{2^128}; elements as (lo, hi) uint64."""
    alo, ahi, blo, bhi = (np.asarray(v, dtype=np.uint64) for v in (alo, ahi, blo, bhi))
    p0 = _tmul_vec_w(alo, blo, 64)
    p1 = _tmul_vec_w(ahi, bhi, 64)
    p2 = _tmul_vec_w(alo ^ ahi, blo ^ bhi, 64)
    P = np.full_like(p1, np.uint64(1 << 63))
    lo = p0 ^ _tmul_vec_w(p1, P, 64)
    hi = p2 ^ p0
    return lo, hi


def tmul(a, b):
    """Scalar product in \\tilde F_{2^128} (Python ints)."""
    lo, hi = tmul_vec(np.array([a & (2**64 - 1)], dtype=np.uint64),
                      np.array([a >> 64], dtype=np.uint64),
                      np.array([b & (2**64 - 1)], dtype=np.uint64),
                      np.array([b >> 64], dtype=np.uint64))
    return int(lo[0]) | (int(hi[0]) << 64)


def tsquare(a):
    return tmul(a, a)


def tpow(a, e):
    r = 1
    while e:
        if e & 1:
            r = tmul(r, a)
        a = tmul(a, a)
        e >>= 1
    return r


def tinv(a):
    """Inverse in \\tilde F_{2^128} as a^(2^128 - 2)."""
    if a == 0:
        raise ZeroDivisionError
    return tpow(a, 2**128 - 2)


# ---------------------------------------------------------------------------
# Subspace vanishing polynomials (Def. 2.2, Corollary in Sec. 3.2.1):
# s_0(x) = x, s_{k+1} = s_k^2 + s_k.


def s1(x):
    return tmul(x, x) ^ x


def s_k(k, x):
    for _ in range(k):
        x = s1(x)
    return x


def s1_vec(lo, hi):
    """s_1 on numpy arrays of elements (lo, hi)."""
    sl, sh = tmul_vec(lo, hi, lo, hi)
    return sl ^ lo, sh ^ hi


def S_table(kmax, tmax):
    """S[k][t] = s_k(v_t) (Sec. 4.4): s_k is GF(2)-linear, so
    s_k(alpha) = XOR of S[k][t] over the set bits t of alpha."""
    lo = np.array([(1 << t) & (2**64 - 1) for t in range(tmax)], dtype=np.uint64)
    hi = np.array([(1 << t) >> 64 for t in range(tmax)], dtype=np.uint64)
    out = []
    for k in range(kmax):
        out.append([int(l) | (int(h) << 64) for l, h in zip(lo, hi)])
        lo, hi = s1_vec(lo, hi)
    return out


def s_k_linear(S, k, alpha):
    r = 0
    t = 0
    while alpha:
        if alpha & 1:
            r ^= S[k][t]
        alpha >>= 1
        t += 1
    return r


# s_i as polynomials in GF(2)[x] (Python ints, bit j = coefficient of x^j).


def gf2_polmul(a, b):
    r = 0
    while b:
        if b & 1:
            r ^= a
        a <<= 1
        b >>= 1
    return r


def s_poly(i):
    """s_i(x) in GF(2)[x] by the recursion s_{i+1} = s_i^2 + s_i."""
    s = 0b10  # x
    for _ in range(i):
        s = gf2_polmul(s, s) ^ s
    return s


def X_poly(k):
    """Novelpoly basis polynomial X_k = prod_{bit i of k} s_i (Def. 2.3)."""
    r = 1
    i = 0
    while k:
        if k & 1:
            r = gf2_polmul(r, s_poly(i))
        k >>= 1
        i += 1
    return r


# ---------------------------------------------------------------------------
# BasisCvt (Alg. 2 VarSubs and Alg. 3), on lists of coefficients that are
# Python ints (64-bit words or 128-bit field elements alike: the divisors have
# coefficients 0/1, so only XOR is used).


def _note(trace, E, e, scale):
    if trace is not None and (E * scale, e * scale) not in trace:
        trace.append((E * scale, e * scale))


def var_subs(f, K, trace=None, scale=1):
    """Alg. 2 with y = x^(2^K) + x: returns h with f = sum_i h_i(x) y^i,
    h_i stored at positions [i 2^K, (i+1) 2^K).  len(f) is a power of two.
    `trace` (optional) collects the divisors x^E + x^e in the order used,
    in units of the original coefficients (`scale` per entry of f)."""
    n = len(f)
    f = list(f)
    if n <= (1 << K):
        return f
    # Largest k = 2^j with deg((x^(2^K)+x)^k) = k 2^K <= n - 1: k 2^K = n/2.
    E = n // 2
    e = E >> K
    _note(trace, E, e, scale)
    # Divide by y^k = x^E + x^e: long division from the top coefficient.
    for p in range(n - 1, E - 1, -1):
        f[p - E + e] ^= f[p]  # the quotient coefficient stays at f[p]
    # f = f0 + y^k f1 with f0 = f[:E], f1 = f[E:]
    return var_subs(f[:E], K, trace, scale) + var_subs(f[E:], K, trace, scale)


def basis_cvt(f, trace=None, scale=1):
    """Alg. 3: monomial coefficients -> novelpoly coefficients."""
    n = len(f)
    if n <= 2:
        return list(f)
    m = n.bit_length() - 1
    K = 1
    while 2 * K <= m - 1:
        K *= 2
    h = var_subs(f, K, trace, scale)
    B = 1 << K
    nb = n // B
    # BasisCvt over y: the y-coefficients are the blocks h[i B:(i+1) B]; the
    # recursion acts on each position inside the blocks independently.
    q = [None] * n
    for t in range(B):
        col = basis_cvt([h[i * B + t] for i in range(nb)], trace, scale * B)
        for i in range(nb):
            q[i * B + t] = col[i]
    out = []
    for i in range(nb):
        out += basis_cvt(q[i * B:(i + 1) * B], trace, scale)
    return out


def basis_cvt_bruteforce(f):
    """Triangular solve: deg X_k = k with leading coefficient 1, so the
    novelpoly coefficients are found from the top: g_k = f_k, f -= g_k X_k."""
    n = len(f)
    f = list(f)
    g = [0] * n
    for k in range(n - 1, -1, -1):
        g[k] = f[k]
        if g[k]:
            X = X_poly(k)
            j = 0
            while X:
                if X & 1:
                    f[j] ^= g[k]
                X >>= 1
                j += 1
    return g


def ibasis_cvt(g):
    """Novelpoly -> monomial by the definition f = sum_k g_k X_k(x)."""
    n = len(g)
    f = [0] * n
    for k in range(n):
        if not g[k]:
            continue
        X = X_poly(k)
        j = 0
        while X:
            if X & 1:
                f[j] ^= g[k]
            X >>= 1
            j += 1
    return f


# ---------------------------------------------------------------------------
# FFT_LCH (Alg. 1) and its inverse, recursive as printed.


def fft_lch(g, alpha=0):
    n = len(g)
    if n == 1:
        return [g[0]]
    k = (n - 1).bit_length() - 1
    h = n // 2
    c = s_k(k, alpha)
    p0, p1 = g[:h], g[h:]
    h0 = [p0[i] ^ tmul(c, p1[i]) for i in range(h)]
    h1 = [h0[i] ^ p1[i] for i in range(h)]
    return fft_lch(h0, alpha) + fft_lch(h1, (1 << k) ^ alpha)


def ifft_lch(vals, alpha=0):
    """Inverse of fft_lch: undo each butterfly (p1 = h0 + h1,
    p0 = h0 + s_k(alpha) p1) after interpolating the two halves."""
    n = len(vals)
    if n == 1:
        return [vals[0]]
    k = (n - 1).bit_length() - 1
    h = n // 2
    h0 = ifft_lch(vals[:h], alpha)
    h1 = ifft_lch(vals[h:], (1 << k) ^ alpha)
    c = s_k(k, alpha)
    p1 = [h0[i] ^ h1[i] for i in range(h)]
    p0 = [h0[i] ^ tmul(c, p1[i]) for i in range(h)]
    return p0 + p1


def eval_novelpoly(g, x):
    """f(x) = sum_j g_j X_j(x) with X_j(x) = prod_{bit i of j} s_i(x)."""
    n = len(g)
    sv = [s_k(i, x) for i in range(max(1, n.bit_length()))]
    acc = 0
    for j in range(n):
        if not g[j]:
            continue
        X = 1
        i = 0
        jj = j
        while jj:
            if jj & 1:
                X = tmul(X, sv[i])
            jj >>= 1
            i += 1
        acc ^= tmul(g[j], X)
    return acc


def _split128(vals):
    lo = np.array([v & (2**64 - 1) for v in vals], dtype=np.uint64)
    hi = np.array([v >> 64 for v in vals], dtype=np.uint64)
    return lo, hi


def novel_basis_at(n, x):
    """X_j(x) for j < n (n a power of two), as (lo, hi) uint64 arrays.
    Def. 2.3 written out over the bits of j: the values for j < 2^(i+1) are
    those for j < 2^i followed by the same values times s_i(x)."""
    lo = np.zeros(n, dtype=np.uint64)
    hi = np.zeros(n, dtype=np.uint64)
    lo[0] = np.uint64(1)
    size, i = 1, 0
    while size < n:
        si = s_k(i, x)
        slo = np.full(size, np.uint64(si & (2**64 - 1)))
        shi = np.full(size, np.uint64(si >> 64))
        lo[size:2 * size], hi[size:2 * size] = tmul_vec(lo[:size], hi[:size], slo, shi)
        size *= 2
        i += 1
    return lo, hi


def eval_novelpoly_np(g_lo, g_hi, x):
    """f(x) = sum_j g_j X_j(x) for coefficients given as (lo, hi) uint64
    arrays of power-of-two length: the same sum as eval_novelpoly, with the
    n products taken by one vectorised tower multiplication."""
    n = len(g_lo)
    Xl, Xh = novel_basis_at(n, x)
    pl, ph = tmul_vec(g_lo, g_hi, Xl, Xh)
    return int(np.bitwise_xor.reduce(pl)) | (int(np.bitwise_xor.reduce(ph)) << 64)


# ---------------------------------------------------------------------------
# changeRepr (Sec. 4.3): 64-bit block p(z) -> p(r) with r = x_7 = v_64.

R_ELEMENT = 1 << 64


@lru_cache(maxsize=None)
def r_powers():
    p = [1]
    for _ in range(127):
        p.append(tmul(p[-1], R_ELEMENT))
    return tuple(p)


def chrepr(word):
    pw = r_powers()
    acc = 0
    i = 0
    while word:
        if word & 1:
            acc ^= pw[i]
        word >>= 1
        i += 1
    return acc


@lru_cache(maxsize=None)
def _ichrepr_rows():
    """Row j of the inverse of [r^0 .. r^127] as a 128-bit mask, by
    Gauss-Jordan elimination over GF(2)."""
    pw = r_powers()
    # Matrix M: column i = r^i (bit j of column i = M[j][i]).  Rows as ints.
    rows = []
    for j in range(128):
        r = 0
        for i in range(128):
            if (pw[i] >> j) & 1:
                r |= 1 << i
        rows.append(r)
    aug = [(rows[j], 1 << j) for j in range(128)]
    for col in range(128):
        piv = next(j for j in range(col, 128) if (aug[j][0] >> col) & 1)
        aug[col], aug[piv] = aug[piv], aug[col]
        for j in range(128):
            if j != col and (aug[j][0] >> col) & 1:
                aug[j] = (aug[j][0] ^ aug[col][0], aug[j][1] ^ aug[col][1])
    return tuple(a[1] for a in aug)


def ichrepr(elem):
    """Inverse of the linear bijection q(z) (deg < 128) -> q(r)."""
    inv = _ichrepr_rows()
    out = 0
    for j in range(128):
        if bin(inv[j] & elem).count("1") & 1:
            out |= 1 << j
    return out


# ---------------------------------------------------------------------------
# Split and InterleavedCombine (Sec. 2.1) and the whole of Alg. 5.


def split(a_words, nbits):
    nw = (nbits + 63) // 64
    w = [int(x) for x in a_words[:nw]]
    if nbits % 64 and nw:
        w[-1] &= (1 << (nbits % 64)) - 1
    return w


def interleaved_combine(coeffs, out_words):
    """z -> x, y -> x^64: word j receives lo(c_j) and hi(c_{j-1})."""
    out = [0] * out_words
    for j, c in enumerate(coeffs):
        lo, hi = c & (2**64 - 1), c >> 64
        if j < out_words:
            out[j] ^= lo
        if j + 1 < out_words:
            out[j + 1] ^= hi
    return out


def fft_size(na_words, nb_words):
    """Smallest power of two N >= na + nb - 1 (at least 2)."""
    need = max(2, na_words + nb_words - 1)
    n = 1
    while n < need:
        n *= 2
    return n


def pad_pow2(n):
    p = 1
    while p < n:
        p *= 2
    return p


def binpolymul(a_words, na_bits, b_words, nb_bits):
    """Alg. 5 end to end, one stage after another; returns the product words
    and a dict of the intermediate stages for stage-by-stage checks."""
    if na_bits == 0 or nb_bits == 0:
        return [], {}
    fa = split(a_words, na_bits)
    fb = split(b_words, nb_bits)
    N = fft_size(len(fa), len(fb))
    Pa, Pb = pad_pow2(len(fa)), pad_pow2(len(fb))
    ga = basis_cvt(fa + [0] * (Pa - len(fa)))
    gb = basis_cvt(fb + [0] * (Pb - len(fb)))
    ta = [chrepr(w) for w in ga] + [0] * (N - Pa)
    tb = [chrepr(w) for w in gb] + [0] * (N - Pb)
    Fa = fft_lch(ta, 0)
    Fb = fft_lch(tb, 0)
    Fc = [tmul(x, y) for x, y in zip(Fa, Fb)]
    gc = ifft_lch(Fc, 0)
    fc = ibasis_cvt(gc)
    cc = [ichrepr(x) for x in fc]
    ow = (na_bits + nb_bits - 1 + 63) // 64
    out = interleaved_combine(cc, ow)
    tot = na_bits + nb_bits - 1
    if tot % 64:
        out[-1] &= (1 << (tot % 64)) - 1
    stages = dict(N=N, ga=ga, gb=gb, ta=ta, tb=tb, Fa=Fa, Fb=Fb, Fc=Fc,
                  gc=gc, fc=fc, cc=cc)
    return out, stages
