"""The F~_{2^256} variant of Alg. 5 (w = 128), step by step, slow and plain.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 4.3 and Table 2 describe a second form of the tower-field method: the
operands are cut into 128-bit blocks (w = 128) instead of 64-bit ones, each
block is mapped into the tower field F~_{2^256} = F~_{2^128}[x_8] /
(x_8^2 + x_8 + x_1 x_2 ... x_7), and the additive FFT runs over half as many
points of that field.  The FFT multipliers s_k(alpha) for the indices used
still lie in the small subfield F~_{2^32}; only pointmul multiplies two
general F~_{2^256} elements.

Elements are Python ints: bit i is the coefficient of the tower basis vector
v_i (Def. 3.1), so the low 128 bits are the subfield F~_{2^128} and bit 128 is
x_8 = v_128.

Readings used here (the paper prints no matrices for this variant either):
  * changeRepr sends a 128-bit block p(z) to p(r) with r = x_8 = v_128, whose
    minimal polynomial has degree 256 (x_8 is outside F~_{2^128}), so the map
    is a ring homomorphism on products of degree <= 254; changeRepr^-1 is the
    inverse of the 256 x 256 matrix [r^0 .. r^255].
  * The recombination is the one of Sec. 2.1 with 128-bit limbs: output
    block j receives the low half of c'_j and the high half of c'_{j-1}.

Parity status: pinned (tests/test_oracle_tower256.py: the field axioms and the
defining relation of x_8, the subfield, the homomorphism and inverse of
changeRepr, direct evaluation of the FFT, and whole products against the
bit-by-bit definition of the product).
"""
from functools import lru_cache

from . import stages as S

M128 = (1 << 128) - 1
V127 = 1 << 127            # x_1 x_2 ... x_7 = v_127, bit 127 of F~_{2^128}
R256 = 1 << 128            # x_8 = v_128


def tmul256(a, b):
    """Product in F~_{2^256} from the defining relation x_8^2 = x_8 + v_127
    (Karatsuba over F~_{2^128}, the products there by oracle.stages.tmul)."""
    a0, a1, b0, b1 = a & M128, a >> 128, b & M128, b >> 128
    p0 = S.tmul(a0, b0)
    p1 = S.tmul(a1, b1)
    p2 = S.tmul(a0 ^ a1, b0 ^ b1)
    lo = p0 ^ S.tmul(p1, V127)
    hi = p2 ^ p0
    return lo | (hi << 128)


def tpow256(a, e):
    r = 1
    while e:
        if e & 1:
            r = tmul256(r, a)
        a = tmul256(a, a)
        e >>= 1
    return r


# ---------------------------------------------------------------------------
# FFT_LCH (Alg. 1) over F~_{2^256}: the multipliers s_k(alpha) are computed in
# F~_{2^128} (alpha is an index below 2^32, so s_k(alpha) lies in F~_{2^32}).


def fft256(g, alpha=0):
    n = len(g)
    if n == 1:
        return [g[0]]
    k = (n - 1).bit_length() - 1
    h = n // 2
    c = S.s_k(k, alpha)
    p0, p1 = g[:h], g[h:]
    h0 = [p0[i] ^ tmul256(c, p1[i]) for i in range(h)]
    h1 = [h0[i] ^ p1[i] for i in range(h)]
    return fft256(h0, alpha) + fft256(h1, (1 << k) ^ alpha)


def ifft256(vals, alpha=0):
    n = len(vals)
    if n == 1:
        return [vals[0]]
    k = (n - 1).bit_length() - 1
    h = n // 2
    h0 = ifft256(vals[:h], alpha)
    h1 = ifft256(vals[h:], (1 << k) ^ alpha)
    c = S.s_k(k, alpha)
    p1 = [h0[i] ^ h1[i] for i in range(h)]
    p0 = [h0[i] ^ tmul256(c, p1[i]) for i in range(h)]
    return p0 + p1


def eval_novelpoly256(g, x):
    """f(x) = sum_j g_j X_j(x), X_j(x) = prod_{bit i of j} s_i(x), for a point
    x of F~_{2^128} and coefficients in F~_{2^256}."""
    n = len(g)
    sv = [S.s_k(i, x) for i in range(max(1, n.bit_length()))]
    acc = 0
    for j in range(n):
        if not g[j]:
            continue
        X = 1
        i, jj = 0, j
        while jj:
            if jj & 1:
                X = S.tmul(X, sv[i])
            jj >>= 1
            i += 1
        acc ^= tmul256(X, g[j])
    return acc


# ---------------------------------------------------------------------------
# changeRepr for 128-bit blocks: p(z) -> p(r), r = x_8.


@lru_cache(maxsize=None)
def r_powers256():
    p = [1]
    for _ in range(255):
        p.append(tmul256(p[-1], R256))
    return tuple(p)


def chrepr256(block):
    """A polynomial of degree < 256 (a 128-bit block, or a product of two)
    evaluated at r."""
    pw = r_powers256()
    acc, i = 0, 0
    while block:
        if block & 1:
            acc ^= pw[i]
        block >>= 1
        i += 1
    return acc


@lru_cache(maxsize=None)
def _ichrepr256_rows():
    """Row j of the inverse of [r^0 .. r^255] as a 256-bit mask (Gauss-Jordan
    elimination over GF(2))."""
    pw = r_powers256()
    rows = []
    for j in range(256):
        r = 0
        for i in range(256):
            if (pw[i] >> j) & 1:
                r |= 1 << i
        rows.append(r)
    aug = [(rows[j], 1 << j) for j in range(256)]
    for col in range(256):
        piv = next(j for j in range(col, 256) if (aug[j][0] >> col) & 1)
        aug[col], aug[piv] = aug[piv], aug[col]
        for j in range(256):
            if j != col and (aug[j][0] >> col) & 1:
                aug[j] = (aug[j][0] ^ aug[col][0], aug[j][1] ^ aug[col][1])
    return tuple(a[1] for a in aug)


def ichrepr256(elem):
    inv = _ichrepr256_rows()
    out = 0
    for j in range(256):
        if bin(inv[j] & elem).count("1") & 1:
            out |= 1 << j
    return out


# ---------------------------------------------------------------------------
# Split into 128-bit blocks, recombination, and the whole of Alg. 5 (w = 128).


def split128(a_words, nbits):
    """128-bit blocks of an nbits-bit polynomial (bits past nbits cleared)."""
    w = S.split(a_words, nbits)
    if len(w) % 2:
        w.append(0)
    return [w[2 * i] | (w[2 * i + 1] << 64) for i in range(len(w) // 2)]


def combine256(coeffs, out_words):
    """128-bit block j of the product receives lo(c_j) and hi(c_{j-1})."""
    blocks = [0] * ((out_words + 1) // 2 + 1)
    for j, c in enumerate(coeffs):
        lo, hi = c & M128, c >> 128
        if j < len(blocks):
            blocks[j] ^= lo
        if j + 1 < len(blocks):
            blocks[j + 1] ^= hi
    out = []
    for b in blocks:
        out += [b & (2**64 - 1), b >> 64]
    return out[:out_words]


def binpolymul256(a_words, na_bits, b_words, nb_bits):
    """Alg. 5 with w = 128, one stage after another; returns the product words
    and the intermediate stages."""
    if na_bits == 0 or nb_bits == 0:
        return [], {}
    fa = split128(a_words, na_bits)
    fb = split128(b_words, nb_bits)
    N = S.fft_size(len(fa), len(fb))
    Pa, Pb = S.pad_pow2(len(fa)), S.pad_pow2(len(fb))
    ga = S.basis_cvt(fa + [0] * (Pa - len(fa)))
    gb = S.basis_cvt(fb + [0] * (Pb - len(fb)))
    ta = [chrepr256(x) for x in ga] + [0] * (N - Pa)
    tb = [chrepr256(x) for x in gb] + [0] * (N - Pb)
    Fa = fft256(ta)
    Fb = fft256(tb)
    Fc = [tmul256(x, y) for x, y in zip(Fa, Fb)]
    gc = ifft256(Fc)
    fc = S.ibasis_cvt(gc)
    cc = [ichrepr256(x) for x in fc]
    ow = (na_bits + nb_bits - 1 + 63) // 64
    out = combine256(cc, ow)
    tot = na_bits + nb_bits - 1
    if tot % 64:
        out[-1] &= (1 << (tot % 64)) - 1
    return out, dict(N=N, ga=ga, gb=gb, ta=ta, tb=tb, Fa=Fa, Fb=Fb, Fc=Fc, gc=gc, fc=fc, cc=cc)
