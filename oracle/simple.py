"""The simple form of the product (Alg. 4, Sec. 3.1), step by step.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The working field is kept in the polynomial basis of the AES-GCM field,
GF(2^128) = GF(2)[z] / (z^128 + z^7 + z^2 + z + 1) (Sec. 2.3), and the LCH FFT
evaluates at the points phi_beta(i) of a Cantor basis (beta_i) of that field
(beta_0 = 1, beta_i^2 + beta_i = beta_{i-1}).  A 64-bit block p(z) is already
a field element of degree < 64, products of two blocks have degree <= 126 and
never wrap, so no change of representation is needed before the FFT or after
the inverse FFT; every multiplication, in the butterflies and in pointmul, is a
general GF(2^128) product.

Readings used here:
  * The butterfly multiplier of layer k for the block whose points are
    alpha + V_{k+1}, alpha = phi_beta(b 2^(k+1)), is s_k(alpha) =
    phi_beta(2 b): in a Cantor basis s_k(phi_beta(j)) = phi_beta(j >> k) (the
    shift property stated with the Cantor basis in Sec. 2.4), and the Cantor
    coordinates are switched to the polynomial basis by the linear map
    sum_i c_i beta_i (the multipliers' field isomorphism of Alg. 4).
  * The Cantor basis is built upward from beta_0 = 1 by solving
    y^2 + y = beta_{i-1}, a GF(2)-linear system of rank 127 whose two roots
    differ by 1; the root with coefficient 0 at z^0 is taken.  Any choice
    gives a Cantor basis and the same product.
  * BasisCvt and its inverse are those of the tower form: the novelpoly
    basis polynomials X_k = prod s_i have coefficients in GF(2) and are the
    same polynomials for any Cantor basis.

Parity status: pinned (tests/test_oracle_simple.py: the modulus and the field
axioms, the Cantor relations and the shift property against s_k computed by
iteration, direct evaluation of the FFT, whole products against the bit-by-bit
definition).
"""
from functools import lru_cache

from . import stages as S

G_POLY = (1 << 128) | 0x87  # z^128 + z^7 + z^2 + z + 1
M128 = (1 << 128) - 1


def pmod(a, m=G_POLY):
    """Remainder of a GF(2)[z] polynomial (Python int) modulo m."""
    dm = m.bit_length() - 1
    while a.bit_length() - 1 >= dm:
        a ^= m << (a.bit_length() - 1 - dm)
    return a


def gmul(a, b):
    """Product in GF(2)[z]/(g): the carry-less product, then the remainder."""
    return pmod(S.gf2_polmul(a, b))


def gpow(a, e):
    r = 1
    while e:
        if e & 1:
            r = gmul(r, a)
        a = gmul(a, a)
        e >>= 1
    return r


def s_k_iter(k, x):
    """s_k(x) by k applications of s_1(x) = x^2 + x, in this field."""
    for _ in range(k):
        x = gmul(x, x) ^ x
    return x


@lru_cache(maxsize=None)
def _trace_free_solver():
    """Rows of the linear map L(y) = y^2 + y (column j = L(z^j)), reduced by
    Gauss-Jordan: pivots and the recorded combinations, for solving
    L(y) = c."""
    cols = [gmul(1 << j, 1 << j) ^ (1 << j) for j in range(128)]
    # system: sum_j y_j cols[j] = c.  Work on rows (bit i of the image).
    rows = []
    for i in range(128):
        r = 0
        for j in range(128):
            if (cols[j] >> i) & 1:
                r |= 1 << j
        rows.append(r)
    return rows


def solve_quadratic(c):
    """A root y of y^2 + y = c with coefficient 0 at z^0 (None if none)."""
    rows = [(r, (c >> i) & 1) for i, r in enumerate(_trace_free_solver())]
    piv_of = {}
    rank = 0
    order = list(range(128))
    for col in range(127, -1, -1):  # eliminate from the top unknown down
        piv = next((i for i in range(rank, 128) if (rows[order[i]][0] >> col) & 1), None)
        if piv is None:
            continue
        order[rank], order[piv] = order[piv], order[rank]
        pr = rows[order[rank]]
        for i in range(128):
            if i != rank and (rows[order[i]][0] >> col) & 1:
                rows[order[i]] = (rows[order[i]][0] ^ pr[0], rows[order[i]][1] ^ pr[1])
        piv_of[col] = order[rank]
        rank += 1
    for i in range(rank, 128):
        if rows[order[i]][1]:
            return None  # inconsistent: c has trace 1
    y = 0
    for col, ri in piv_of.items():
        if rows[ri][1]:
            y |= 1 << col
    return y


@lru_cache(maxsize=None)
def cantor_basis(n=128):
    beta = [1]
    for i in range(1, n):
        y = solve_quadratic(beta[-1])
        if y is None:
            raise ValueError("no Cantor basis element %d" % i)
        beta.append(y)
    return tuple(beta)


def phi_beta(j):
    """The field element represented by the integer j under the Cantor basis."""
    beta = cantor_basis()
    r, i = 0, 0
    while j:
        if j & 1:
            r ^= beta[i]
        j >>= 1
        i += 1
    return r


# ---------------------------------------------------------------------------
# FFT_LCH (Alg. 1) at the points phi_beta(i), alpha given by its Cantor
# coordinates (an integer).


def fft_simple(g, alpha=0):
    n = len(g)
    if n == 1:
        return [g[0]]
    k = (n - 1).bit_length() - 1
    h = n // 2
    c = phi_beta(alpha >> k)  # s_k(phi_beta(alpha))
    p0, p1 = g[:h], g[h:]
    h0 = [p0[i] ^ gmul(c, p1[i]) for i in range(h)]
    h1 = [h0[i] ^ p1[i] for i in range(h)]
    return fft_simple(h0, alpha) + fft_simple(h1, alpha | (1 << k))


def ifft_simple(vals, alpha=0):
    n = len(vals)
    if n == 1:
        return [vals[0]]
    k = (n - 1).bit_length() - 1
    h = n // 2
    h0 = ifft_simple(vals[:h], alpha)
    h1 = ifft_simple(vals[h:], alpha | (1 << k))
    c = phi_beta(alpha >> k)
    p1 = [h0[i] ^ h1[i] for i in range(h)]
    p0 = [h0[i] ^ gmul(c, p1[i]) for i in range(h)]
    return p0 + p1


def eval_novelpoly_simple(g, x):
    """f(x) = sum_j g_j X_j(x), X_j = prod_{bit i of j} s_i, in this field."""
    n = len(g)
    sv = [s_k_iter(i, x) for i in range(max(1, n.bit_length()))]
    acc = 0
    for j in range(n):
        if not g[j]:
            continue
        X, i, jj = 1, 0, j
        while jj:
            if jj & 1:
                X = gmul(X, sv[i])
            jj >>= 1
            i += 1
        acc ^= gmul(g[j], X)
    return acc


def combine_simple(coeffs, out_words):
    """z -> x, y -> x^64: word j gets the low 64 bits of c_j and the high 64
    bits of c_{j-1} (Sec. 2.1)."""
    return S.interleaved_combine(coeffs, out_words)


def binpolymul_simple(a_words, na_bits, b_words, nb_bits):
    """Alg. 4 end to end; returns the product words and the stages."""
    if na_bits == 0 or nb_bits == 0:
        return [], {}
    fa = S.split(a_words, na_bits)
    fb = S.split(b_words, nb_bits)
    N = S.fft_size(len(fa), len(fb))
    Pa, Pb = S.pad_pow2(len(fa)), S.pad_pow2(len(fb))
    ga = S.basis_cvt(fa + [0] * (Pa - len(fa))) + [0] * (N - Pa)
    gb = S.basis_cvt(fb + [0] * (Pb - len(fb))) + [0] * (N - Pb)
    Fa = fft_simple(ga)
    Fb = fft_simple(gb)
    Fc = [gmul(x, y) for x, y in zip(Fa, Fb)]
    gc = ifft_simple(Fc)
    fc = S.ibasis_cvt(gc)
    ow = (na_bits + nb_bits - 1 + 63) // 64
    out = combine_simple(fc, ow)
    tot = na_bits + nb_bits - 1
    if tot % 64:
        out[-1] &= (1 << (tot % 64)) - 1
    return out, dict(N=N, ga=ga, gb=gb, Fa=Fa, Fb=Fb, Fc=Fc, gc=gc, fc=fc)
