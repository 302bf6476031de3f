"""The Frobenius partition / truncated additive FFT form (Appendix C), plain.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Instead of cutting the operands into 64-bit blocks (Kronecker segmentation),
Appendix C evaluates the polynomial a(x) in GF(2)[x] itself -- its coefficients
taken as elements of GF(2^128) -- at the n = 2^m points alpha + V_m with
alpha = beta_{m+64}: the map E: GF(2)[x]_{<128 n} -> GF(2^128)^n is a bijection
(Proposition C.1: the 128 Frobenius conjugates of the coset alpha + V_m are
128 different cosets), and it is multiplicative, so a product c = a b of
degree < 128 n is E^-1(E(a) E(b)) with half as many points as the Kronecker
form needs.

E is a truncated additive FFT: BasisCvt of the 128 n one-bit coefficients,
then the FFT at alpha + V_{m+7} keeping only the first 1/128 of its outputs.
In the first seven layers (k = m+6 .. m) only the left branch survives:
  g'[i] = g[i] + s_k(alpha) g[i + 2^k],
which in total is an "encoding" of the 128 bits g[i + j n] (j < 128) of each
output position i into one field element, sum_j g[i + j n] w_j with
w_j = prod over the set bits l of j of s_{m+l}(alpha).  The remaining m layers
are an ordinary LCH FFT at alpha + V_m.

Field, points and multipliers are those of oracle/simple.py (the polynomial
basis of GF(2^128) and its Cantor basis), where s_k(phi_beta(j)) =
phi_beta(j >> k): the encoding multipliers are s_{m+l}(beta_{m+64}) =
beta_{64-l}, independent of m, and the multiplier of layer k < m for block b is
beta_{m+64-k} + phi_beta(2b).

Readings: the paper writes the map for n = 2^m with m < 63 and the
evaluation points beta_{m+64} + V_m; the number of points of a product is the
smallest n = 2^m with 128 n >= deg(c) + 1.  The inverse of the encoding is the
inverse of the 128 x 128 matrix [w_0 .. w_127] over GF(2) (invertible because
E is a bijection; checked here for small m).

Parity status: pinned (tests/test_oracle_frobenius.py: the bijection by rank
for small m, E against direct evaluation at every point, the encoding and its
inverse, whole products against the bit-by-bit definition).
"""
from functools import lru_cache

from . import simple as SM
from . import stages as S


def points_log(na_bits, nb_bits):
    """m with n = 2^m the smallest power of two such that 128 n >= na + nb - 1."""
    need = (na_bits + nb_bits - 1 + 127) // 128
    m = 0
    while (1 << m) < need:
        m += 1
    return m


def alpha_index(m):
    """Cantor coordinates of alpha = beta_{m+64}."""
    return 1 << (m + 64)


@lru_cache(maxsize=None)
def enc_multipliers():
    """w_j = prod over set bits l of j of beta_{64-l}, j < 128."""
    beta = SM.cantor_basis()
    w = []
    for j in range(128):
        x, l, jj = 1, 0, j
        while jj:
            if jj & 1:
                x = SM.gmul(x, beta[64 - l])
            jj >>= 1
            l += 1
        w.append(x)
    return tuple(w)


def encode(bits128):
    """The element sum_j bit_j w_j of a 128-bit column (bit j of the int)."""
    w = enc_multipliers()
    acc, j = 0, 0
    while bits128:
        if bits128 & 1:
            acc ^= w[j]
        bits128 >>= 1
        j += 1
    return acc


@lru_cache(maxsize=None)
def _dec_rows():
    """Row t of the inverse of the matrix with columns w_j (Gauss-Jordan)."""
    w = enc_multipliers()
    rows = []
    for t in range(128):
        r = 0
        for j in range(128):
            if (w[j] >> t) & 1:
                r |= 1 << j
        rows.append(r)
    aug = [(rows[t], 1 << t) for t in range(128)]
    for col in range(128):
        piv = next(t for t in range(col, 128) if (aug[t][0] >> col) & 1)
        aug[col], aug[piv] = aug[piv], aug[col]
        for t in range(128):
            if t != col and (aug[t][0] >> col) & 1:
                aug[t] = (aug[t][0] ^ aug[col][0], aug[t][1] ^ aug[col][1])
    return tuple(a[1] for a in aug)


def decode(elem):
    """The 128-bit column whose encoding is elem."""
    inv = _dec_rows()
    out = 0
    for j in range(128):
        if bin(inv[j] & elem).count("1") & 1:
            out |= 1 << j
    return out


def _bits_of(words, nbits, total):
    w = S.split(words, nbits)
    out = [0] * total
    for i in range(min(nbits, total)):
        out[i] = (w[i >> 6] >> (i & 63)) & 1
    return out


def truncate7(g, m):
    """The seven left-branch layers k = m+6 .. m of FFT(g, alpha) on the
    2^(m+7) novelpoly coefficients g (field elements)."""
    a = alpha_index(m)
    g = list(g)
    for k in range(m + 6, m - 1, -1):
        c = SM.phi_beta(a >> k)  # s_k(alpha)
        h = 1 << k
        g = [g[i] ^ SM.gmul(c, g[i + h]) for i in range(h)]
    return g


def E_map(words, nbits, m):
    """E(a): the values a(beta_{m+64} + phi_beta(i)), i < 2^m, by BasisCvt of
    the bits, the encoding (seven truncated layers) and the FFT of the other
    m layers."""
    n = 1 << m
    bits = _bits_of(words, nbits, 128 * n)
    g = S.basis_cvt(bits)
    g7 = truncate7(g, m)
    return SM.fft_simple(g7, alpha_index(m)), dict(g=g, g7=g7)


def E_inverse(vals, m):
    """The bits (list of 0/1, 128 n of them) of the polynomial with E = vals."""
    n = 1 << m
    g7 = SM.ifft_simple(list(vals), alpha_index(m))
    g = [0] * (128 * n)
    for i in range(n):
        col = decode(g7[i])
        for j in range(128):
            g[i + j * n] = (col >> j) & 1
    return S.ibasis_cvt(g), dict(g7=g7, g=g)


def eval_bits_at(words, nbits, x):
    """a(x) for a in GF(2)[x] (bits) at a field element x, by Horner."""
    w = S.split(words, nbits)
    acc = 0
    for i in range(nbits - 1, -1, -1):
        acc = SM.gmul(acc, x)
        if (w[i >> 6] >> (i & 63)) & 1:
            acc ^= 1
    return acc


def binpolymul_frobenius(a_words, na_bits, b_words, nb_bits):
    """c = a b by E^-1(E(a) E(b)); returns the product words and the stages."""
    if na_bits == 0 or nb_bits == 0:
        return [], {}
    m = points_log(na_bits, nb_bits)
    Ea, sa = E_map(a_words, na_bits, m)
    Eb, sb = E_map(b_words, nb_bits, m)
    Ec = [SM.gmul(x, y) for x, y in zip(Ea, Eb)]
    cbits, sc = E_inverse(Ec, m)
    tot = na_bits + nb_bits - 1
    ow = (tot + 63) // 64
    out = [0] * ow
    for i in range(tot):
        if cbits[i]:
            out[i >> 6] |= 1 << (i & 63)
    return out, dict(m=m, Ea=Ea, Eb=Eb, Ec=Ec, ga=sa["g"], g7a=sa["g7"], gc7=sc["g7"],
                     gc=sc["g"], cbits=cbits)
