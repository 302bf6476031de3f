/*
 * CPU oracle for products in GF(2)[x].  TEST INFRASTRUCTURE ONLY: nothing in
 * the product path (the CUDA library and its Python binding) may load or call
 * this file; only the tests, __graft_entry__.smoke() and bench.py's CPU
 * baseline do.
 *
 * What it computes is the plain definition of the method's output
 * (Sec. 2.1 and Alg. 5 of the paper: c(x) = a(x) * b(x) in GF(2)[x]), written
 * out without any FFT:
 *
 *   clmul64        the 64x64 -> 128-bit carry-less product, bit by bit (the
 *                  definition; the pin for the two faster forms below).
 *   clmul64_win4   the same product by 4-bit windows of y (a 16-entry table
 *                  of x times every 4-bit polynomial), portable C.
 *   clmul64_pmull  the same product by the aarch64 PMULL instruction, built
 *                  only where the compiler targets aarch64 and used only where
 *                  the CPU reports it; tests cross-check it against clmul64.
 *   mul_schoolbook the word-level schoolbook product built on clmul64.
 *   mul_karatsuba  Karatsuba's three-product recursion over the schoolbook,
 *                  optionally OpenMP-parallel at the top levels.
 *   mul_bits       c_k = XOR_{i+j=k} a_i b_j, one bit at a time (the pin for
 *                  the two above on small inputs).
 *   poly_mod64     a(x) mod r(x) for a degree-64 modulus r, the modular
 *                  fingerprint used where a full product is too slow.
 *
 * Packing (reading of Sec. 2.1, which fixes only the coefficient order): bit i
 * of 64-bit word j is the coefficient of x^(64 j + i) (little-endian words).
 *
 * Built with plain gcc.  The only machine-specific code is the optional PMULL
 * form (compiled with -DGF2O_PMULL on aarch64 only); the products are the same
 * on x86_64 and aarch64 hosts.  Parity status: pinned (brute force, closed
 * forms, invariants; see tests/test_oracle_product.py).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#if defined(GF2O_PMULL) && defined(__aarch64__)
#include <arm_neon.h>
#include <sys/auxv.h>
#ifndef HWCAP_PMULL
#define HWCAP_PMULL (1 << 4)
#endif
#endif

/* 64x64 carry-less multiply, shift-and-add over the bits of y. */
void gf2o_clmul64(uint64_t x, uint64_t y, uint64_t *lo, uint64_t *hi)
{
    uint64_t l = 0, h = 0;
    for (int i = 0; i < 64; i++) {
        if ((y >> i) & 1u) {
            l ^= x << i;
            if (i) h ^= x >> (64 - i);
        }
    }
    *lo = l;
    *hi = h;
}

/* The same product by 4-bit windows of y from the top: acc = acc * x^4 +
 * T[nibble], T[t] = x * t(x) for the 16 polynomials t of degree < 4. */
void gf2o_clmul64_win4(uint64_t x, uint64_t y, uint64_t *lo, uint64_t *hi)
{
    uint64_t tl[16], th[16];
    tl[0] = 0;
    th[0] = 0;
    for (int t = 1; t < 16; t++) {
        uint64_t l = 0, h = 0;
        for (int i = 0; i < 4; i++) {
            if ((t >> i) & 1) {
                l ^= x << i;
                if (i) h ^= x >> (64 - i);
            }
        }
        tl[t] = l;
        th[t] = h;
    }
    uint64_t l = 0, h = 0;
    for (int k = 60; k >= 0; k -= 4) {
        unsigned t = (unsigned)(y >> k) & 15u;
        h = (h << 4) | (l >> 60);
        l <<= 4;
        l ^= tl[t];
        h ^= th[t];
    }
    *lo = l;
    *hi = h;
}

#if defined(GF2O_PMULL) && defined(__aarch64__)
__attribute__((target("+crypto")))
static void clmul64_pmull(uint64_t x, uint64_t y, uint64_t *lo, uint64_t *hi)
{
    poly128_t p = vmull_p64((poly64_t)x, (poly64_t)y);
    uint64x2_t v = vreinterpretq_u64_p128(p);
    *lo = vgetq_lane_u64(v, 0);
    *hi = vgetq_lane_u64(v, 1);
}
#endif

typedef void (*clmul_fn)(uint64_t, uint64_t, uint64_t *, uint64_t *);

/* The fastest form this host has: 1 = PMULL, 0 = 4-bit windows. */
static clmul_fn pick_clmul(int *kind)
{
#if defined(GF2O_PMULL) && defined(__aarch64__)
    if (getauxval(AT_HWCAP) & HWCAP_PMULL) {
        *kind = 1;
        return clmul64_pmull;
    }
#endif
    *kind = 0;
    return gf2o_clmul64_win4;
}

static clmul_fn g_clmul = 0;
static int g_clmul_kind = -1;

static clmul_fn clmul_fast(void)
{
    if (!g_clmul) {
        int k = 0;
        clmul_fn f = pick_clmul(&k);
        g_clmul_kind = k;
        g_clmul = f;
    }
    return g_clmul;
}

/* Which form the schoolbook, Karatsuba and product-word routines use. */
int gf2o_clmul_kind(void)
{
    clmul_fast();
    return g_clmul_kind;
}

/* The product by that form (exported so that tests can check it against the
 * bit-by-bit definition). */
void gf2o_clmul64_fast(uint64_t x, uint64_t y, uint64_t *lo, uint64_t *hi)
{
    clmul_fast()(x, y, lo, hi);
}

#if defined(GF2O_PMULL) && defined(__aarch64__)
/* Schoolbook rows with the PMULL product inline. */
__attribute__((target("+crypto")))
static void schoolbook_pmull(const uint64_t *a, int64_t na, const uint64_t *b,
                             int64_t nb, uint64_t *out)
{
    for (int64_t i = 0; i < na; i++) {
        if (!a[i]) continue;
        const poly64_t x = (poly64_t)a[i];
        for (int64_t j = 0; j < nb; j++) {
            uint64x2_t v = vreinterpretq_u64_p128(vmull_p64(x, (poly64_t)b[j]));
            out[i + j] ^= vgetq_lane_u64(v, 0);
            out[i + j + 1] ^= vgetq_lane_u64(v, 1);
        }
    }
}
#endif

/* Schoolbook rows by 4-bit windows, the table of a[i] built once per row. */
static void schoolbook_win4(const uint64_t *a, int64_t na, const uint64_t *b,
                            int64_t nb, uint64_t *out)
{
    uint64_t tl[16], th[16];
    for (int64_t i = 0; i < na; i++) {
        const uint64_t x = a[i];
        if (!x) continue;
        tl[0] = 0;
        th[0] = 0;
        for (int t = 1; t < 16; t++) {
            uint64_t l = 0, h = 0;
            for (int q = 0; q < 4; q++) {
                if ((t >> q) & 1) {
                    l ^= x << q;
                    if (q) h ^= x >> (64 - q);
                }
            }
            tl[t] = l;
            th[t] = h;
        }
        for (int64_t j = 0; j < nb; j++) {
            const uint64_t y = b[j];
            uint64_t l = 0, h = 0;
            for (int k = 60; k >= 0; k -= 4) {
                unsigned t = (unsigned)(y >> k) & 15u;
                h = (h << 4) | (l >> 60);
                l <<= 4;
                l ^= tl[t];
                h ^= th[t];
            }
            out[i + j] ^= l;
            out[i + j + 1] ^= h;
        }
    }
}

/* out[0 .. na+nb) = a[0..na) * b[0..nb), words; out must not alias a or b.
 * Each term a_i b_j x^(64(i+j)) is one carry-less word product (the fastest
 * form the host has, see gf2o_clmul_kind). */
void gf2o_mul_schoolbook(const uint64_t *a, int64_t na, const uint64_t *b,
                         int64_t nb, uint64_t *out)
{
    memset(out, 0, (size_t)(na + nb) * sizeof(uint64_t));
#if defined(GF2O_PMULL) && defined(__aarch64__)
    if (gf2o_clmul_kind() == 1) {
        schoolbook_pmull(a, na, b, nb, out);
        return;
    }
#endif
    schoolbook_win4(a, na, b, nb, out);
}

#define KARA_BASE 32

/* Karatsuba on equal halves of n words (n a power of two or anything >= 1):
 * out[0..2n) = a[0..n) * b[0..n).  tmp needs 4n words. */
static void kara_rec(const uint64_t *a, const uint64_t *b, int64_t n,
                     uint64_t *out, uint64_t *tmp, int par_depth)
{
    if (n <= KARA_BASE || (n & 1)) {
        gf2o_mul_schoolbook(a, n, b, n, out);
        return;
    }
    int64_t h = n / 2;
    const uint64_t *a0 = a, *a1 = a + h, *b0 = b, *b1 = b + h;
    uint64_t *sa = tmp, *sb = tmp + h, *mid = tmp + 2 * h; /* mid: 2h words */
    for (int64_t i = 0; i < h; i++) {
        sa[i] = a0[i] ^ a1[i];
        sb[i] = b0[i] ^ b1[i];
    }
    uint64_t *lo = out, *hiw = out + 2 * h; /* a0 b0 and a1 b1 */
    if (par_depth > 0) {
        /* Three independent sub-products as OpenMP tasks (the caller runs
         * the top call inside a parallel region); each has its own scratch. */
        uint64_t *t1 = (uint64_t *)malloc((size_t)4 * h * sizeof(uint64_t));
        uint64_t *t2 = (uint64_t *)malloc((size_t)4 * h * sizeof(uint64_t));
        uint64_t *t3 = (uint64_t *)malloc((size_t)4 * h * sizeof(uint64_t));
#ifdef _OPENMP
#pragma omp task
#endif
        kara_rec(a0, b0, h, lo, t1, par_depth - 1);
#ifdef _OPENMP
#pragma omp task
#endif
        kara_rec(a1, b1, h, hiw, t2, par_depth - 1);
#ifdef _OPENMP
#pragma omp task
#endif
        kara_rec(sa, sb, h, mid, t3, par_depth - 1);
#ifdef _OPENMP
#pragma omp taskwait
#endif
        free(t1);
        free(t2);
        free(t3);
    } else {
        uint64_t *rest = tmp + 4 * h; /* caller gives 4n = 8h words */
        kara_rec(a0, b0, h, lo, rest, 0);
        kara_rec(a1, b1, h, hiw, rest, 0);
        kara_rec(sa, sb, h, mid, rest, 0);
    }
    /* a*b = lo + x^(64h) (mid + lo + hi) + x^(128h) hi */
    for (int64_t i = 0; i < 2 * h; i++) mid[i] ^= lo[i] ^ hiw[i];
    for (int64_t i = 0; i < 2 * h; i++) out[h + i] ^= mid[i];
}

/* Karatsuba product of two operands of any word lengths.  The shorter operand
 * is zero-padded to the longer one's length for the recursion; the result is
 * the exact product, na+nb words.  par_depth > 0 runs that many top levels in
 * parallel with OpenMP. */
int gf2o_mul_karatsuba(const uint64_t *a, int64_t na, const uint64_t *b,
                       int64_t nb, uint64_t *out, int par_depth)
{
    if (na == 0 || nb == 0) return 0;
    int64_t n = na > nb ? na : nb;
    int64_t p = 1;
    while (p < n) p <<= 1;
    uint64_t *pa = (uint64_t *)calloc((size_t)p, sizeof(uint64_t));
    uint64_t *pb = (uint64_t *)calloc((size_t)p, sizeof(uint64_t));
    uint64_t *po = (uint64_t *)calloc((size_t)2 * p, sizeof(uint64_t));
    uint64_t *tmp = (uint64_t *)calloc((size_t)8 * p + 64, sizeof(uint64_t));
    if (!pa || !pb || !po || !tmp) {
        free(pa); free(pb); free(po); free(tmp);
        return -2;
    }
    memcpy(pa, a, (size_t)na * sizeof(uint64_t));
    memcpy(pb, b, (size_t)nb * sizeof(uint64_t));
    clmul_fast(); /* pick the form before any thread uses it */
    if (par_depth > 0) {
#ifdef _OPENMP
#pragma omp parallel
#pragma omp single
#endif
        kara_rec(pa, pb, p, po, tmp, par_depth);
    } else {
        kara_rec(pa, pb, p, po, tmp, 0);
    }
    memcpy(out, po, (size_t)(na + nb) * sizeof(uint64_t));
    free(pa); free(pb); free(po); free(tmp);
    return 0;
}

/* Bit-by-bit product: c_k = XOR_{i+j=k} a_i b_j.  out has na+nb words.
 * Quadratic in bits; only for small inputs. */
void gf2o_mul_bits(const uint64_t *a, int64_t na_bits, const uint64_t *b,
                   int64_t nb_bits, uint64_t *out, int64_t out_words)
{
    memset(out, 0, (size_t)out_words * sizeof(uint64_t));
    for (int64_t i = 0; i < na_bits; i++) {
        if (!((a[i >> 6] >> (i & 63)) & 1u)) continue;
        for (int64_t j = 0; j < nb_bits; j++) {
            if ((b[j >> 6] >> (j & 63)) & 1u) {
                int64_t k = i + j;
                out[k >> 6] ^= (uint64_t)1 << (k & 63);
            }
        }
    }
}

/* a(x) mod r(x), r = x^64 + r_low (r_low the 64 low coefficients), Horner over
 * the words from the top: acc = acc * x^64 + a_j (mod r). */
uint64_t gf2o_poly_mod64(const uint64_t *a, int64_t nwords, uint64_t r_low)
{
    uint64_t acc = 0;
    for (int64_t j = nwords - 1; j >= 0; j--) {
        /* acc * x^64 mod r: shift bit by bit, folding x^64 = r_low. */
        uint64_t v = acc;
        for (int i = 0; i < 64; i++) {
            uint64_t top = v >> 63;
            v <<= 1;
            if (top) v ^= r_low;
        }
        acc = v ^ a[j];
    }
    return acc;
}

/* (x * y) mod r for x, y of degree < 64, r = x^64 + r_low. */
uint64_t gf2o_mulmod64(uint64_t x, uint64_t y, uint64_t r_low)
{
    uint64_t lo, hi;
    gf2o_clmul64(x, y, &lo, &hi);
    uint64_t words[2] = {lo, hi};
    return gf2o_poly_mod64(words, 2, r_low);
}

int gf2o_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Word j of the product a*b straight from the definition: the words a_i and
 * b_{j-i} meet at word j through the low half of their carry-less product
 * and a_i, b_{j-1-i} through the high half.  O(min(na, nb)) per word; used
 * to check sampled words of products too long for a full oracle run.
 * Operands must already have their bits past the length cleared. */
uint64_t gf2o_product_word(const uint64_t *a, int64_t na, const uint64_t *b,
                           int64_t nb, int64_t j)
{
    clmul_fn mul = clmul_fast();
    uint64_t acc = 0;
    int64_t i0 = j - (nb - 1);
    if (i0 < 0) i0 = 0;
    for (int64_t i = i0; i <= j && i < na; i++) {
        uint64_t lo, hi;
        mul(a[i], b[j - i], &lo, &hi);
        acc ^= lo;
    }
    i0 = j - 1 - (nb - 1);
    if (i0 < 0) i0 = 0;
    for (int64_t i = i0; i <= j - 1 && i < na; i++) {
        uint64_t lo, hi;
        mul(a[i], b[j - 1 - i], &lo, &hi);
        acc ^= hi;
    }
    return acc;
}
