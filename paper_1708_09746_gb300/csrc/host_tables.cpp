// Host-side precompute: tower arithmetic, s_k tables, changeRepr tables,
// GF(256) log/exp, and the BasisCvt level schedule.  Runs once per process.
#include <cstring>
#include <mutex>
#include <stdexcept>

#include "gf2x_internal.h"

namespace gf2x {

// Tower multiplication (Sec. 3.2): an element of width 2W is lo + hi*X with
// X^2 = X + v_{W-1}; Karatsuba gives
//   lo' = a0 b0 + a1 (b1 v_{W-1}),  hi' = (a0+a1)(b0+b1) + a0 b0.
uint64_t tower_mul64(uint64_t a, uint64_t b, int width) {
    if (width == 1) return a & b & 1u;
    int h = width / 2;
    uint64_t m = (h == 64) ? ~0ull : ((1ull << h) - 1);
    uint64_t a0 = a & m, a1 = a >> h, b0 = b & m, b1 = b >> h;
    uint64_t b1p = tower_mul64(b1, 1ull << (h - 1), h);
    uint64_t r0 = tower_mul64(a0, b0, h);
    uint64_t r1 = tower_mul64(a1, b1p, h);
    uint64_t r2 = tower_mul64(a0 ^ a1, b0 ^ b1, h);
    return (r0 ^ r1) | ((r2 ^ r0) << h);
}

u128 tower_mul128(u128 a, u128 b) {
    uint64_t b1p = tower_mul64(b.hi, 1ull << 63, 64);
    uint64_t r0 = tower_mul64(a.lo, b.lo, 64);
    uint64_t r1 = tower_mul64(a.hi, b1p, 64);
    uint64_t r2 = tower_mul64(a.lo ^ a.hi, b.lo ^ b.hi, 64);
    return u128{r0 ^ r1, r2 ^ r0};
}

static u128 x128(u128 a, u128 b) { return u128{a.lo ^ b.lo, a.hi ^ b.hi}; }

static void build(HostTables &T) {
    std::memset(&T, 0, sizeof(T));
    // s_k(v_t): s_0 = id, s_{k+1} = s_k^2 + s_k (Corollary of Prop. 3.1).
    for (int t = 0; t < 32; t++) {
        uint64_t x = 1ull << t;
        for (int k = 0; k < 32; k++) {
            T.S[k][t] = (uint32_t)x;
            x = tower_mul64(x, x, 64) ^ x;
        }
    }
    // changeRepr: r = x_7 = v_64.  Powers r^i, i < 128.
    u128 rp[128];
    rp[0] = u128{1, 0};
    const u128 r{0, 1};
    for (int i = 1; i < 128; i++) rp[i] = tower_mul128(rp[i - 1], r);
    for (int p = 0; p < 8; p++)
        for (int v = 0; v < 256; v++) {
            u128 acc{0, 0};
            for (int j = 0; j < 8; j++)
                if ((v >> j) & 1) acc = x128(acc, rp[8 * p + j]);
            T.chr_in[p][v] = acc;
        }
    // Inverse of the matrix with columns r^i: Gauss-Jordan on the system
    // sum_i z_i r^i = e.  Each working row is (tower element, polynomial)
    // kept so that element = sum over polynomial bits of r^i; reduce the
    // element parts to unit vectors v_j.
    u128 elem[128], poly[128];
    for (int i = 0; i < 128; i++) {
        elem[i] = rp[i];
        poly[i] = u128{i < 64 ? (1ull << i) : 0, i >= 64 ? (1ull << (i - 64)) : 0};
    }
    auto bit = [](const u128 &x, int j) -> int {
        return j < 64 ? (int)((x.lo >> j) & 1) : (int)((x.hi >> (j - 64)) & 1);
    };
    for (int j = 0; j < 128; j++) {
        int piv = -1;
        for (int i = j; i < 128; i++)
            if (bit(elem[i], j)) { piv = i; break; }
        if (piv < 0) throw std::runtime_error("changeRepr matrix is singular");
        std::swap(elem[j], elem[piv]);
        std::swap(poly[j], poly[piv]);
        for (int i = 0; i < 128; i++)
            if (i != j && bit(elem[i], j)) {
                elem[i] = x128(elem[i], elem[j]);
                poly[i] = x128(poly[i], poly[j]);
            }
    }
    // Now elem[j] = v_j and psi(v_j) = poly[j].
    for (int p = 0; p < 16; p++)
        for (int v = 0; v < 256; v++) {
            u128 acc{0, 0};
            for (int j = 0; j < 8; j++)
                if ((v >> j) & 1) acc = x128(acc, poly[8 * p + j]);
            T.chr_out[p][v] = acc;
        }
    // GF(256) generator: order 255 = 3 * 5 * 17.
    auto pw8 = [](uint64_t g, int e) {
        uint64_t r = 1;
        for (int i = 0; i < e; i++) r = tower_mul64(r, g, 8);
        return r;
    };
    int gen = -1;
    for (int g = 2; g < 256 && gen < 0; g++)
        if (pw8(g, 255) == 1 && pw8(g, 85) != 1 && pw8(g, 51) != 1 && pw8(g, 15) != 1)
            gen = g;
    if (gen < 0) throw std::runtime_error("no generator of F~_{2^8}");
    uint64_t x = 1;
    for (int i = 0; i < 255; i++) {
        T.exp8[i] = (uint8_t)x;
        T.log8[x] = (uint16_t)i;
        x = tower_mul64(x, (uint64_t)gen, 8);
    }
    for (int i = 255; i <= 508; i++) T.exp8[i] = T.exp8[i - 255];
    T.log8[0] = 512;
    for (int v = 0; v < 256; v++) T.mul80[v] = (uint8_t)tower_mul64(v, 0x80, 8);
    for (int c = 0; c < 256; c++)
        for (int x = 0; x < 256; x++) {
            // through the log tables: c * x = g^(log c + log x)
            T.mul8[(c << 8) | x] = T.exp8[T.log8[c] + T.log8[x]];
        }
    for (int t = 0; t < 32; t++)
        for (int l = 0; l < 32; l++) {
            for (int w = 0; w < 6; w++)
                T.shfl_basis[t][w][l] =
                    (uint32_t)tower_mul64(1ull << t, (uint64_t)l << (5 * w), 32);
            T.shfl_basis[t][6][l] = (uint32_t)tower_mul64(1ull << t, (uint64_t)(l & 3) << 30, 32);
        }
    for (int p = 0; p < 4; p++)
        for (int v = 0; v < 256; v++)
            for (int w = 0; w < 7; w++)
                for (int l = 0; l < 32; l++) {
                    uint32_t acc = 0;
                    for (int j = 0; j < 8; j++)
                        if ((v >> j) & 1) acc ^= T.shfl_basis[8 * p + j][w][l];
                    T.shfl_m4r[p][v][w][l] = acc;
                }
}

void shfl_table_of(uint32_t c, uint32_t out[7][32]) {
    const HostTables &T = host_tables();
    for (int w = 0; w < 7; w++)
        for (int l = 0; l < 32; l++) out[w][l] = 0;
    for (int t = 0; t < 32; t++)
        if ((c >> t) & 1)
            for (int w = 0; w < 7; w++)
                for (int l = 0; l < 32; l++) out[w][l] ^= T.shfl_basis[t][w][l];
}

const HostTables &host_tables() {
    static HostTables T;
    static std::once_flag once;
    std::call_once(once, [] { build(T); });
    return T;
}

// Alg. 3 on 2^m coefficients of `scale_log`-sized blocks: y = s_K with K the
// largest power of two <= m-1; VarSubs divides by y^(2^j) = x^E + x^e from
// the top (E = 2^a, e = 2^(a-K), a = m-1 .. K); then BasisCvt over each block
// and BasisCvt over y (the blocks of 2^K coefficients as coefficients).  The
// last two act on disjoint index bits (below K, and K and above: the same map
// on every block, and the same map on every position inside the blocks), so
// they commute; Alg. 3 takes them the other way round.  Converting the blocks
// first lets their levels share a shared-memory tile with the VarSubs levels
// just above them.
static void levels_rec(int m, int scale_log, LevelList &out) {
    if (m <= 1) return;
    int K = 1;
    while (2 * K <= m - 1) K *= 2;
    for (int a = m - 1; a >= K; a--)
        out.push(Level{(int8_t)(a + scale_log), (int8_t)(a - K + scale_log)});
    levels_rec(K, scale_log, out);
    levels_rec(m - K, scale_log + K, out);
}

LevelList basis_cvt_levels(int m) {
    LevelList v;
    levels_rec(m, 0, v);
    return v;
}

}  // namespace gf2x
