// Internal declarations shared by the host planner and the CUDA kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

namespace gf2x {

// 128-bit tower element: lo = bits 0..63 (the subfield F~_{2^64}),
// hi = bits 64..127 (the coefficient of v_64 = x_7).
struct u128 {
    uint64_t lo, hi;
};

// ---- Host tower-field arithmetic (Sec. 3.2) --------------------------------
uint64_t tower_mul64(uint64_t a, uint64_t b, int width);  // width <= 64
u128 tower_mul128(u128 a, u128 b);

// ---- Size-independent tables, built once per process on the host ---------
struct HostTables {
    // S[k][t] = s_k(v_t) for k, t < 32 (Sec. 4.4); s_k(alpha) is the XOR of
    // S[k][t] over the set bits t of alpha.
    uint32_t S[32][32];
    // changeRepr, 8-bit method-of-four-Russians tables (Sec. 4.3):
    // phi(w) = XOR_p chr_in[p][byte p of w], chr_in[p][v] = phi(v << 8p).
    u128 chr_in[8][256];
    // changeRepr^-1: psi(e) = XOR_p chr_out[p][byte p of e].
    u128 chr_out[16][256];
    // GF(256) = F~_{2^8} logarithms to a generator g; log8[0] = 512.
    uint16_t log8[256];
    // exp8[i] = g^(i mod 255) for i <= 508, 0 for 509 <= i < 1040.
    uint8_t exp8[1040];
    // mul80[x] = x * v_7 in F~_{2^8} (v_7 = 0x80 closes F~_{2^16}).
    uint8_t mul80[256];
    // Full F~_{2^8} product table: mul8[(c << 8) | x] = c * x.
    uint8_t mul8[65536];
    // Warp-shuffle product tables of the basis vectors v_t, t < 32: for a
    // multiplier c, lane l holds T_w[l] = c * (l << 5w) (w < 6) and
    // T_6[l] = c * ((l & 3) << 30); the table of c is the XOR of the tables
    // of v_t over the set bits t of c (linearity in c).
    uint32_t shfl_basis[32][7][32];
    // The same tables for every byte value at each byte position p of the
    // multiplier: shfl_m4r[p][v] = table of (v << 8p), so the table of c is
    // the XOR of four entries (method of four Russians over c's bytes).
    uint32_t shfl_m4r[4][256][7][32];
};
const HostTables &host_tables();

// Warp-shuffle product table of a multiplier c (layout [7][32]).
void shfl_table_of(uint32_t c, uint32_t out[7][32]);

// ---- BasisCvt schedule (Alg. 2 / Alg. 3) -----------------------------------
// One level = division by the binomial x^E + x^e, E = 2^logE, e = 2^loge,
// applied to every segment of 2E consecutive coefficients.
struct Level {
    int8_t logE, loge;
};
// A fixed-capacity list of levels (no heap allocation).
struct LevelList {
    static constexpr int kMax = 128;
    int n = 0;
    Level v[kMax];
    void push(Level l) {
        if (n < kMax) v[n++] = l;
    }
};
// Levels of BasisCvt on 2^m coefficients, in the forward order.
LevelList basis_cvt_levels(int m);

}  // namespace gf2x
