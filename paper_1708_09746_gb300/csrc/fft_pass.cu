// Fused multi-layer passes of FFT_LCH (Alg. 1) and its inverse.
//
// A pass covers the g consecutive layers k_lo .. k_lo+g-1 of the N-point
// transform.  Its CTA owns a tile of 2^g "rows" (index bits k_lo .. k_lo+g-1)
// by 2^c "columns" (index bits 0 .. c-1, consecutive elements, so that the
// tile moves through HBM in runs of at least 512 bytes); the remaining index
// bits name the tile.  The tile is loaded into shared memory once (bulk
// copies completed on an mbarrier), all g layers are applied, and it is
// written back once.  A strided pass has c = 12 - g >= 5 (g <= 7); the bottom
// pass is contiguous (c = 0) over the layers 0 .. 11 of 4096 elements.
//
// Multiplier of a butterfly of layer k = k_lo + r at tile row `row`:
//   s_k(phi(idx with bits <= k cleared))
//     = s_k(phi(hi << (k_lo+g)))  XOR  s_k(phi((row >> (r+1)) << (k+1)))
//     =        cval[r]            XOR       d(k, row >> (r+1))
// by the linearity of s_k (Sec. 4.4).  cval[r] is the same for the whole tile;
// d(k, prefix) is the same for every tile and is precomputed per pass.
//
// How each row's butterflies multiply (gf2x_mul.cuh):
//  * rows whose butterflies can be laid out so that the 32 lanes of a warp
//    share the multiplier (column bits plus lower rows span >= 5 index bits):
//    whole elements in registers, up to three rows per register sub-pass,
//    warp-shuffle tables (the table of cval[r] is built once per tile, the
//    table of d is precomputed; the table of their sum is the XOR of the two;
//    seven shuffles per 32-bit limb in the strided passes, six in the bottom
//    pass with the top two bits on the integer pipe);
//  * rows 3-5 of the bottom pass: one limb-wise sub-pass (a lane holds one
//    32-bit limb of 8 elements, so a warp's lanes share the multiplier of a
//    group of up to 64 elements) with the same shuffle tables, the tables of
//    a group's other blocks as block 0's plus precomputed offsets;
//  * rows 0-2 of a bottom tile of at least 2^8 elements: one register
//    sub-pass per lane group of 8 elements; the multiplier's warp-uniform part
//    through the shuffle tables, its per-lane F~_{2^8} part through a per-lane
//    byte table;
//  * lane-varying rows of smaller tiles: the F~_{2^8} product table in shared
//    memory, one row per sweep.
#include <algorithm>
#include <cstddef>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "fft_pass.h"
#include "gf2x_internal.h"
#include "gf2x_mul.cuh"
#include "kernels.h"
#include "launch.h"
#include "tma.cuh"

namespace gf2x {

// shfl6_table_sum reads words 194, 195 of each seven-word shuffle table as one
// 8-byte load: the rows 0-2 tables must start on 8-byte boundaries too
static_assert(offsetof(DevTables, low_shfl) % 16 == 0, "low_shfl alignment");

namespace {
std::atomic<uint32_t> g_wait_spins{kWaitSpins};
}

void set_wait_spins(int64_t spins) {
    g_wait_spins.store(spins < 0 ? kWaitSpins : (uint32_t)std::min<int64_t>(spins, 0xffffffffll));
}
uint32_t wait_spins() { return g_wait_spins.load(); }

// Which product the register sub-passes use (shfl6_mul128 or shfl_mul128).
#ifndef GF2X_SHFL6_STRIDED
#define GF2X_SHFL6_STRIDED 0
#endif
#ifndef GF2X_SHFL6_BOTTOM
#define GF2X_SHFL6_BOTTOM 1
#endif
constexpr bool kShfl6Strided = GF2X_SHFL6_STRIDED != 0;
constexpr bool kShfl6Bottom = GF2X_SHFL6_BOTTOM != 0;

// Rows (from the lowest) of a strided three-row sub-pass whose block tables are
// block 0's plus kept offset tables; 1: also the lower row of a paired two-row
// sub-pass.
#ifndef GF2X_STRIDED_OFFSET_ROWS
#define GF2X_STRIDED_OFFSET_ROWS 2
#endif
#ifndef GF2X_PAIR_OFFSET
#define GF2X_PAIR_OFFSET 0
#endif
constexpr int kStridedOffsetRows = GF2X_STRIDED_OFFSET_ROWS;
constexpr bool kPairOffset = GF2X_PAIR_OFFSET != 0;

// ---------------------------------------------------------------------------
// Register sub-pass: G layers (tile rows r_lo .. r_lo+G-1) on columns of 2^G
// elements held by one thread.  Requires c + r_lo >= 5 so that a warp's lanes
// differ only in bits below the sub-pass (warp-uniform multipliers).  SIX: the
// six-shuffle product (two bits on the integer pipe), else seven shuffles.
template <int G, bool INV, bool SIX>
__device__ __forceinline__ void reg_subpass(uint4 *s, int c, int g, int r_lo, int uf,
                                            const uint32_t *ctab, const uint32_t *__restrict__ d_shfl) {
    const int r_hi = r_lo + G - 1;
    const uint32_t items = 1u << (g + c - G);
    const int lane = threadIdx.x & 31;
    const uint32_t cmask = (1u << c) - 1, lomask = (1u << r_lo) - 1;
    // strided three-row sub-passes: the tables of d(k, 1), d(k, 2) of the lowest
    // row, read once per call
    ShflTab R1, R2, R3, T0s;
    if (!SIX && G == 3 && kStridedOffsetRows > 0) {
        const uint32_t off0 = (1u << (g - uf)) - (1u << (g - r_lo));
        const uint32_t off1 = (1u << (g - uf)) - (1u << (g - r_lo - 1));
#pragma unroll
        for (int w = 0; w < 7; w++) {
            R1.t[w] = __ldg(d_shfl + (size_t)(off0 + 1) * 224 + 32 * w + lane);
            R2.t[w] = __ldg(d_shfl + (size_t)(off0 + 2) * 224 + 32 * w + lane);
            R3.t[w] = __ldg(d_shfl + (size_t)(off1 + 1) * 224 + 32 * w + lane);
        }
    }
    for (uint32_t q = threadIdx.x; q < items; q += blockDim.x) {
        const uint32_t col = q & cmask, rest = q >> c;
        const uint32_t lo_rows = rest & lomask, hi_rows = rest >> r_lo;
        const uint32_t base_row = (hi_rows << (r_hi + 1)) | lo_rows;
        uint4 e[1 << G];
#pragma unroll
        for (int m = 0; m < (1 << G); m++) e[m] = s[((base_row | ((uint32_t)m << r_lo)) << c) | col];
#pragma unroll
        for (int step = 0; step < G; step++) {
            const int rr = INV ? step : (G - 1 - step);
            const int r = r_lo + rr;
            // offset (in multipliers) of layer r's precomputed tables
            const uint32_t off = (1u << (g - uf)) - (1u << (g - r));
#pragma unroll
            for (int B = 0; B < (1 << (G - 1 - rr)); B++) {
                const uint32_t prefix = (hi_rows << (r_hi - r)) | (uint32_t)B;
                const uint32_t *ct = ctab + (r - uf) * 224;
                const uint32_t *dt = d_shfl + (size_t)(off + prefix) * 224;
                if constexpr (SIX) {
                    const ShflTab6 T = shfl6_table_sum(ct, dt, lane);
#pragma unroll
                    for (int j = 0; j < (1 << rr); j++) {
                        uint4 &u = e[B * (2 << rr) + j];
                        uint4 &v = e[B * (2 << rr) + j + (1 << rr)];
                        if (!INV) {
                            u = xor4(u, shfl6_mul128(v, T));
                            v = xor4(v, u);
                        } else {
                            v = xor4(v, u);
                            u = xor4(u, shfl6_mul128(v, T));
                        }
                    }
                } else {
                    ShflTab T;
                    if (G == 3 && rr < kStridedOffsetRows) {
                        // block B's table = block 0's + the kept table of d(k, B)
                        if (B == 0) {
#pragma unroll
                            for (int w = 0; w < 7; w++) T0s.t[w] = ct[32 * w + lane] ^ __ldg(dt + 32 * w + lane);
                        }
                        if (rr == 0) {
#pragma unroll
                            for (int w = 0; w < 7; w++)
                                T.t[w] = T0s.t[w] ^ ((B & 1) ? R1.t[w] : 0u) ^ ((B & 2) ? R2.t[w] : 0u);
                        } else {
#pragma unroll
                            for (int w = 0; w < 7; w++) T.t[w] = T0s.t[w] ^ ((B & 1) ? R3.t[w] : 0u);
                        }
                    } else {
#pragma unroll
                        for (int w = 0; w < 7; w++) T.t[w] = ct[32 * w + lane] ^ __ldg(dt + 32 * w + lane);
                    }
#pragma unroll
                    for (int j = 0; j < (1 << rr); j++) {
                        uint4 &u = e[B * (2 << rr) + j];
                        uint4 &v = e[B * (2 << rr) + j + (1 << rr)];
                        if (!INV) {
                            u = xor4(u, shfl_mul128(v, T));
                            v = xor4(v, u);
                        } else {
                            v = xor4(v, u);
                            u = xor4(u, shfl_mul128(v, T));
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int m = 0; m < (1 << G); m++) s[((base_row | ((uint32_t)m << r_lo)) << c) | col] = e[m];
    }
}

// Two-row sub-pass of a strided tile (c >= 6) with two columns per thread, col
// and col + 32: the columns share every multiplier, so each table read serves
// both (eight elements in registers, as in a three-row sub-pass).  Pair p
// takes the items q = 64 (p >> 5) + (p & 31) and q + 32; the 32 lanes of a warp
// hold consecutive columns of one row group.
#ifndef GF2X_STRIDED_PAIR
#define GF2X_STRIDED_PAIR 1
#endif
template <bool INV>
__device__ __forceinline__ void reg_subpass2_pair(uint4 *s, int c, int g, int r_lo, int uf,
                                                  const uint32_t *ctab,
                                                  const uint32_t *__restrict__ d_shfl) {
    const int r_hi = r_lo + 1;
    const uint32_t pairs = 1u << (g + c - 3);
    const int lane = threadIdx.x & 31;
    const uint32_t cmask = (1u << c) - 1, lomask = (1u << r_lo) - 1;
    // the lower row's block 1 table = block 0's + the kept table of d(k, 1)
    ShflTab R1, T0;
    if (kPairOffset) {
        const uint32_t off0 = (1u << (g - uf)) - (1u << (g - r_lo));
#pragma unroll
        for (int w = 0; w < 7; w++) R1.t[w] = __ldg(d_shfl + (size_t)(off0 + 1) * 224 + 32 * w + lane);
    }
    for (uint32_t p = threadIdx.x; p < pairs; p += blockDim.x) {
        const uint32_t q = ((p >> 5) << 6) | (p & 31);
        const uint32_t col = q & cmask, rest = q >> c;
        const uint32_t lo_rows = rest & lomask, hi_rows = rest >> r_lo;
        const uint32_t base_row = (hi_rows << (r_hi + 1)) | lo_rows;
        uint4 e[2][4];
#pragma unroll
        for (int h = 0; h < 2; h++)
#pragma unroll
            for (int m = 0; m < 4; m++)
                e[h][m] = s[((base_row | ((uint32_t)m << r_lo)) << c) | (col | (uint32_t)(h << 5))];
#pragma unroll
        for (int step = 0; step < 2; step++) {
            const int rr = INV ? step : 1 - step;
            const int r = r_lo + rr;
            const uint32_t off = (1u << (g - uf)) - (1u << (g - r));
#pragma unroll
            for (int B = 0; B < (2 >> rr); B++) {
                const uint32_t prefix = (hi_rows << (r_hi - r)) | (uint32_t)B;
                const uint32_t *ct = ctab + (r - uf) * 224;
                const uint32_t *dt = d_shfl + (size_t)(off + prefix) * 224;
                ShflTab T;
                if (kPairOffset && rr == 0 && B == 1) {
#pragma unroll
                    for (int w = 0; w < 7; w++) T.t[w] = T0.t[w] ^ R1.t[w];
                } else {
#pragma unroll
                    for (int w = 0; w < 7; w++) T.t[w] = ct[32 * w + lane] ^ __ldg(dt + 32 * w + lane);
                    if (kPairOffset && rr == 0) T0 = T;
                }
#pragma unroll
                for (int h = 0; h < 2; h++)
#pragma unroll
                    for (int j = 0; j < (1 << rr); j++) {
                        uint4 &u = e[h][B * (2 << rr) + j];
                        uint4 &v = e[h][B * (2 << rr) + j + (1 << rr)];
                        if (!INV) {
                            u = xor4(u, shfl_mul128(v, T));
                            v = xor4(v, u);
                        } else {
                            v = xor4(v, u);
                            u = xor4(u, shfl_mul128(v, T));
                        }
                    }
            }
        }
#pragma unroll
        for (int h = 0; h < 2; h++)
#pragma unroll
            for (int m = 0; m < 4; m++)
                s[((base_row | ((uint32_t)m << r_lo)) << c) | (col | (uint32_t)(h << 5))] = e[h][m];
    }
}

template <bool INV, bool SIX>
__device__ __forceinline__ void run_subpass(int G, uint4 *s, int c, int g, int r_lo, int uf,
                                            const uint32_t *ctab, const uint32_t *d_shfl) {
    switch (G) {
        case 1: reg_subpass<1, INV, SIX>(s, c, g, r_lo, uf, ctab, d_shfl); break;
        case 2:
            if (GF2X_STRIDED_PAIR && !SIX && c >= 6)
                reg_subpass2_pair<INV>(s, c, g, r_lo, uf, ctab, d_shfl);
            else
                reg_subpass<2, INV, SIX>(s, c, g, r_lo, uf, ctab, d_shfl);
            break;
        case 3: reg_subpass<3, INV, SIX>(s, c, g, r_lo, uf, ctab, d_shfl); break;
        default: reg_subpass<3, INV, SIX>(s, c, g, r_lo, uf, ctab, d_shfl); break;
    }
}

// Layers 3 .. 3+NR-1 of a contiguous tile (c = 0), NR = 1 .. 3, with
// warp-uniform multipliers: a thread holds ONE 32-bit limb of the elements
// that differ in index bits 3 .. 2+NR of a group of 2^(3+NR) elements, and the
// 32 lanes of a warp are the 4 limbs x 8 elements (bits 0..2) of that group.
// All lanes then share the group's multipliers, so the shuffle tables apply
// here although a butterfly block of these layers is smaller than a warp of
// whole elements (Prop. 3.2: the limbs are multiplied independently).  Lane l
// reads word (element << 2) + (l & 3) of element base + (l >> 2): one
// conflict-free 128-byte row per value.
//
// Row r of a group has 2^(NR-1-(r-3)) butterfly blocks B, and by linearity in
// the index bits the multiplier of block B is that of block 0 plus d(k, B),
// the same in every group and tile.  The tables of d(k, 1) and d(k, 2) are
// read once per call and kept in registers, so that a group reads one table
// per row instead of one per block.
template <int NR, bool INV>
__device__ __forceinline__ void limb_subpass(uint4 *s, int g, int uf, const uint32_t *ctab,
                                             const uint32_t *__restrict__ d_shfl) {
    uint32_t *wds = reinterpret_cast<uint32_t *>(s);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t groups = 1u << (g - 3 - NR);
    ShflTab6 R[NR][2];  // [row - 3][bit]: the table of d(k, 1 << bit)
#pragma unroll
    for (int rr = 0; rr < NR; rr++) {
        const uint32_t off = (1u << (g - uf)) - (1u << (g - 3 - rr));
#pragma unroll
        for (int bit = 0; bit < 2; bit++)
            if ((2 << bit) <= (1 << (NR - 1 - rr)))
                R[rr][bit] = shfl6_table(d_shfl + (size_t)(off + (1u << bit)) * 224, lane);
    }
    for (uint32_t grp = warp; grp < groups; grp += nwarps) {
        uint32_t v[1 << NR];
#pragma unroll
        for (int m = 0; m < (1 << NR); m++)
            v[m] = wds[((((grp << NR) | (uint32_t)m) << 3) << 2) + lane];
#pragma unroll
        for (int step = 0; step < NR; step++) {
            const int rr = INV ? step : (NR - 1 - step);
            const int r = 3 + rr;
            const uint32_t off = (1u << (g - uf)) - (1u << (g - r));
            const ShflTab6 T0 = shfl6_table_sum(
                ctab + (r - uf) * 224, d_shfl + (size_t)(off + (grp << (NR - 1 - rr))) * 224, lane);
#pragma unroll
            for (int B = 0; B < (1 << (NR - 1 - rr)); B++) {
                ShflTab6 T = T0;
                if (B & 1) shfl6_xor(T, R[rr][0]);
                if (B & 2) shfl6_xor(T, R[rr][1]);
#pragma unroll
                for (int j = 0; j < (1 << rr); j++) {
                    uint32_t &u = v[B * (2 << rr) + j];
                    uint32_t &x = v[B * (2 << rr) + j + (1 << rr)];
                    if (!INV) {
                        u ^= shfl6_mul32(x, T);
                        x ^= u;
                    } else {
                        x ^= u;
                        u ^= shfl6_mul32(x, T);
                    }
                }
            }
        }
#pragma unroll
        for (int m = 0; m < (1 << NR); m++)
            wds[((((grp << NR) | (uint32_t)m) << 3) << 2) + lane] = v[m];
    }
}

// Rows 0, 1, 2 of a contiguous tile (c = 0) of at least 2^8 elements.  The
// multiplier of row r at index i is s_r(phi(i with bits 0..r cleared)), linear
// in the index bits (Sec. 4.4), so it splits into
//   cval[r]            the bits above the tile (the same for the whole tile),
//   D(r, blk, h)       bits 8.. of the tile index (blk, the same for a warp) and
//                      bits r+1..2 (h, the butterfly block inside a group of 8),
//   delta_r(l)         bits 3..7 = the lane l (the same for every tile and warp).
// Lane l holds the 8 elements of group (blk << 5) | l in registers, so the three
// rows take one shared-memory round trip.  The product by cval[r] ^ D uses the
// warp's shuffle table of that sum (the tile's table XOR the precomputed one);
// the product by delta_r(l), an element of F~_{2^8}, is 16 byte lookups in the
// lane's own table (byte r + 1 of word x * 32 + l).  The lane reads its group in
// the order m ^ (l & 7), so the eight lanes of each 128-byte request hit eight
// different 16-byte bank groups, and three conditional register swaps put the
// elements back in index order (and out of it again before the writes).
__device__ __forceinline__ void swap8(uint4 (&e)[8], uint32_t sig) {
#pragma unroll
    for (int bit = 0; bit < 3; bit++) {
        const bool p = (sig >> bit) & 1u;
#pragma unroll
        for (int m = 0; m < 8; m++) {
            if (m & (1 << bit)) continue;
            const int n = m | (1 << bit);
            const uint4 x = e[m], y = e[n];
            e[m] = p ? y : x;
            e[n] = p ? x : y;
        }
    }
}

template <int R>
__device__ __forceinline__ uint32_t lane_mul32(const uint8_t *lt, uint32_t x) {
    const uint32_t b0 = lt[((x & 255u) << 7) + R + 1];
    const uint32_t b1 = lt[(((x >> 8) & 255u) << 7) + R + 1];
    const uint32_t b2 = lt[(((x >> 16) & 255u) << 7) + R + 1];
    const uint32_t b3 = lt[((x >> 24) << 7) + R + 1];
    return b0 | (b1 << 8) | (b2 << 16) | (b3 << 24);
}

template <int R>
__device__ __forceinline__ uint4 low_mul128(uint4 v, const ShflTab6 &T, const uint8_t *lt) {
    const uint4 p = shfl6_mul128(v, T);
    return make_uint4(p.x ^ lane_mul32<R>(lt, v.x), p.y ^ lane_mul32<R>(lt, v.y),
                      p.z ^ lane_mul32<R>(lt, v.z), p.w ^ lane_mul32<R>(lt, v.w));
}

template <int R, bool INV>
__device__ __forceinline__ void low_row(uint4 (&e)[8], uint32_t blk, const uint32_t *ctab,
                                        const uint32_t *__restrict__ low_shfl, const uint8_t *lt) {
    const int lane = threadIdx.x & 31;
    // D(R, blk, h) = D(R, blk, 0) + D(R, 0, h): one table per block of 8 and
    // the tables of D(R, 0, 1) and D(R, 0, 2)
    constexpr int lo = kLowOff[R];
    const ShflTab6 T0 =
        shfl6_table_sum(ctab + R * 224, low_shfl + (size_t)(lo + blk * (4 >> R)) * 224, lane);
    ShflTab6 H[2];
#pragma unroll
    for (int bit = 0; bit < 2; bit++)
        if ((2 << bit) <= (4 >> R)) H[bit] = shfl6_table(low_shfl + (size_t)(lo + (1 << bit)) * 224, lane);
#pragma unroll
    for (int h = 0; h < (4 >> R); h++) {
        ShflTab6 T = T0;
        if (h & 1) shfl6_xor(T, H[0]);
        if (h & 2) shfl6_xor(T, H[1]);
#pragma unroll
        for (int j = 0; j < (1 << R); j++) {
            uint4 &u = e[h * (2 << R) + j];
            uint4 &v = e[h * (2 << R) + j + (1 << R)];
            if (!INV) {
                u = xor4(u, low_mul128<R>(v, T, lt));
                v = xor4(v, u);
            } else {
                v = xor4(v, u);
                u = xor4(u, low_mul128<R>(v, T, lt));
            }
        }
    }
}

template <bool INV>
__device__ __forceinline__ void low3_subpass(uint4 *s, int g, const uint32_t *ctab,
                                             const uint32_t *__restrict__ low_shfl,
                                             const uint32_t *lane_tab) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t sig = lane & 7;
    const uint8_t *lt = reinterpret_cast<const uint8_t *>(lane_tab + lane);
    const uint32_t nblk = 1u << (g - 8);
    for (uint32_t blk = warp; blk < nblk; blk += nwarps) {
        uint4 *grp = s + ((((blk << 5) | (uint32_t)lane)) << 3);
        uint4 e[8];
#pragma unroll
        for (int m = 0; m < 8; m++) e[m] = grp[m ^ sig];
        swap8(e, sig);
        if (!INV) {
            low_row<2, false>(e, blk, ctab, low_shfl, lt);
            low_row<1, false>(e, blk, ctab, low_shfl, lt);
            low_row<0, false>(e, blk, ctab, low_shfl, lt);
        } else {
            low_row<0, true>(e, blk, ctab, low_shfl, lt);
            low_row<1, true>(e, blk, ctab, low_shfl, lt);
            low_row<2, true>(e, blk, ctab, low_shfl, lt);
        }
        swap8(e, sig);
#pragma unroll
        for (int m = 0; m < 8; m++) grp[m ^ sig] = e[m];
    }
}

// One lane-varying layer r of a contiguous tile (c = 0) swept in shared memory.
template <bool INV>
__device__ __forceinline__ void smem_layer(uint4 *s, int g, int r, const MtRef &mt, uint32_t cv,
                                           const uint32_t *__restrict__ d_val) {
    const uint32_t half = 1u << (g - 1);
    const uint32_t voff = (1u << g) - (1u << (g - r));
    for (uint32_t w = threadIdx.x; w < half; w += blockDim.x) {
        const uint32_t prefix = w >> r, j = w & ((1u << r) - 1);
        const uint32_t iu = (prefix << (r + 1)) | j, iv = iu | (1u << r);
        const MtConst mc = mt_prep(mt, cv ^ __ldg(d_val + voff + prefix));
        uint4 u = s[iu], v = s[iv];
        if (!INV) {
            u = xor4(u, mt_cmul128(mt, v, mc));
            v = xor4(v, u);
        } else {
            v = xor4(v, u);
            u = xor4(u, mt_cmul128(mt, v, mc));
        }
        s[iu] = u;
        s[iv] = v;
    }
}

__device__ __forceinline__ uint4 chrepr_ldg(const DevTables *__restrict__ T, uint64_t w) {
    uint4 acc = make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int p = 0; p < 8; p++) acc = xor4(acc, __ldg(&T->chr_in[p][(w >> (8 * p)) & 255]));
    return acc;
}

// Multiplier s_k(phi(hi << (k_lo + g))) shared by a tile of layer k = k_lo + r
// (hi = the tile index bits above the tile).
__device__ __forceinline__ uint32_t tile_cval(const FftPassArgs &a, uint64_t tt, int r) {
    const uint64_t hi = tt >> (a.k_lo - a.c);
    return s_k_of(&a.T->S[a.k_lo + r][0], (uint32_t)(hi << (a.k_lo + a.g)));
}

// Starts the asynchronous copies of the byte-sliced shuffle tables of the
// multipliers cv[r], r = tb .. g-1 (Sec. 4.4: the table of c is the XOR of
// the tables of its four bytes) into stab[(r - tb) * 4 + byte][224].
__device__ __forceinline__ void prefetch_tables(const FftPassArgs &a, int tb, const uint32_t *cv,
                                                uint32_t *stab) {
    const int gt = a.g - tb;
    for (int q = threadIdx.x; q < gt * 4 * 56; q += blockDim.x) {
        const int piece = q / 56, chunk = q - piece * 56;
        const int r = tb + (piece >> 2), p = piece & 3;
        const uint32_t byte = (cv[r] >> (8 * p)) & 255;
        cp_async16(stab + piece * 224 + chunk * 4, &a.T->shfl_m4r[p][byte][0][0] + chunk * 4);
    }
    cp_async_commit();
}

// Persistent kernel: each CTA walks the tiles blockIdx.x, +gridDim.x, ...
// Two instantiations: STRIDED for the passes with c > 0 (register sub-passes
// only), the other for the contiguous bottom passes (limb-wise rows, rows 0-2,
// changeRepr on the way in, pointmul).
// with one or two tile buffers.  While one tile is computed, the next one is
// being loaded by bulk copies (TMA) and the previous one stored; warp 0 issues
// all copies.  The first strided pass of a transform loads the changeRepr'd
// blocks (P elements, read periodically); a bottom pass that is also the
// first reads the 64-bit blocks and applies changeRepr on the way in.  The
// shuffle tables of the next tile's multipliers are copied in
// asynchronously while the current tile is computed.
template <bool STRIDED>
__global__ void __launch_bounds__(512, 1) k_fft_pass(FftPassArgs a) {
    // the register sub-passes' product: six shuffles in the bottom passes,
    // seven in the strided ones (measured: the strided passes wait on their
    // table loads, not on the shuffle pipe, and lose with the longer chain)
    constexpr bool SIX = STRIDED ? kShfl6Strided : kShfl6Bottom;
    pdl_release();
    extern __shared__ __align__(128) unsigned char smem[];
    const int g = a.g, c = a.c, uf = a.uf;
    // shuffle tables of the tile's multipliers for rows tb .. g-1 (all rows
    // when rows 0-2 run in registers with per-lane tables)
    const int tb = a.low3 ? 0 : uf, gt = g - tb;
    // rows [uf, ul) run limb-wise (only the contiguous bottom pass: rows 3-5,
    // or 3-4 in a tile of 2^5 elements)
    const int ul = (c == 0 && uf == 3 && g >= 5) ? min(g, 6) : uf;
    const uint32_t tile = 1u << (g + c);
    const int NB = a.nbuf;
    uint4 *const buf0 = reinterpret_cast<uint4 *>(smem);  // buffer b at buf0 + b * tile
    uint32_t *ctab = reinterpret_cast<uint32_t *>(smem + 16 * (size_t)tile * NB);  // [gt][7][32]
    uint32_t *stab = ctab + gt * 224;                                         // [gt][4][224]
    uint32_t *cval = stab + gt * 4 * 224;                                     // [32]
    uint32_t *cnext = cval + 32;                                              // [32]
    uint64_t *bar = reinterpret_cast<uint64_t *>(cnext + 32);                 // [4]
    unsigned char *tail = reinterpret_cast<unsigned char *>(bar + 4);
    const bool from_g = a.g64 != nullptr;
    const bool pipe = !from_g;                // tiles by bulk copies
    uint8_t *mt = tail;                       // 64 KiB if needed
    // per-lane tables (v_7 and the rows 0-2 products) after the product table
    uint32_t *lane_tab = reinterpret_cast<uint32_t *>(tail + (a.needs_mt ? 65536 : 0));
    const uint32_t *ctab_u = ctab + (uf - tb) * 224;  // row uf's table

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const TileGeom G{c, a.k_lo, g, 4};
    // tiles of every product: t = (product << tiles_log) | tile
    const int tiles_log = a.M - g - c;
    const uint64_t ntiles = (uint64_t)a.count << tiles_log;
    const uint64_t tmask = (1ull << tiles_log) - 1;
    const uint32_t cmask = (1u << c) - 1;
    // Source of tile t.  Normally the tile itself; the first pass of a
    // transform reads the changeRepr'd blocks (a.Fsrc, P elements) at the
    // index taken modulo P: the pass's layers lie below log2 P, so only the
    // tile's high bits are reduced (the fan-out of the layers above).
    const int mid_bits = a.k_lo - c;
    const uint4 *src_base = a.Fsrc ? a.Fsrc : a.F;
    auto src_of = [&](uint64_t t) { return src_base + (t >> tiles_log) * a.strideF; };
    auto src_tile = [&](uint64_t tt) -> uint64_t {
        if (!a.Fsrc) return tt;
        return (((tt >> mid_bits) & (a.pmask >> (a.k_lo + g))) << mid_bits) |
               (tt & ((1ull << mid_bits) - 1));
    };

    if (threadIdx.x == 0) {
        for (int i = 0; i < 3; i++) mbar_init(&bar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (!STRIDED && a.needs_mt) {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.T->mul8);
        uint4 *dst = reinterpret_cast<uint4 *>(mt);
        for (int i = threadIdx.x; i < 4096; i += blockDim.x) dst[i] = __ldg(src + i);
    }
    if (!STRIDED && (a.needs_mt || a.low3)) {
        const uint4 *src = reinterpret_cast<const uint4 *>(&a.T->low_lane[0][0]);
        uint4 *dst = reinterpret_cast<uint4 *>(lane_tab);
        for (int i = threadIdx.x; i < (int)(kLaneTabBytes / 16); i += blockDim.x) dst[i] = __ldg(src + i);
    }
    const MtRef M = mt_ref(mt, lane_tab);
    if ((int)threadIdx.x < g && blockIdx.x < ntiles)
        cnext[threadIdx.x] = tile_cval(a, blockIdx.x & tmask, threadIdx.x);
    __syncthreads();
    if (blockIdx.x < ntiles) prefetch_tables(a, tb, cnext, stab);
    // everything above reads constant tables only; the tiles come from the
    // previous kernels of the stream
    pdl_acquire();
    if (blockIdx.x < ntiles && warp == 0 && pipe)
        tile_load_issue(G, src_of(blockIdx.x), src_tile(blockIdx.x & tmask), buf0, &bar[0], lane);

    bool aborted = false, prefetched = false;
    uint32_t i = 0;
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x, i++) {
        const int b = NB == 2 ? (i & 1) : 0;
        uint4 *s = buf0 + (b ? tile : 0);
        const uint64_t tn = t + gridDim.x;
        const uint64_t y = t >> tiles_log, tt = t & tmask;  // product, tile
        uint4 *const Fy = a.F + y * a.strideF;
        bool ok = true;
        prefetched = false;
        if (pipe) {
            if (NB == 2 && warp == 0 && tn < ntiles) {
                bulk_wait_read_all();  // the stores out of buf[b^1] have read it
                __syncwarp();
                tile_load_issue(G, src_of(tn), src_tile(tn & tmask), buf0 + (b ? 0 : tile),
                                &bar[b ^ 1], lane);
                prefetched = true;
            }
            ok = mbar_wait_bounded(&bar[b], NB == 2 ? (i >> 1) & 1 : i & 1, a.wait_spins);
        } else {
            if (warp == 0) bulk_wait_read_all();  // the stores out of buf[b] have read it
        }
        cp_async_wait_all();
        if (!__syncthreads_and(ok)) {
            aborted = true;
            break;
        }
        // this tile's shuffle tables and multipliers
        for (int q = threadIdx.x; q < gt * 224; q += blockDim.x) {
            const uint32_t *p4 = stab + (q / 224) * 896 + (q % 224);
            ctab[q] = p4[0] ^ p4[224] ^ p4[448] ^ p4[672];
        }
        if (threadIdx.x < 32) cval[threadIdx.x] = cnext[threadIdx.x];
        const uint64_t base = tile_base(G, tt);
        if (!STRIDED && from_g) {
            const uint64_t *gy = a.g64 + y * a.strideW;
            for (uint32_t q = threadIdx.x; q < tile; q += blockDim.x) {
                const uint64_t idx = base | ((uint64_t)(q >> c) << a.k_lo) | (q & cmask);
                s[q] = chrepr_ldg(a.T, __ldg(gy + (idx & a.pmask)));
            }
        }
        __syncthreads();
        // the next tile's multipliers and their tables
        if ((int)threadIdx.x < g && tn < ntiles) cnext[threadIdx.x] = tile_cval(a, tn & tmask, threadIdx.x);
        __syncthreads();
        if (tn < ntiles) prefetch_tables(a, tb, cnext, stab);

        if (a.mode != 1) {  // forward layers g_f-1 .. 0
            for (int r_hi = a.g_f - 1; r_hi >= ul; r_hi -= 3) {
                const int r_lo = max(ul, r_hi - 2);
                run_subpass<false, SIX>(r_hi - r_lo + 1, s, c, g, r_lo, uf, ctab_u, a.d_shfl);
                __syncthreads();
            }
            if (!STRIDED && ul > uf && a.g_f > uf) {  // rows 3 .. min(g_f, ul) - 1 limb-wise
                const int nr = min(a.g_f, ul) - uf;
                if (nr >= 3)
                    limb_subpass<3, false>(s, g, uf, ctab_u, a.d_shfl);
                else if (nr == 2)
                    limb_subpass<2, false>(s, g, uf, ctab_u, a.d_shfl);
                else
                    limb_subpass<1, false>(s, g, uf, ctab_u, a.d_shfl);
                __syncthreads();
            }
            if (STRIDED) {
            } else if (a.low3 && a.g_f >= 3) {  // rows 2, 1, 0 in registers
                low3_subpass<false>(s, g, ctab, a.T->low_shfl[0][0], &lane_tab[0]);
                __syncthreads();
            } else {
                for (int r = min(uf, a.g_f) - 1; r >= 0; r--) {
                    smem_layer<false>(s, g, r, M, cval[r], a.d_val);
                    __syncthreads();
                }
            }
        }
        if (!STRIDED && a.mode == 2) {  // pointmul with the other operand's transform
            for (uint32_t q = threadIdx.x; q < tile; q += blockDim.x) {
                const uint64_t idx = base | ((uint64_t)(q >> c) << a.k_lo) | (q & cmask);
                s[q] = mt_gmul128(M, s[q], __ldg(a.FA + y * a.strideFA + idx));
            }
            __syncthreads();
        }
        if (a.mode != 0) {  // inverse layers 0 .. g-1
            if (STRIDED) {
            } else if (a.low3) {  // rows 0, 1, 2 in registers
                low3_subpass<true>(s, g, ctab, a.T->low_shfl[0][0], &lane_tab[0]);
                __syncthreads();
            } else {
                for (int r = 0; r < min(uf, g); r++) {
                    smem_layer<true>(s, g, r, M, cval[r], a.d_val);
                    __syncthreads();
                }
            }
            if (!STRIDED && ul > uf) {  // rows 3 .. ul - 1 limb-wise
                if (ul - uf >= 3)
                    limb_subpass<3, true>(s, g, uf, ctab_u, a.d_shfl);
                else
                    limb_subpass<2, true>(s, g, uf, ctab_u, a.d_shfl);
                __syncthreads();
            }
            for (int r_lo = ul; r_lo < g; r_lo += 3) {
                const int r_hi = min(g - 1, r_lo + 2);
                run_subpass<true, SIX>(r_hi - r_lo + 1, s, c, g, r_lo, uf, ctab_u, a.d_shfl);
                __syncthreads();
            }
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (warp == 0) tile_store_issue(G, Fy, tt, s, lane);
        // one buffer: the next tile comes in once this one has been read out
        if (pipe && NB == 1 && warp == 0 && tn < ntiles) {
            bulk_wait_read_all();
            __syncwarp();
            tile_load_issue(G, src_of(tn), src_tile(tn & tmask), buf0, &bar[0], lane);
        }
    }
    if (aborted) {
        if (threadIdx.x == 0) {
            atomicExch(a.status, -4);  // GF2X_ETIMEOUT
            // Let every load still in flight land before the CTA exits (its
            // shared memory may be handed to another CTA next): the tile whose
            // wait ran out, and the next tile if it was already prefetched.
            // These waits take the default bound, not the caller's.
            if (pipe) {
                const int b = NB == 2 ? (i & 1) : 0;
                mbar_wait_bounded(&bar[b], NB == 2 ? (i >> 1) & 1 : i & 1);
            }
            if (prefetched) mbar_wait_bounded(&bar[(i & 1) ^ 1], ((i + 1) >> 1) & 1);
        }
        __syncthreads();
    }
    cp_async_wait_all();
    if (warp == 0) bulk_wait_all();
}

// ---------------------------------------------------------------------------
// pointmul alone (stage entry point): C[i] = A[i] * B[i].
__global__ void __launch_bounds__(256) k_pointmul_mt(const uint4 *__restrict__ A, const uint4 *B,
                                                      uint4 *C, uint64_t n,
                                                      const DevTables *__restrict__ T) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint8_t *mt = smem;
    const uint4 *src = reinterpret_cast<const uint4 *>(T->mul8);
    uint32_t *lane_tab = reinterpret_cast<uint32_t *>(smem + 65536);
    for (int i = threadIdx.x; i < 4096; i += blockDim.x) reinterpret_cast<uint4 *>(mt)[i] = __ldg(src + i);
    const uint4 *lsrc = reinterpret_cast<const uint4 *>(&T->low_lane[0][0]);
    for (int i = threadIdx.x; i < (int)(kLaneTabBytes / 16); i += blockDim.x)
        reinterpret_cast<uint4 *>(lane_tab)[i] = __ldg(lsrc + i);
    __syncthreads();
    const MtRef M = mt_ref(mt, lane_tab);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        C[i] = mt_gmul128(M, A[i], B[i]);
}

// ===========================================================================
// Host side: per-pass tables and pass schedules.

void pass_tables_size(int g, int uf, size_t *n_val, size_t *n_shfl) {
    *n_val = std::max<size_t>(((size_t)1 << g) - 1, 1);
    size_t m = 0;
    for (int r = uf; r < g; r++) m += (size_t)1 << (g - 1 - r);
    *n_shfl = 224 * m;
}

void pass_tables_fill(int k_lo, int g, int uf, uint32_t *val, uint32_t *shfl) {
    const HostTables &H = host_tables();
    auto s_of = [&](int k, uint64_t alpha) {
        uint32_t r = 0;
        for (int t = 0; t < 32; t++)
            if ((alpha >> t) & 1) r ^= H.S[k][t];
        return r;
    };
    val[0] = 0;
    size_t sh = 0;
    for (int r = 0; r < g; r++) {
        const int k = k_lo + r;
        const uint32_t voff = (1u << g) - (1u << (g - r));
        for (uint32_t p = 0; p < (1u << (g - 1 - r)); p++) {
            const uint32_t d = s_of(k, (uint64_t)p << (k + 1));
            val[voff + p] = d;
            if (r >= uf) {
                uint32_t t[7][32];
                shfl_table_of(d, t);
                for (int q = 0; q < 224; q++) shfl[sh + q] = (&t[0][0])[q];
                sh += 224;
            }
        }
    }
}

void pass_tables_host(int k_lo, int g, int uf, std::vector<uint32_t> &val,
                      std::vector<uint32_t> &shfl) {
    size_t nv, ns;
    pass_tables_size(g, uf, &nv, &ns);
    val.assign(nv, 0);
    shfl.assign(ns, 0);
    pass_tables_fill(k_lo, g, uf, val.data(), shfl.data());
}

namespace {

struct PassTables {
    uint32_t *d_val = nullptr;
    uint32_t *d_shfl = nullptr;
};

std::mutex g_pt_mu;
std::map<std::tuple<int, int, int, int>, PassTables> g_pt;  // (device, k_lo, g, uf)

// The library's own table source: built on the host once per (device, pass)
// and kept in device allocations.
int cached_pass_tables(int k_lo, int g, int uf, const uint32_t **d_val, const uint32_t **d_shfl) {
    int dev;
    if (cudaGetDevice(&dev) != cudaSuccess) return -3;
    auto key = std::make_tuple(dev, k_lo, g, uf);
    std::lock_guard<std::mutex> lk(g_pt_mu);
    auto it = g_pt.find(key);
    if (it == g_pt.end()) {
        std::vector<uint32_t> val, shfl;
        pass_tables_host(k_lo, g, uf, val, shfl);
        PassTables pt;
        if (cudaMalloc(&pt.d_val, val.size() * 4) != cudaSuccess) return -2;
        cudaMemcpy(pt.d_val, val.data(), val.size() * 4, cudaMemcpyHostToDevice);
        if (!shfl.empty()) {
            if (cudaMalloc(&pt.d_shfl, shfl.size() * 4) != cudaSuccess) return -2;
            cudaMemcpy(pt.d_shfl, shfl.data(), shfl.size() * 4, cudaMemcpyHostToDevice);
        }
        if (cudaGetLastError() != cudaSuccess) return -3;
        it = g_pt.emplace(key, pt).first;
    }
    *d_val = it->second.d_val;
    *d_shfl = it->second.d_shfl;
    return 0;
}

// Shared memory of a pass: one or two tile buffers, the shuffle tables of the
// tile's multipliers (rows uf.., or all rows with low3) and their staged byte
// slices, the multipliers, four mbarriers, then the F~_{2^8} product table if
// needed and the per-lane tables (with the product table or low3).
size_t pass_smem(int g, int c, int uf, bool needs_mt, int nbuf, bool low3) {
    size_t b = ((size_t)16 * nbuf) << (g + c);
    b += (size_t)(g - (low3 ? 0 : uf)) * 224 * 4 * 5 + 64 * 4 + 4 * 8;
    if (needs_mt) b += 65536;
    if (needs_mt || low3) b += kLaneTabBytes;
    return b;
}

int make_pass(int k_lo, int g, int c, int uf, int mode, int g_f, PassTableFn src, FftPassCfg *p,
              int nbuf = 2) {
    // register sub-passes need a warp's 32 lanes inside the column bits and
    // the rows below the sub-pass, so that the lanes share the multiplier; a
    // contiguous pass may start them at row 3 (rows 3, 4 limb-wise)
    const bool limb34 = c == 0 && uf == 3 && g >= 5;
    if (uf < g && c + uf < 5 && !limb34) return -1;
    int rc = (src ? src : cached_pass_tables)(k_lo, g, uf, &p->d_val, &p->d_shfl);
    if (rc) return rc;
    // the passes read two words of each shuffle table as one 8-byte load
    // (shfl6_table_sum): a table array that does not start on a 16-byte
    // boundary is refused here rather than launched
    if (reinterpret_cast<uintptr_t>(p->d_shfl) & 15) return -3;
    p->k_lo = k_lo;
    p->g = g;
    p->c = c;
    p->uf = uf;
    p->mode = mode;
    p->g_f = g_f;
    // rows 0-2 of a contiguous tile of 2^8.. elements in registers (low3);
    // the product table for the other lane-varying rows and for pointmul
    p->low3 = c == 0 && uf == 3 && g >= 8;
    p->needs_mt = (uf > 0 && !p->low3) || mode == 2;
    // one buffer where two CTAs then fit an SM (no product table), or where
    // two buffers would not fit
    p->nbuf = (nbuf == 1 && !p->needs_mt) ? 1 : 2;
    if (pass_smem(g, c, uf, p->needs_mt, p->nbuf, p->low3) > kMaxPassSmem) p->nbuf = 1;
    p->smem = pass_smem(g, c, uf, p->needs_mt, p->nbuf, p->low3);
    p->threads = std::max(32, std::min(p->nbuf == 1 ? 256 : 512, (1 << (g + c)) / 2));
    return 0;
}

int push_pass(PassList &out, const FftPassCfg &p) {
    if (out.n >= PassList::kMax) return -1;
    out.v[out.n++] = p;
    return 0;
}

// Strided passes covering layers [lo, hi) from the top down (forward) or
// bottom up (inverse), at most kFftGlobalMax layers each, balanced; each
// tile is 2^g rows by 2^(12-g) columns.
int global_passes(int lo, int hi, bool inverse, PassTableFn src, PassList &out, int depth,
                  int nbuf) {
    const int L = hi - lo;
    if (L <= 0) return 0;
    depth = std::max(1, std::min(depth, kFftGlobalMax));
    depth = std::max(depth, (L + PassList::kMax - 1) / PassList::kMax);  // at most kMax passes
    const int n = (L + depth - 1) / depth;
    if (n > PassList::kMax) return -1;
    int klo[PassList::kMax], gg[PassList::kMax];
    int k = lo;
    for (int i = 0; i < n; i++) {
        gg[i] = L / n + (i < L % n ? 1 : 0);
        klo[i] = k;
        k += gg[i];
    }
    for (int q = 0; q < n; q++) {
        const int i = inverse ? q : n - 1 - q;
        FftPassCfg p;
        int rc = make_pass(klo[i], gg[i], kFftTileLog - gg[i], 0, inverse ? 1 : 0, gg[i], src, &p,
                           nbuf);
        if (rc || (rc = push_pass(out, p))) return rc;
    }
    return 0;
}

}  // namespace

int plan_fft_forward(int M, int log_p, PassList &out, PassTableFn src, int depth, int nbuf) {
    out.n = 0;
    int rc = global_passes(kFftTileLog, log_p, false, src, out, depth, nbuf);
    if (rc) return rc;
    const int gl = std::min(log_p, kFftTileLog);
    FftPassCfg p;
    if ((rc = make_pass(0, gl, 0, bottom_uf(gl), 0, gl, src, &p))) return rc;
    (void)M;
    return push_pass(out, p);
}

int plan_fft_inverse(int M, PassList &out, PassTableFn src, int depth, int nbuf) {
    out.n = 0;
    const int gl = std::min(M, kFftTileLog);
    FftPassCfg p;
    int rc = make_pass(0, gl, 0, bottom_uf(gl), 1, gl, src, &p);
    if (rc || (rc = push_pass(out, p))) return rc;
    return global_passes(kFftTileLog, M, true, src, out, depth, nbuf);
}

int plan_fft_fused(int M, int log_p, PassList &fwd_global, FftPassCfg &local, PassList &inv_global,
                   PassTableFn src, int depth, int nbuf) {
    fwd_global.n = 0;
    inv_global.n = 0;
    int rc = global_passes(kFftTileLog, log_p, false, src, fwd_global, depth, nbuf);
    if (rc) return rc;
    const int gl = std::min(M, kFftTileLog);
    const int gf = std::min(log_p, kFftTileLog);
    if ((rc = make_pass(0, gl, 0, bottom_uf(gl), 2, gf, src, &local))) return rc;
    return global_passes(kFftTileLog, M, true, src, inv_global, depth, nbuf);
}

void prepare_fft_attributes() {
    ensure_smem_attr(reinterpret_cast<const void *>(k_fft_pass<false>), 227 * 1024);
    ensure_smem_attr(reinterpret_cast<const void *>(k_fft_pass<true>), 227 * 1024);
    ensure_smem_attr(reinterpret_cast<const void *>(k_pointmul_mt), 65536);
    num_sms();
}

// CTAs of k_fft_pass resident per SM for this block size and shared memory
// (at least 1): 128 registers per thread of 64 Ki, 228 KiB of shared memory
// per SM with 1 KiB reserved per CTA.  Computed rather than queried so that it
// is safe while a stream is being captured.
static int resident_ctas(int threads, size_t smem) {
    const int by_regs = 65536 / std::max(1, threads * 128);
    const int by_smem = (int)(233472 / (smem + 1024));
    return std::max(1, std::min(by_regs, by_smem));
}

int launch_fft_pass(const FftPassCfg &p, int M, uint4 *F, const uint64_t *g64, uint64_t P,
                    const uint4 *FA, const DevTables *T, int *status, cudaStream_t s, int count,
                    uint64_t strideF, uint64_t strideW, const uint4 *Fsrc, uint64_t strideFA) {
    const bool strided = p.c > 0;
    ensure_smem_attr(strided ? reinterpret_cast<const void *>(k_fft_pass<true>)
                             : reinterpret_cast<const void *>(k_fft_pass<false>),
                     227 * 1024);
    FftPassArgs a;
    a.F = F;
    a.Fsrc = Fsrc;
    a.g64 = g64;
    a.pmask = P ? P - 1 : 0;
    a.FA = FA;
    a.T = T;
    a.d_val = p.d_val;
    a.d_shfl = p.d_shfl;
    a.k_lo = p.k_lo;
    a.g = p.g;
    a.c = p.c;
    a.uf = p.uf;
    a.mode = p.mode;
    a.g_f = p.g_f;
    a.needs_mt = p.needs_mt;
    a.low3 = p.low3;
    a.M = M;
    a.status = status;
    a.count = count;
    a.strideF = strideF;
    a.strideFA = strideFA == ~0ull ? strideF : strideFA;
    a.strideW = strideW;
    a.nbuf = p.nbuf;
    a.wait_spins = wait_spins();
    const uint64_t tiles = ((1ull << M) >> (p.g + p.c)) * (uint64_t)count;
    const size_t smem = pass_smem(p.g, p.c, p.uf, p.needs_mt, p.nbuf, p.low3);
    // persistent CTAs: as many as are resident at once; a CTA alone on its SM
    // (shared memory too large for two) gets the full 512 threads
    int threads = p.threads;
    int per_sm = resident_ctas(threads, smem);
    if (per_sm == 1) threads = std::max(threads, std::min(512, (1 << (p.g + p.c)) / 2));
    const uint64_t ctas = (uint64_t)num_sms() * per_sm;
    const unsigned grid = (unsigned)std::min<uint64_t>(tiles, ctas);
    launch_k(strided ? k_fft_pass<true> : k_fft_pass<false>, grid, threads, smem, s, a);
    return 0;
}

void launch_pointmul_mt(const uint4 *A, const uint4 *B, uint4 *C, uint64_t n, const DevTables *T,
                        cudaStream_t s) {
    const int smem = 65536 + (int)kLaneTabBytes;
    ensure_smem_attr(reinterpret_cast<const void *>(k_pointmul_mt), smem);
    uint64_t blocks = std::min<uint64_t>((n + 255) / 256, 152 * 2);
    k_pointmul_mt<<<(unsigned)std::max<uint64_t>(1, blocks), 256, smem, s>>>(A, B, C, n, T);
}

}  // namespace gf2x
