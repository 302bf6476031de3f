// CUDA kernels of the product path (Alg. 5) other than the FFT passes, and
// their host launchers.  Every launcher takes a product count: the products of
// one batch share a plan and lie in one workspace at a fixed stride, so a
// batch costs one launch per kernel (blockIdx.y = product).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <set>
#include <tuple>
#include <vector>

#include "gf2x_dev.cuh"
#include "gf2x_internal.h"
#include "kernels.h"
#include "launch.h"

namespace gf2x {

bool pdl_enabled() {
    static const bool on = [] {
        const char *e = std::getenv("GF2X_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}

// ---------------------------------------------------------------------------
// Split (Sec. 2.1): copy the operand's words, clear bits past its length and
// zero-pad to P words.  Product y reads `many[y]` (or `one` if many is null)
// and writes w + y * stride.
__global__ void k_split_pad(OperandDesc one, const OperandDesc *__restrict__ many,
                            uint64_t *__restrict__ w, uint64_t P, uint64_t stride) {
    pdl_release();
    pdl_acquire();
    const OperandDesc d = many ? many[blockIdx.y] : one;
    w += blockIdx.y * stride;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < P;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t v = 0;
        if (i < d.nw) {
            v = d.src[i];
            if (i == d.nw - 1) v &= d.mask;
        }
        w[i] = v;
    }
}

// ---------------------------------------------------------------------------
// BasisCvt levels (Alg. 2 / Alg. 3).  Division of every segment of 2E
// coefficients by x^E + x^e (e | E, E >= 2e) is two data-parallel steps:
//   step 1: f[E+q]  ^= f[2E-e+q]   for 0 <= q < e
//   step 2: f[e+t]  ^= f[E+t]      for 0 <= t < E-e
// Step 2 reads f[E .. E+e) after step 1, so the work item t < e does both:
// it owns f[E+t] and f[e+t].  The inverse undoes step 2 first.

__device__ __forceinline__ uint64_t xr(uint64_t a, uint64_t b) { return a ^ b; }
__device__ __forceinline__ uint4 xr(uint4 a, uint4 b) { return xor4(a, b); }

template <typename T>
__device__ __forceinline__ void bcvt_item(T *f, uint64_t base, uint64_t E, uint64_t e, uint64_t t,
                                          int inverse) {
    if (t < e) {
        T hi = f[base + E + t];
        T top = f[base + 2 * E - e + t];
        if (!inverse) {
            T q = xr(hi, top);
            f[base + E + t] = q;
            f[base + e + t] = xr(f[base + e + t], q);
        } else {
            f[base + e + t] = xr(f[base + e + t], hi);
            f[base + E + t] = xr(hi, top);
        }
    } else {
        f[base + e + t] = xr(f[base + e + t], f[base + E + t]);
    }
}

template <typename T>
__global__ void k_bcvt_level(T *f, uint64_t n_half, int logE, int loge, int inverse,
                             uint64_t stride) {
    pdl_release();
    pdl_acquire();
    f += blockIdx.y * stride;
    const uint64_t E = 1ull << logE, e = 1ull << loge;
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < n_half;
         w += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t s = w >> logE, t = w & (E - 1);
        if (t >= E - e) continue;
        bcvt_item(f, s << (logE + 1), E, e, t, inverse);
    }
}

// A run of G consecutive levels (a, a - K), a = a_top .. a_top - G + 1, in
// one sweep over a shared-memory tile.  Every XOR of level a joins indices
// that differ by E - e = 2^(a - a_low) S, S = (2^K - 1) 2^(a_low - K), inside
// the aligned segments of Z = 2^(a_top + 1) elements, so each segment splits
// into the classes {r + n S : r + n S < Z}, r < S, which the G levels never
// mix (at most ceil(Z / S) <= RM rows; the host picks G so that they fit).  A
// thread loads one class into registers, applies the G divisions with the
// exact step conditions of each row's position, and stores it back: one
// shared-memory round trip per run instead of one per level.
// Shared-memory position of tile index x: the low four bits are XORed with
// bits 4..7, so that threads reading groups of 16 consecutive elements at the
// same offset hit different banks (a bijection on every aligned 256-element
// block; runs of consecutive indices stay consecutive up to a permutation
// inside each aligned 16-element block).
__device__ __forceinline__ uint32_t sw(uint32_t x) { return x ^ ((x >> 4) & 15u); }

// Rows of one class for a run of G levels with step K: ceil(2^(G+K) / (2^K - 1)).
__host__ __device__ constexpr int run_rows(int G, int K) {
    return (int)((((1u << (G + K)) + (1u << K) - 2) / ((1u << K) - 1)));
}

// K and G are known at compile time (bcvt_run_k).  All positions of a
// class r are multiples of e_low = 2^(a_low - K) plus r mod e_low, and E, e
// and the segment sizes are multiples of e_low, so the step conditions of a
// row depend only on r_hi = r >> (a_low - K); on a boundary class
// (r_hi < 2^G) they are evaluated here at compile time for each r_hi:
// row n sits at o = (r_hi + n (2^K - 1)) mod 2^(jj + K + 1) in units of
// e_low, with E = 2^(jj + K) and e = 2^jj.
template <int K, int G, int RH>
__host__ __device__ constexpr bool bnd_valid(int n) {
    return RH + n * ((1 << K) - 1) < (1 << (K + G));
}

template <int K, int RH, bool INV>
__host__ __device__ constexpr bool bnd_act(int jj, int st, int n) {
    const int o = (RH + n * ((1 << K) - 1)) & ((2 << (jj + K)) - 1);
    const int E = 1 << (jj + K), e = 1 << jj;
    const bool step1 = (st == 0) != INV;
    return step1 ? (o >= E && o - E < e) : (o >= e && o - e < E - e);
}

template <typename T, int K, int G, int RH, bool INV>
__device__ __forceinline__ void bnd_class(T *s, uint32_t sb, uint32_t S) {
    constexpr int RM = run_rows(G, K);
    T v[RM];
#pragma unroll
    for (int n = 0; n < RM; n++)
        if (bnd_valid<K, G, RH>(n)) v[n] = s[sw(sb + n * S)];
#pragma unroll
    for (int it = 0; it < G; it++) {
        const int jj = INV ? it : G - 1 - it;
#pragma unroll
        for (int st = 0; st < 2; st++)
#pragma unroll
            for (int n = 0; n + (1 << jj) < RM; n++)
                if (bnd_valid<K, G, RH>(n) && bnd_act<K, RH, INV>(jj, st, n))
                    v[n] = xr(v[n], v[n + (1 << jj)]);
    }
#pragma unroll
    for (int n = 0; n < RM; n++)
        if (bnd_valid<K, G, RH>(n)) s[sw(sb + n * S)] = v[n];
}

template <typename T, int K, int G, bool INV, int RH = 0>
__device__ __forceinline__ void bnd_dispatch(T *s, uint32_t sb, uint32_t S, uint32_t rh) {
    if constexpr (RH < (1 << G)) {
        if (rh == RH) {
            bnd_class<T, K, G, RH, INV>(s, sb, S);
            return;
        }
        bnd_dispatch<T, K, G, INV, RH + 1>(s, sb, S, rh);
    }
}

template <typename T, int K, int G, bool INV>
__device__ __forceinline__ void bcvt_run_k(T *s, uint32_t tile, int a_top) {
    const int a_low = a_top - G + 1, sh = a_low - K;
    const uint32_t S = ((1u << K) - 1) << sh;
    const uint32_t Z = 1u << (a_top + 1);
    const uint32_t items = (tile >> (a_top + 1)) * S;
    // Classes r >= 2^G e_low are interior: writing r + n S = n 2^a_low +
    // (r - n e_low), row n sits at (n mod 2^(jj+1)) 2^a_low + (r - n e_low) in
    // its level segment, so step 1 never applies and step 2 applies exactly to
    // the rows with bit jj of n clear: the run is a superset-sum over the G row
    // bits (order-free, its own inverse).
    const uint32_t r_int = (1u << G) << sh;
    // q / S as a multiply-high: with m = ceil(2^32 / S) the quotient is exact
    // while q * S < 2^32 (q, S < 2^16 in a tile; S = (2^K - 1) 2^sh >= 3)
    const uint32_t mS = 0xffffffffu / S + 1u;
    for (uint32_t q = threadIdx.x; q < items; q += blockDim.x) {
        const uint32_t seg = __umulhi(q, mS), r = q - seg * S;
        const uint32_t sb = seg * Z + r;
        if (r >= r_int) {  // interior: superset-sum over the G row bits
            T v[1 << G];
#pragma unroll
            for (int n = 0; n < (1 << G); n++) v[n] = s[sw(sb + n * S)];
#pragma unroll
            for (int jj = 0; jj < G; jj++)
#pragma unroll
                for (int n = 0; n < (1 << G); n++)
                    if (!((n >> jj) & 1)) v[n] = xr(v[n], v[n + (1 << jj)]);
#pragma unroll
            for (int n = 0; n < (1 << G); n++) s[sw(sb + n * S)] = v[n];
        } else {
            bnd_dispatch<T, K, G, INV>(s, sb, S, r >> sh);
        }
    }
}

template <typename T, bool INV>
__device__ __forceinline__ void bcvt_run_any(T *s, uint32_t tile, int a_top, int K, int G) {
    // the (K, G) pairs of tile runs (bcvt_tile_run_ok on the host)
    switch (K * 8 + G) {
        case 2 * 8 + 1: bcvt_run_k<T, 2, 1, INV>(s, tile, a_top); return;
        case 4 * 8 + 1: bcvt_run_k<T, 4, 1, INV>(s, tile, a_top); return;
        case 4 * 8 + 2: bcvt_run_k<T, 4, 2, INV>(s, tile, a_top); return;
        case 8 * 8 + 1: bcvt_run_k<T, 8, 1, INV>(s, tile, a_top); return;
        case 8 * 8 + 2: bcvt_run_k<T, 8, 2, INV>(s, tile, a_top); return;
        case 8 * 8 + 3: bcvt_run_k<T, 8, 3, INV>(s, tile, a_top); return;
        default: return;
    }
}

static bool bcvt_tile_run_ok(int K, int G) {
    return (K == 2 && G == 1) || (K == 4 && G >= 1 && G <= 2) || (K == 8 && G >= 1 && G <= 3);
}

// A run of G divisions (a, a - K), a = a_top .. a_top - G + 1, as one
// streaming pass over the whole array (runs too wide for a shared-memory
// tile: K >= 8).  The classes {r + n S} of bcvt_run_k are taken straight from
// global memory, one 32-bit limb of one class per thread (the divisions act
// bitwise); consecutive threads take consecutive (class, limb) pairs, so every
// row is read and written in full 128-byte lines.  Interior classes
// (r >= 2^G e_low) are a superset-sum over the row bits; the others apply the
// exact step conditions of each row's position.
template <typename T, int G, int RM, bool INV, bool BND>
__global__ void __launch_bounds__(256) k_bcvt_class(T *f, int a_top, int K, uint64_t n_el,
                                                    uint64_t stride) {
    pdl_release();
    pdl_acquire();
    constexpr int L = sizeof(T) / 4;
    f += blockIdx.y * stride;
    uint32_t *const F = reinterpret_cast<uint32_t *>(f);
    const int a_low = a_top - G + 1;
    const uint64_t e_low = 1ull << (a_low - K);
    const uint64_t S = ((1ull << K) - 1) * e_low;
    const uint64_t Z = 1ull << (a_top + 1);
    const uint64_t r_int = e_low << G;
    // this launch's classes in each segment: [0, r_int) or [r_int, S)
    const uint64_t r0 = BND ? 0 : r_int, nr = BND ? r_int : S - r_int;
    const uint64_t items = (n_el / Z) * nr * L;
    const uint64_t rowstep = S * L;
    // rest / nr as a multiply-high: with m = ceil(2^64 / nr) the quotient is
    // exact while rest * nr < 2^64
    const uint64_t mnr = nr > 1 ? ~0ull / nr + 1ull : 0;
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < items;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t rest = q / L;
        const uint64_t seg = nr > 1 ? __umul64hi(rest, mnr) : rest, r = r0 + (rest - seg * nr);
        uint32_t *const base = F + (seg * Z + r) * L + (q % L);
        if constexpr (!BND) {
            uint32_t v[1 << G];
#pragma unroll
            for (int n = 0; n < (1 << G); n++) v[n] = base[n * rowstep];
#pragma unroll
            for (int jj = 0; jj < G; jj++)
#pragma unroll
                for (int n = 0; n < (1 << G); n++)
                    if (!((n >> jj) & 1)) v[n] ^= v[n + (1 << jj)];
#pragma unroll
            for (int n = 0; n < (1 << G); n++) base[n * rowstep] = v[n];
        } else {
            uint32_t v[RM];
            uint32_t valid = 0;
#pragma unroll
            for (int n = 0; n < RM; n++) {
                v[n] = 0;
                if (r + (uint64_t)n * S < Z) {
                    valid |= 1u << n;
                    v[n] = base[n * rowstep];
                }
            }
#pragma unroll
            for (int it = 0; it < G; it++) {
                const int jj = INV ? it : G - 1 - it;
                const int a = a_low + jj;
                const uint64_t E = 1ull << a, e = 1ull << (a - K), msk = 2 * E - 1;
#pragma unroll
                for (int st = 0; st < 2; st++) {
                    const bool step1 = (st == 0) != INV;
#pragma unroll
                    for (int n = 0; n < RM; n++) {
                        const int p = n + (1 << jj);
                        if (p >= RM || !((valid >> n) & 1u)) continue;
                        const uint64_t o = (r + (uint64_t)n * S) & msk;
                        if (step1 ? (o - E < e) : (o - e < E - e)) v[n] ^= v[p];
                    }
                }
            }
#pragma unroll
            for (int n = 0; n < RM; n++)
                if ((valid >> n) & 1u) base[n * rowstep] = v[n];
        }
    }
}

// One division by x^E + x^e on every segment of 2E registers of v (Alg. 2
// steps 1 and 2; the inverse undoes step 2 first).
template <int N, int E, int e, bool INV, typename T>
__device__ __forceinline__ void div_regs(T (&v)[N]) {
#pragma unroll
    for (int s0 = 0; s0 < N; s0 += 2 * E) {
        if (!INV) {
#pragma unroll
            for (int q = 0; q < e; q++) v[s0 + E + q] = xr(v[s0 + E + q], v[s0 + 2 * E - e + q]);
#pragma unroll
            for (int t = 0; t < E - e; t++) v[s0 + e + t] = xr(v[s0 + e + t], v[s0 + E + t]);
        } else {
#pragma unroll
            for (int t = 0; t < E - e; t++) v[s0 + e + t] = xr(v[s0 + e + t], v[s0 + E + t]);
#pragma unroll
            for (int q = 0; q < e; q++) v[s0 + E + q] = xr(v[s0 + E + q], v[s0 + 2 * E - e + q]);
        }
    }
}

// The whole BasisCvt of M = 2 or 4 index bits at scale sc (Alg. 3 on 2^M
// coefficients spaced 2^sc apart): a thread holds one group in registers and
// applies its divisions, known at compile time.  For M = 4 they are
// (x^8 + x^2), (x^4 + x) on each half, then (x^2 + x) and (x^8 + x^4) on each
// quarter (the children in the library's order); for M = 2 the single
// (x^2 + x).
template <typename T, int M, bool INV>
__device__ __forceinline__ void bcvt_sub(T *s, uint32_t tile, int sc) {
    constexpr int N = 1 << M;
    const uint32_t groups = tile >> M, lowmask = (1u << sc) - 1;
    for (uint32_t q = threadIdx.x; q < groups; q += blockDim.x) {
        const uint32_t sb = ((q >> sc) << (sc + M)) | (q & lowmask);
        T v[N];
#pragma unroll
        for (int i = 0; i < N; i++) v[i] = s[sw(sb + (i << sc))];
        if constexpr (M == 2) {
            div_regs<4, 2, 1, INV>(v);
        } else if constexpr (!INV) {
            div_regs<16, 8, 2, false>(v);
            div_regs<16, 4, 1, false>(v);
            div_regs<16, 2, 1, false>(v);
            div_regs<16, 8, 4, false>(v);
        } else {
            div_regs<16, 8, 4, true>(v);
            div_regs<16, 2, 1, true>(v);
            div_regs<16, 4, 1, true>(v);
            div_regs<16, 8, 2, true>(v);
        }
#pragma unroll
        for (int i = 0; i < N; i++) s[sw(sb + (i << sc))] = v[i];
    }
}

template <typename T, bool INV>
__device__ __forceinline__ void bcvt_op(T *s, uint32_t tile, const BcvtOp &op) {
    if (op.kind == 1)
        bcvt_sub<T, 2, INV>(s, tile, op.a_top);
    else if (op.kind == 2)
        bcvt_sub<T, 4, INV>(s, tile, op.a_top);
    else
        bcvt_run_any<T, INV>(s, tile, op.a_top, op.K, op.G);
}

// A strided tile: index bits [0, c) ("columns", consecutive in memory) and
// [lo, lo + w) ("rows"); the other bits name the CTA.  A level whose mixing
// bits [loge, logE] lie inside the rows acts on the tile-local index
// (row << c) | col exactly as on the global index, with logE and loge moved
// by c - lo (the steps in `lb` are given in tile-local form).
// SMALL: launched with at most 256 threads and 64 KiB of shared memory; for
// 64-bit coefficients four such CTAs share an SM (64 registers per thread).
// 128-bit tiles of at most 64 KiB: at most 85 registers per thread so that three
// 256-thread CTAs share an SM (iBasisCvt 0.41 -> 0.37 ms at 2^28; four CTAs,
// 64 registers, spill and come to 0.39 ms).
#ifndef GF2X_BCVT128_MINB
#define GF2X_BCVT128_MINB 3
#endif
//
// PHI (64-bit blocks, the last pass of a forward conversion): the tile leaves
// as changeRepr'd 128-bit elements (tile_store_phi) to phi.out and f is not
// written; three CTAs per SM (80 registers, no spills; at 64 registers the
// store's tables spill).
constexpr int kPhiTabWords = 4 * 2 * 7 * 32;  // DevTables::phi_shfl

// changeRepr of a tile's blocks on the way out: word o of phi(b) is the XOR of
// the 14 five-bit-window entries of b's two 32-bit halves (DevTables::phi_shfl,
// staged in shared memory; lane l holds entry l of a window's table and a
// lookup is one shuffle).  A warp takes 128 consecutive tile entries (lane l:
// entries l + 32 k), one output word of phi at a time, and writes each
// element at its global index.
__device__ __forceinline__ void tile_store_phi(const uint64_t *s, uint32_t tile, uint4 *out,
                                               uint64_t base, int c, int lo, const uint32_t *tab) {
    constexpr int K = 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t cmask = (1u << c) - 1;
    for (uint32_t c0 = warp * 32u * K; c0 < tile; c0 += nw * 32u * K) {
        uint32_t b[K][2];
#pragma unroll
        for (int k = 0; k < K; k++) {
            const uint32_t i = c0 + 32 * k + lane;
            const uint64_t v = i < tile ? s[sw(i)] : 0;
            b[k][0] = (uint32_t)v;
            b[k][1] = (uint32_t)(v >> 32);
        }
        uint32_t r[K][4] = {};
#pragma unroll 1
        for (int o = 0; o < 4; o++) {
            uint32_t tb[14];
#pragma unroll
            for (int qw = 0; qw < 14; qw++) tb[qw] = tab[(o * 14 + qw) * 32 + lane];
#pragma unroll
            for (int k = 0; k < K; k++) {
                uint32_t wv[2] = {b[k][0], b[k][1]};
                asm volatile("" : "+r"(wv[0]), "+r"(wv[1]));  // shifts stay inside the loop over o
                uint32_t acc = 0;
#pragma unroll
                for (int q = 0; q < 2; q++) {
#pragma unroll
                    for (int wd = 0; wd < 6; wd++)
                        acc ^= __shfl_sync(0xffffffffu, tb[q * 7 + wd], wv[q] >> (5 * wd));
                    acc ^= __shfl_sync(0xffffffffu, tb[q * 7 + 6], wv[q] >> 30);
                }
#pragma unroll
                for (int oo = 0; oo < 4; oo++) r[k][oo] = o == oo ? acc : r[k][oo];
            }
        }
#pragma unroll
        for (int k = 0; k < K; k++) {
            const uint32_t i = c0 + 32 * k + lane;
            if (i < tile)
                out[base | ((uint64_t)(i >> c) << lo) | (i & cmask)] =
                    make_uint4(r[k][0], r[k][1], r[k][2], r[k][3]);
        }
    }
}

template <typename T, bool SMALL, bool PHI>
__global__ void __launch_bounds__(SMALL ? 256 : 512,
                                  SMALL ? (sizeof(T) == 8 ? (PHI ? 3 : 4) : GF2X_BCVT128_MINB) : 1)
    k_bcvt_tile(T *f, int c, int lo, int w, LevelBatch lb,
                                                      int inverse, uint64_t stride, PhiOut phi) {
    static_assert(!PHI || sizeof(T) == 8, "changeRepr applies to 64-bit blocks");
    pdl_release();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s = reinterpret_cast<T *>(smem_raw);
    const uint32_t tile = 1u << (c + w);
    uint32_t *phi_tab = reinterpret_cast<uint32_t *>(smem_raw + sizeof(T) * (size_t)tile);
    if (PHI) {  // constant tables: before the wait
        const uint4 *src = reinterpret_cast<const uint4 *>(&phi.T->phi_shfl[0][0][0][0]);
        for (int i = threadIdx.x; i < kPhiTabWords / 4; i += blockDim.x)
            reinterpret_cast<uint4 *>(phi_tab)[i] = __ldg(src + i);
    }
    pdl_acquire();
    f += blockIdx.y * stride;
    const int mid_bits = lo - c;
    const uint64_t mid = blockIdx.x & ((1ull << mid_bits) - 1);
    const uint64_t hi = (uint64_t)blockIdx.x >> mid_bits;
    const uint64_t base = (hi << (lo + w)) | (mid << c);
    const uint32_t cmask = (1u << c) - 1;
    // U independent loads per thread in flight (the tile is one CTA's only work)
    constexpr int U = sizeof(T) == 8 ? 16 : 8;
    for (uint32_t i0 = threadIdx.x; i0 < tile; i0 += U * blockDim.x) {
        T v[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint32_t i = i0 + u * blockDim.x;
            if (i < tile) v[u] = f[base | ((uint64_t)(i >> c) << lo) | (i & cmask)];
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint32_t i = i0 + u * blockDim.x;
            if (i < tile) s[sw(i)] = v[u];
        }
    }
    __syncthreads();
    for (int L = 0; L < lb.count; L++) {
        if (inverse)
            bcvt_op<T, true>(s, tile, lb.op[L]);
        else
            bcvt_op<T, false>(s, tile, lb.op[L]);
        __syncthreads();
    }
    if constexpr (PHI) {
        tile_store_phi(s, tile, phi.out + blockIdx.y * phi.stride, base, c, lo, phi_tab);
        return;
    }
    for (uint32_t i = threadIdx.x; i < tile; i += blockDim.x)
        f[base | ((uint64_t)(i >> c) << lo) | (i & cmask)] = s[sw(i)];
}

// ---------------------------------------------------------------------------
// The top VarSubs of a BasisCvt of 2^m coefficients, m = 16 + h with
// 1 <= h <= 8 (Alg. 3 with K = 16): the h divisions by x^E + x^e with
// E = 2^(16+j), e = 2^j, j = h-1 .. 0.  These are the only levels whose
// mixing range (17 index bits) is too wide for a shared-memory tile.
//
// Every XOR of division j joins two indices that differ by E - e = 2^j D,
// D = 2^16 - 1, so the array splits into independent classes
// {c + n D : n >= 0}, c < D, whose members we call rows n.  As
// c + n D = n 2^16 + (c - n), for a class with c >= 3 * 2^(h-1) (so that
// c - n >= 2^(h-1) >= e for every row n < 2^h) the position of row n inside
// its segment of 2E coefficients is (n mod 2^(j+1)) 2^16 + (c - n): step 1
// never applies and step 2 applies exactly to the rows with bit j of n clear,
// row[n] ^= row[n + 2^j].  On such a class the h divisions are therefore the
// transform row[n] = XOR of row[n'] over n' containing the bits of n, which
// is its own inverse and does not depend on the order of the levels.  A
// thread holds one 32-bit limb of 2^HR rows of a class in registers (the
// divisions act bitwise, so limbs are independent); the remaining h - HR row
// bits are spread over lanes and joined by shuffles.  The classes
// c < 3 * 2^(h-1) (at most 384, where a row may sit at the start of its
// segment) take the two steps of every division exactly, in shared memory.

constexpr uint32_t kTopD = 65535;         // 2^16 - 1
constexpr int kTopThreads = 128;
constexpr uint32_t kTopBoundaryClasses = 8;  // classes per boundary CTA

__host__ __device__ constexpr uint32_t top_boundary(int h) { return (1u << h) + (1u << (h - 1)); }

template <typename T, int HR>
__global__ void __launch_bounds__(kTopThreads) k_bcvt_top(T *f, int h, int inverse,
                                                          uint32_t n_bnd_ctas, uint64_t stride) {
    pdl_release();
    pdl_acquire();
    f += blockIdx.y * stride;
    const uint32_t B = top_boundary(h);
    if (blockIdx.x < n_bnd_ctas) {
        // boundary classes [c0, c0 + 8) intersected with [0, B)
        extern __shared__ __align__(16) unsigned char smem_raw[];
        T *s = reinterpret_cast<T *>(smem_raw);
        const uint64_t n_el = 1ull << (16 + h);
        const uint32_t R = (1u << h) + 1, items = kTopBoundaryClasses * R;
        const uint32_t c0 = blockIdx.x * kTopBoundaryClasses;
        for (uint32_t q = threadIdx.x; q < items; q += blockDim.x) {
            const uint32_t c = c0 + q / R;
            const uint64_t x = c + (uint64_t)(q % R) * kTopD;
            T v;
            memset(&v, 0, sizeof(T));
            if (c < B && x < n_el) v = f[x];
            s[q] = v;
        }
        __syncthreads();
        for (int it = 0; it < h; it++) {
            const int j = inverse ? it : h - 1 - it;
            const uint64_t E = 1ull << (16 + j), e = 1ull << j;
            for (int st = 0; st < 2; st++) {
                // forward: step 1 then step 2; inverse: step 2 then step 1
                const bool step1 = (st == 0) != (inverse != 0);
                for (uint32_t q = threadIdx.x; q < items; q += blockDim.x) {
                    const uint32_t c = c0 + q / R, n = q % R;
                    if (c >= B || n + (1u << j) >= R) continue;
                    const uint64_t x = c + (uint64_t)n * kTopD;
                    if (x + ((uint64_t)kTopD << j) >= n_el) continue;
                    const uint64_t o = x & (2 * E - 1);
                    const bool act = step1 ? (o >= E && o < E + e) : (o >= e && o < E);
                    if (act) s[q] = xr(s[q], s[q + (1u << j)]);
                }
                __syncthreads();
            }
        }
        for (uint32_t q = threadIdx.x; q < items; q += blockDim.x) {
            const uint32_t c = c0 + q / R;
            const uint64_t x = c + (uint64_t)(q % R) * kTopD;
            if (c < B && x < n_el) f[x] = s[q];
        }
        return;
    }
    // interior classes
    constexpr int L = sizeof(T) / 4;
    const int LB = h - HR;      // row bits held across lanes (0 .. 2)
    const int G = 32 >> LB;     // lanes per row group
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cl = lane & (G - 1), nh = lane >> (5 - LB);
    const uint32_t cls_per_warp = G / L;
    const uint32_t c = B + (blockIdx.x - n_bnd_ctas) * (cls_per_warp * (kTopThreads / 32)) +
                       warp * cls_per_warp + cl / L;
    const bool valid = c < kTopD;
    uint32_t *F = reinterpret_cast<uint32_t *>(f) + (uint64_t)c * L + (cl % L);
    const uint64_t rowstep = (uint64_t)kTopD * L;
    uint32_t v[1 << HR];
#pragma unroll
    for (int i = 0; i < (1 << HR); i++)
        v[i] = valid ? F[(((uint64_t)nh << HR) | i) * rowstep] : 0u;
#pragma unroll
    for (int j = 0; j < HR; j++)
#pragma unroll
        for (int i = 0; i < (1 << HR); i++)
            if (!((i >> j) & 1)) v[i] ^= v[i + (1 << j)];
    for (int b = 0; b < LB; b++) {
#pragma unroll
        for (int i = 0; i < (1 << HR); i++) {
            const uint32_t p = __shfl_xor_sync(0xffffffffu, v[i], G << b);
            if (!((nh >> b) & 1)) v[i] ^= p;
        }
    }
    if (valid) {
#pragma unroll
        for (int i = 0; i < (1 << HR); i++) F[(((uint64_t)nh << HR) | i) * rowstep] = v[i];
    }
}

// ---------------------------------------------------------------------------
// changeRepr (Sec. 4.3): F[i] = phi(g[i mod P]), phi by 8-bit tables.  The
// periodic copy realises the fan-out of the FFT layers whose upper half is
// zero (Fig. 2).  (The product path fuses changeRepr into its first FFT pass;
// this kernel serves the stage entry point.)
__global__ void k_chrepr(const uint64_t *__restrict__ g, uint64_t pmask, uint4 *__restrict__ F,
                         uint64_t n, const DevTables *__restrict__ T) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t w = g[i & pmask];
        uint4 acc = make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int p = 0; p < 8; p++) acc = xor4(acc, __ldg(&T->chr_in[p][(w >> (8 * p)) & 255]));
        F[i] = acc;
    }
}

// changeRepr of `count` operands ahead of their first strided FFT pass:
// F[i] = phi(g[i]) for i < P (product y at g + y * strideW, F + y * strideF).
// phi is F_2-linear: word o of phi(b) is the XOR over the 14 five-bit windows
// of the block b (seven per 32-bit half) of a table entry that lane `window`
// holds in a register, one shuffle per window.  A warp takes chunks of 256
// consecutive blocks (8 per lane), one output word of phi at a time.
constexpr int kChreprK = 8;

__global__ void __launch_bounds__(256, 2) k_chrepr_stage(const uint64_t *__restrict__ g, uint64_t P,
                                                      uint64_t strideW, uint4 *__restrict__ F,
                                                      uint64_t strideF,
                                                      const DevTables *__restrict__ T) {
    pdl_release();
    __shared__ __align__(16) uint32_t tab[4 * 2 * 7 * 32];
    const uint4 *src = reinterpret_cast<const uint4 *>(&T->phi_shfl[0][0][0][0]);
    for (int i = threadIdx.x; i < 4 * 2 * 7 * 32 / 4; i += blockDim.x)
        reinterpret_cast<uint4 *>(tab)[i] = __ldg(src + i);
    __syncthreads();
    pdl_acquire();
    g += blockIdx.y * strideW;
    F += blockIdx.y * strideF;
    const int lane = threadIdx.x & 31;
    constexpr uint64_t per = 32 * kChreprK;
    const uint64_t chunks = (P + per - 1) / per;
    const uint64_t wpb = blockDim.x >> 5;
    for (uint64_t ch = blockIdx.x * wpb + (threadIdx.x >> 5); ch < chunks; ch += gridDim.x * wpb) {
        const uint64_t i0 = ch * per + lane;
        uint32_t b[kChreprK][2];
#pragma unroll
        for (int k = 0; k < kChreprK; k++) {
            const uint64_t i = i0 + 32 * k;
            const uint64_t w = i < P ? g[i] : 0;
            b[k][0] = (uint32_t)w;
            b[k][1] = (uint32_t)(w >> 32);
        }
        uint32_t r[kChreprK][4];
#pragma unroll 1
        for (int o = 0; o < 4; o++) {
            uint32_t tb[14];
#pragma unroll
            for (int qw = 0; qw < 14; qw++) tb[qw] = tab[(o * 14 + qw) * 32 + lane];
#pragma unroll
            for (int k = 0; k < kChreprK; k++) {
                uint32_t wv[2] = {b[k][0], b[k][1]};
                // keep the window shifts inside the loop over o
                asm volatile("" : "+r"(wv[0]), "+r"(wv[1]));
                uint32_t acc = 0;
#pragma unroll
                for (int q = 0; q < 2; q++) {
#pragma unroll
                    for (int w = 0; w < 6; w++) acc ^= __shfl_sync(0xffffffffu, tb[q * 7 + w], wv[q] >> (5 * w));
                    acc ^= __shfl_sync(0xffffffffu, tb[q * 7 + 6], wv[q] >> 30);
                }
#pragma unroll
                for (int oo = 0; oo < 4; oo++) r[k][oo] = o == oo ? acc : r[k][oo];
            }
        }
#pragma unroll
        for (int k = 0; k < kChreprK; k++) {
            const uint64_t i = i0 + 32 * k;
            if (i < P) F[i] = make_uint4(r[k][0], r[k][1], r[k][2], r[k][3]);
        }
    }
}

// ---------------------------------------------------------------------------
// changeRepr^-1 and InterleavedCombine (Sec. 2.1): psi(F[j]) is a polynomial
// of degree < 128 in z; z -> x and y -> x^64 add its high word into the next
// output word.  psi is F_2-linear, so word o of psi(x) is the XOR over the 28
// windows of x (seven per input word q, as in shfl_mul32) of the table entry
// psi_shfl[o][q][w][window value]; lane l holds entry l of each window's table
// in a register and a window lookup is one shuffle (the six 5-bit windows of a
// word; its 2-bit window as two masked XORs of warp-uniform entries).  A warp takes chunks of
// 32 K consecutive elements (lane l: elements l, l + 32, ...) and writes the
// 32 K - 1 output words that need only those elements; chunks overlap by one
// element.
constexpr int kCombineK = 8;
// 1: the 2-bit window of every input word through the integer pipe (24
// shuffles per output word instead of 28)
#ifndef GF2X_PSI_SHFL6
#define GF2X_PSI_SHFL6 1
#endif

__global__ void __launch_bounds__(256, 2) k_ichrepr_combine(const uint4 *__restrict__ F, uint64_t n,
                                                         uint64_t stride, OutputDesc one,
                                                         const OutputDesc *__restrict__ many,
                                                         const DevTables *__restrict__ T,
                                                         uint64_t j_begin, uint64_t j_end,
                                                         int accumulate) {
    pdl_release();
    __shared__ __align__(16) uint32_t tab[4 * 4 * 7 * 32];
    const uint4 *src = reinterpret_cast<const uint4 *>(&T->psi_shfl[0][0][0][0]);
    for (int i = threadIdx.x; i < 4 * 4 * 7 * 32 / 4; i += blockDim.x)
        reinterpret_cast<uint4 *>(tab)[i] = __ldg(src + i);
    __syncthreads();
    pdl_acquire();
    const OutputDesc d = many ? many[blockIdx.y] : one;
    F += blockIdx.y * stride;
    const int lane = threadIdx.x & 31;
    const uint64_t j_stop = j_end < d.words ? j_end : d.words;  // words [j_begin, j_stop)
    if (j_stop <= j_begin) return;
    constexpr uint64_t per = 32 * kCombineK - 1;  // output words per chunk
    const uint64_t chunks = (j_stop - j_begin + per - 1) / per;
    const uint64_t wpb = blockDim.x >> 5;
    for (uint64_t ch = blockIdx.x * wpb + (threadIdx.x >> 5); ch < chunks; ch += gridDim.x * wpb) {
        // element t = 32 k + lane of the chunk is index s0 - 1 + t; output
        // word s0 - 1 + t (t >= 1) is lo(psi(element t)) ^ hi(psi(element t - 1))
        const uint64_t s0 = j_begin + ch * per;
        uint4 e[kCombineK];
#pragma unroll
        for (int k = 0; k < kCombineK; k++) {
            const uint64_t t = 32 * k + lane;
            e[k] = make_uint4(0, 0, 0, 0);
            if (s0 + t >= 1 && s0 + t - 1 < n) e[k] = F[s0 + t - 1];
        }
        // one output word of psi at a time, so that only its 28 table
        // registers are live (the word index is kept out of register names)
        uint32_t r[kCombineK][4];
#pragma unroll 1
        for (int o = 0; o < 4; o++) {
#if GF2X_PSI_SHFL6
            // the 2-bit window of each input word on the integer pipe: its
            // entries for 2^31 and 2^30 + 2^31 are lanes 2 and 3 of table w = 6
            uint32_t tb[24], c1[4], c2[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
#pragma unroll
                for (int w = 0; w < 6; w++) tb[q * 6 + w] = tab[(o * 28 + q * 7 + w) * 32 + lane];
                const uint2 p = *reinterpret_cast<const uint2 *>(&tab[(o * 28 + q * 7 + 6) * 32 + 2]);
                c2[q] = p.x;
                c1[q] = p.x ^ p.y;
            }
#else
            uint32_t tb[28];
#pragma unroll
            for (int qw = 0; qw < 28; qw++) tb[qw] = tab[(o * 28 + qw) * 32 + lane];
#endif
#pragma unroll
            for (int k = 0; k < kCombineK; k++) {
                uint32_t wv[4] = {e[k].x, e[k].y, e[k].z, e[k].w};
                // keep the window shifts inside the loop over o (hoisting
                // them would hold 28 K values in registers)
#pragma unroll
                for (int q = 0; q < 4; q++) asm volatile("" : "+r"(wv[q]));
                uint32_t acc = 0;
#pragma unroll
                for (int q = 0; q < 4; q++) {
#if GF2X_PSI_SHFL6
#pragma unroll
                    for (int w = 0; w < 6; w++) acc ^= __shfl_sync(0xffffffffu, tb[q * 6 + w], wv[q] >> (5 * w));
                    const uint32_t m31 = (uint32_t)((int32_t)wv[q] >> 31);
                    const uint32_t m30 = (uint32_t)((int32_t)(wv[q] << 1) >> 31);
                    acc ^= (m30 & c1[q]) ^ (m31 & c2[q]);
#else
#pragma unroll
                    for (int w = 0; w < 6; w++) acc ^= __shfl_sync(0xffffffffu, tb[q * 7 + w], wv[q] >> (5 * w));
                    acc ^= __shfl_sync(0xffffffffu, tb[q * 7 + 6], wv[q] >> 30);
#endif
                }
#pragma unroll
                for (int oo = 0; oo < 4; oo++) r[k][oo] = o == oo ? acc : r[k][oo];
            }
        }
#pragma unroll
        for (int k = 0; k < kCombineK; k++) {
            uint32_t hz = __shfl_up_sync(0xffffffffu, r[k][2], 1);
            uint32_t hw = __shfl_up_sync(0xffffffffu, r[k][3], 1);
            if (k > 0) {  // lane 0: the last element of the previous row
                const uint32_t pz = __shfl_sync(0xffffffffu, r[k > 0 ? k - 1 : 0][2], 31);
                const uint32_t pw = __shfl_sync(0xffffffffu, r[k > 0 ? k - 1 : 0][3], 31);
                if (lane == 0) {
                    hz = pz;
                    hw = pw;
                }
            }
            const uint64_t t = 32 * k + lane, j = s0 + t - 1;
            if (t >= 1 && j < j_stop) {
                uint64_t v = ((uint64_t)r[k][0] | ((uint64_t)r[k][1] << 32)) ^
                             ((uint64_t)hz | ((uint64_t)hw << 32));
                if (j == d.words - 1) v &= d.mask;
                if (accumulate) v ^= d.out[j];
                d.out[j] = v;
            }
        }
    }
}

// ===========================================================================
// Host launchers.

void ensure_smem_attr(const void *func, int bytes) {
    static std::mutex mu;
    static std::set<std::tuple<int, const void *, int>> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_tuple(dev, func, bytes);
    if (done.count(key)) return;
    cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    done.insert(key);
}

unsigned num_sms() {
    static std::mutex mu;
    static std::map<int, unsigned> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    unsigned v = n > 0 ? (unsigned)n : 1u;
    cache[dev] = v;
    return v;
}

// Blocks along x for `work` items per product when `count` products share the
// launch: enough to fill the GPU a few times over, at least one.
static inline unsigned grid_for(uint64_t work, unsigned block, int count = 1) {
    uint64_t g = (work + block - 1) / block;
    uint64_t cap = std::max<uint64_t>(1, (uint64_t)num_sms() * 16 / (uint64_t)std::max(count, 1));
    g = std::min(g, std::max<uint64_t>(cap, 1));
    return (unsigned)std::max<uint64_t>(g, 1);
}

void launch_split_pad(const OperandDesc &one, const OperandDesc *many, int count, uint64_t *w,
                      uint64_t P, uint64_t stride, cudaStream_t s) {
    dim3 grid(grid_for(P, 256, count), count);
    launch_k(k_split_pad, grid, 256, 0, s, one, many, w, P, stride);
}

// Tiles of 128 KiB: 2^14 words or 2^13 128-bit elements; rows of at least
// 128 bytes of consecutive elements when the tile is strided.
template <typename T>
static int tile_log_for() {
    return sizeof(T) == 8 ? 14 : 13;
}
template <typename T>
static int min_cols_for() {
    return sizeof(T) == 8 ? 4 : 3;
}

// Number of leading forward levels that form the top VarSubs with K = 16
// (k_bcvt_top), 0 when the size has none or it is handled level by level.
static int top_levels(int m, const LevelList &fwd) {
    if (m < 17 || m > 24) return 0;
    const int h = m - 16;
    if (fwd.n < h) return 0;
    for (int q = 0; q < h; q++)
        if (fwd.v[q].logE != m - 1 - q || fwd.v[q].loge != h - 1 - q) return 0;
    return h;
}

template <typename T>
static void launch_bcvt_top(T *f, int h, int inverse, cudaStream_t s, int count, uint64_t stride) {
    constexpr int L = sizeof(T) / 4;
    const int HR = std::min(h, 6), LB = h - HR;
    const uint32_t B = top_boundary(h);
    const uint32_t nb = (B + kTopBoundaryClasses - 1) / kTopBoundaryClasses;
    const uint32_t per_cta = (uint32_t)(kTopThreads / 32) * (uint32_t)((32 >> LB) / L);
    const uint32_t ni = (kTopD - B + per_cta - 1) / per_cta;
    const dim3 grid(nb + ni, count);
    const size_t smem = (size_t)kTopBoundaryClasses * ((1u << h) + 1) * sizeof(T);
    switch (HR) {
        case 1: launch_k(k_bcvt_top<T, 1>, grid, kTopThreads, smem, s, f, h, inverse, nb, stride); break;
        case 2: launch_k(k_bcvt_top<T, 2>, grid, kTopThreads, smem, s, f, h, inverse, nb, stride); break;
        case 3: launch_k(k_bcvt_top<T, 3>, grid, kTopThreads, smem, s, f, h, inverse, nb, stride); break;
        case 4: launch_k(k_bcvt_top<T, 4>, grid, kTopThreads, smem, s, f, h, inverse, nb, stride); break;
        case 5: launch_k(k_bcvt_top<T, 5>, grid, kTopThreads, smem, s, f, h, inverse, nb, stride); break;
        default: launch_k(k_bcvt_top<T, 6>, grid, kTopThreads, smem, s, f, h, inverse, nb, stride); break;
    }
}

// Steps of a BasisCvt of 2^m coefficients in forward order (global index
// bits), from the recursion of Alg. 3: a node of 2 or 4 bits is one
// register transform; a larger node's VarSubs divisions (a, a - K) become
// runs of at most max_g(K, a) levels, followed by its two children, the low
// one (bits below K) first: the children commute, and the low one then
// shares a tile with the VarSubs runs above it.
struct OpList {
    static constexpr int kMax = 64;
    int n = 0;
    BcvtOp v[kMax];
    bool push(BcvtOp o) {
        if (n >= kMax) return false;
        v[n++] = o;
        return true;
    }
};

template <typename F>
static bool ops_rec(int m, int sc, OpList &out, const F &max_g) {
    if (m <= 1) return true;
    if (m == 2) return out.push(BcvtOp{1, (int8_t)sc, 1, 1});
    if (m == 4) return out.push(BcvtOp{2, (int8_t)sc, 2, 4});
    int K = 1;
    while (2 * K <= m - 1) K *= 2;
    for (int a = m - 1 + sc, left = m - K; left > 0;) {
        const int g = std::min(left, max_g(K, a));
        if (!out.push(BcvtOp{0, (int8_t)a, (int8_t)K, (int8_t)g})) return false;
        a -= g;
        left -= g;
    }
    return ops_rec(K, sc, out, max_g) && ops_rec(m - K, sc + K, out, max_g);
}

// The divisions (logE, loge) of a step, in forward order.
static int op_levels(const BcvtOp &o, Level *lv) {
    const int s = o.a_top;
    if (o.kind == 1) {
        lv[0] = Level{(int8_t)(s + 1), (int8_t)s};
        return 1;
    }
    if (o.kind == 2) {  // VarSubs, then the low child, then the high one
        lv[0] = Level{(int8_t)(s + 3), (int8_t)(s + 1)};
        lv[1] = Level{(int8_t)(s + 2), (int8_t)s};
        lv[2] = Level{(int8_t)(s + 1), (int8_t)s};
        lv[3] = Level{(int8_t)(s + 3), (int8_t)(s + 2)};
        return 4;
    }
    const int g = std::min<int>(o.G, 4);  // runs have at most 4 levels
    for (int i = 0; i < g; i++) lv[i] = Level{(int8_t)(o.a_top - i), (int8_t)(o.a_top - i - o.K)};
    return g;
}

static void op_range(const BcvtOp &o, int *lo, int *hi) {
    Level lv[4];
    const int k = op_levels(o, lv);
    *lo = 64;
    *hi = -1;
    for (int i = 0; i < k; i++) {
        *lo = std::min(*lo, (int)lv[i].loge);
        *hi = std::max(*hi, (int)lv[i].logE);
    }
}

template <typename T>
static void launch_bcvt_class(T *f, int m, const BcvtOp &o, int inverse, cudaStream_t s, int count,
                              uint64_t stride) {
    constexpr int L = sizeof(T) / 4;
    const uint64_t n = 1ull << m;
    const int a_low = o.a_top - o.G + 1;
    const uint64_t e_low = 1ull << (a_low - o.K);
    const uint64_t S = ((1ull << o.K) - 1) * e_low, r_int = e_low << o.G;
    const uint64_t segs = n >> (o.a_top + 1);
    const dim3 gi(grid_for(segs * (S - r_int) * L, 256, count), count);
    const dim3 gb(grid_for(segs * r_int * L, 256, count), count);
#define GF2X_CLASS_LAUNCH(GG, INV)                                                              \
    {                                                                                           \
        launch_k(k_bcvt_class<T, GG, (1 << GG) + 1, INV, false>, gi, 256, 0, s, f, (int)o.a_top, \
                 (int)o.K, n, stride);                                                          \
        launch_k(k_bcvt_class<T, GG, (1 << GG) + 1, INV, true>, gb, 256, 0, s, f, (int)o.a_top,  \
                 (int)o.K, n, stride);                                                          \
    }
    switch (o.G * 2 + (inverse ? 1 : 0)) {
        case 2: GF2X_CLASS_LAUNCH(1, false) break;
        case 3: GF2X_CLASS_LAUNCH(1, true) break;
        case 4: GF2X_CLASS_LAUNCH(2, false) break;
        case 5: GF2X_CLASS_LAUNCH(2, true) break;
        case 6: GF2X_CLASS_LAUNCH(3, false) break;
        case 7: GF2X_CLASS_LAUNCH(3, true) break;
        case 8: GF2X_CLASS_LAUNCH(4, false) break;
        default: GF2X_CLASS_LAUNCH(4, true) break;
    }
#undef GF2X_CLASS_LAUNCH
}

// Tile passes: consecutive steps whose index ranges fit one tile together
// (>= min_cols low column bits, or contiguous) share one pass; a step too wide
// for any tile runs as streaming passes, one per division.  The top VarSubs
// of sizes 2^17 .. 2^24 is one k_bcvt_top pass (first in the forward
// direction, last in the inverse).  The steps are checked against the level
// list `fwd` (the divisions of Alg. 3 in order) before anything is launched.
template <typename T>
uint64_t run_basis_cvt(T *f, int m, const LevelList &fwd, int inverse, cudaStream_t s, int count,
                       uint64_t stride, const BcvtTune &tune, const PhiOut *phi, bool *phi_done) {
    if (phi_done) *phi_done = false;
    const bool want_phi = sizeof(T) == 8 && !inverse && phi && phi->out && phi->T;
    ensure_smem_attr(reinterpret_cast<const void *>(k_bcvt_tile<T, false, false>),
                     (int)(sizeof(T) << tile_log_for<T>()));
    ensure_smem_attr(reinterpret_cast<const void *>(k_bcvt_tile<T, true, false>), 65536);
    if constexpr (sizeof(T) == 8) {
        ensure_smem_attr(reinterpret_cast<const void *>(k_bcvt_tile<T, false, true>),
                         (int)((sizeof(T) << tile_log_for<T>()) + 4 * kPhiTabWords));
        ensure_smem_attr(reinterpret_cast<const void *>(k_bcvt_tile<T, true, true>), 65536);
    }
    uint64_t launches = 0;
    const int h_top = top_levels(m, fwd);
    const int budget = std::min(tile_log_for<T>(), m), cmin = min_cols_for<T>();
    const uint64_t n = 1ull << m;
    auto fits = [&](int glo, int ghi) {
        if (ghi + 1 <= budget) return true;
        return glo >= cmin && (ghi - glo + 1) + cmin <= budget;
    };
    // runs with K >= 8 that do not fit a contiguous tile are streaming class
    // passes of up to 4 levels; other runs: 2 levels for K <= 4 (more
    // interior classes), 3 otherwise, fewer if the run would not fit a tile
    auto streamed = [&](const BcvtOp &o) { return o.kind == 0 && o.K >= 8 && o.a_top + 1 > budget; };
    auto max_g = [&](int K, int a) {
        if (K >= 8 && a + 1 > budget) return 4;
        int g = K <= 4 ? 2 : 3;
        while (g > 1 && !(a + 1 <= budget || K + g + cmin <= budget)) g--;
        return g;
    };
    OpList ops;
    bool ok = h_top ? (ops_rec(16, 0, ops, max_g) && ops_rec(m - 16, 16, ops, max_g))
                    : ops_rec(m, 0, ops, max_g);
    {  // the steps must expand to exactly the remaining divisions of fwd
        int q = h_top;
        for (int i = 0; ok && i < ops.n; i++) {
            const BcvtOp &o = ops.v[i];
            // tile runs need a compiled (K, G) variant
            ok = o.kind != 0 || streamed(o) || bcvt_tile_run_ok(o.K, o.G);
            Level lv[4];
            const int k = op_levels(o, lv);
            for (int t = 0; ok && t < k; t++, q++)
                ok = q < fwd.n && fwd.v[q].logE == lv[t].logE && fwd.v[q].loge == lv[t].loge;
        }
        ok = ok && q == fwd.n;
    }
    if (!ok) {  // not expected: apply the divisions one by one
        for (int q = 0; q < fwd.n; q++) {
            const Level &L = fwd.v[inverse ? fwd.n - 1 - q : q];
            dim3 grid(grid_for(n / 2, 256, count), count);
            launch_k(k_bcvt_level<T>, grid, 256, 0, s, f, n / 2, (int)L.logE, (int)L.loge, inverse, stride);
            launches++;
        }
        return launches;
    }
    if (h_top && !inverse) {
        launch_bcvt_top<T>(f, h_top, 0, s, count, stride);
        launches++;
    }
    auto op_at = [&](int i) -> const BcvtOp & { return ops.v[inverse ? ops.n - 1 - i : i]; };
    int i = 0;
    while (i < ops.n) {
        int glo, ghi;
        op_range(op_at(i), &glo, &ghi);
        if (streamed(op_at(i))) {
            launch_bcvt_class<T>(f, m, op_at(i), inverse, s, count, stride);
            launches += 2;
            i++;
            continue;
        }
        if (!fits(glo, ghi)) {
            Level lv[4];
            const int k = op_levels(op_at(i), lv);
            for (int t = 0; t < k; t++) {
                const Level &L = lv[inverse ? k - 1 - t : t];
                dim3 grid(grid_for(n / 2, 256, count), count);
                launch_k(k_bcvt_level<T>, grid, 256, 0, s, f, n / 2, (int)L.logE, (int)L.loge, inverse, stride);
                launches++;
            }
            i++;
            continue;
        }
        int j = i + 1;
        while (j < ops.n && j - i < LevelBatch::kMax && !streamed(op_at(j))) {
            int lo2, hi2;
            op_range(op_at(j), &lo2, &hi2);
            if (!fits(std::min(glo, lo2), std::max(ghi, hi2))) break;
            glo = std::min(glo, lo2);
            ghi = std::max(ghi, hi2);
            j++;
        }
        // the smallest tile that holds the steps (at least 2^11 elements):
        // small tiles let two CTAs share an SM and overlap their phases
        const int tmin = std::min(m, std::max(4, std::min(tune.tile_min_log, tile_log_for<T>())));
        int c, lo, w;
        if (ghi + 1 <= budget) {  // contiguous tile
            c = 0;
            lo = 0;
            w = std::min(budget, std::max(ghi + 1, tmin));
        } else {
            w = ghi - glo + 1;
            c = std::min(std::min(glo, budget - w), std::max(cmin, tmin - w));
            lo = glo;
        }
        LevelBatch lb{};
        lb.count = j - i;
        for (int q = i; q < j; q++) {
            BcvtOp o = op_at(q);
            o.a_top = (int8_t)(o.a_top - lo + c);  // tile-local index bits
            lb.op[q - i] = o;
        }
        // the last pass of a forward conversion (the top VarSubs comes first)
        // writes the changeRepr'd elements when asked to
        PhiOut po;
        if (want_phi && j == ops.n) {
            po = *phi;
            if (phi_done) *phi_done = true;
        }
        size_t smem = sizeof(T) << (c + w);
        const int small = std::max(32, std::min(512, tune.small_threads));
        int threads = std::max(32, std::min(smem > 65536 ? 512 : small, 1 << (c + w - 1)));
        if (po.out) smem += 4 * kPhiTabWords;
        dim3 grid((unsigned)(n >> (c + w)), count);
        const bool sm = threads <= 256 && smem <= 65536;
        if constexpr (sizeof(T) == 8) {
            if (po.out) {
                launch_k(sm ? k_bcvt_tile<T, true, true> : k_bcvt_tile<T, false, true>, grid,
                         threads, smem, s, f, c, lo, w, lb, inverse, stride, po);
                launches++;
                i = j;
                continue;
            }
        }
        launch_k(sm ? k_bcvt_tile<T, true, false> : k_bcvt_tile<T, false, false>, grid, threads,
                 smem, s, f, c, lo, w, lb, inverse, stride, po);
        launches++;
        i = j;
    }
    if (h_top && inverse) {
        launch_bcvt_top<T>(f, h_top, 1, s, count, stride);
        launches++;
    }
    return launches;
}

void prepare_bcvt_attributes() {
    ensure_smem_attr(reinterpret_cast<const void *>(k_bcvt_tile<uint64_t, false, false>),
                     (int)(sizeof(uint64_t) << tile_log_for<uint64_t>()));
    ensure_smem_attr(reinterpret_cast<const void *>(k_bcvt_tile<uint64_t, false, true>),
                     (int)((sizeof(uint64_t) << tile_log_for<uint64_t>()) + 4 * kPhiTabWords));
    ensure_smem_attr(reinterpret_cast<const void *>(k_bcvt_tile<uint4, false, false>),
                     (int)(sizeof(uint4) << tile_log_for<uint4>()));
    ensure_smem_attr(reinterpret_cast<const void *>(k_bcvt_tile<uint64_t, true, false>), 65536);
    ensure_smem_attr(reinterpret_cast<const void *>(k_bcvt_tile<uint64_t, true, true>), 65536);
    ensure_smem_attr(reinterpret_cast<const void *>(k_bcvt_tile<uint4, true, false>), 65536);
    num_sms();
}

template uint64_t run_basis_cvt<uint64_t>(uint64_t *, int, const LevelList &, int, cudaStream_t,
                                          int, uint64_t, const BcvtTune &, const PhiOut *, bool *);
template uint64_t run_basis_cvt<uint4>(uint4 *, int, const LevelList &, int, cudaStream_t, int,
                                       uint64_t, const BcvtTune &, const PhiOut *, bool *);

void launch_chrepr_stage(const uint64_t *g, uint64_t P, uint64_t strideW, uint4 *F,
                         uint64_t strideF, int count, const DevTables *T, cudaStream_t s) {
    // a warp takes chunks of 32 kChreprK blocks
    const uint64_t per = std::max<uint64_t>(1, (uint64_t)num_sms() * 4 / (uint64_t)std::max(count, 1));
    const uint64_t need = (P + 8 * 32 * kChreprK - 1) / (8 * 32 * kChreprK);
    dim3 grid((unsigned)std::max<uint64_t>(1, std::min<uint64_t>(need, per)), count);
    launch_k(k_chrepr_stage, grid, 256, 0, s, g, P, strideW, F, strideF, T);
}

void launch_chrepr(const uint64_t *g, uint64_t P, uint4 *F, uint64_t n, const DevTables *T,
                   cudaStream_t s) {
    k_chrepr<<<grid_for(n, 256), 256, 0, s>>>(g, P - 1, F, n, T);
}

void launch_ichrepr_combine(const uint4 *F, uint64_t n, uint64_t stride, const OutputDesc &one,
                            const OutputDesc *many, int count, uint64_t max_words,
                            const DevTables *T, cudaStream_t s, uint64_t j_begin,
                            uint64_t j_end, bool accumulate) {
    // a few resident CTAs per SM, each loading the 14 KiB of tables once; a
    // warp takes chunks of 32 kCombineK - 1 output words
    const uint64_t per = std::max<uint64_t>(1, (uint64_t)num_sms() * 4 / (uint64_t)std::max(count, 1));
    const uint64_t span = std::min(j_end, max_words) > j_begin ? std::min(j_end, max_words) - j_begin : 0;
    const uint64_t need = (span + 8 * (32 * kCombineK - 1) - 1) / (8 * (32 * kCombineK - 1));
    dim3 grid((unsigned)std::max<uint64_t>(1, std::min(need, per)), count);
    launch_k(k_ichrepr_combine, grid, 256, 0, s, F, n, stride, one, many, T, j_begin, j_end,
             accumulate ? 1 : 0);
}

__global__ void k_chunk_descs(const uint64_t *x, uint64_t xw, uint64_t x_mask, uint64_t L,
                              uint64_t C, uint64_t *out, uint64_t out_words, uint64_t out_mask,
                              uint64_t chunk_words, OperandDesc *dx, OutputDesc *dout) {
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= C) return;
    const uint64_t nw = xw - i * L < L ? xw - i * L : L;
    dx[i] = OperandDesc{x + i * L, nw, i == C - 1 ? x_mask : ~0ull};
    const uint64_t left = out_words - i * L;
    const uint64_t w = chunk_words < left ? chunk_words : left;
    const uint64_t slot = (i & 1) ? (C + 1) / 2 + i / 2 : i / 2;
    dout[slot] = OutputDesc{out + i * L, w, i * L + w == out_words ? out_mask : ~0ull};
}

void launch_chunk_descs(const uint64_t *x, uint64_t xw, uint64_t x_mask, uint64_t L, uint64_t C,
                        uint64_t *out, uint64_t out_words, uint64_t out_mask,
                        uint64_t chunk_words, OperandDesc *dx, OutputDesc *dout, cudaStream_t s) {
    k_chunk_descs<<<(unsigned)((C + 255) / 256), 256, 0, s>>>(x, xw, x_mask, L, C, out, out_words,
                                                             out_mask, chunk_words, dx, dout);
}

}  // namespace gf2x
