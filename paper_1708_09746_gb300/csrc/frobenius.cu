// The Frobenius-partition form of the product (Appendix C): no Kronecker
// segmentation.  A polynomial a(x) in GF(2)[x] of degree < 128 n (n = 2^m) is
// evaluated, its coefficients taken as elements of GF(2^128), at the n points
// alpha + V_m, alpha = beta_{m+64}; this map E is a bijection onto GF(2^128)^n
// (Proposition C.1) and multiplicative, so c = a b (degree < 128 n) is
// E^-1(E(a) E(b)) with half as many points as the 64-bit Kronecker form.
//
// E is a truncated additive FFT (Sec. C.2/C.3), computed here as:
//  1. BasisCvt of the one-bit coefficients (Alg. 3 on bits: every division by
//     x^E + x^e is a shifted XOR of bit ranges, see below);
//  2. the encoding -- the first seven FFT layers of which only the left branch
//     is kept -- element i = sum_j g[i + j n] w_j over the 128 bits at stride
//     n, w_j = prod_{bits l of j} s_{m+l}(alpha) = prod beta_{64-l} (fixed
//     constants: s_k(phi_beta(j)) = phi_beta(j >> k) in a Cantor basis), by
//     byte tables of the 128 x 128 matrix [w_0 .. w_127];
//  3. an m-layer LCH FFT at alpha + V_m in the polynomial basis of GF(2^128)
//     (poly_field.cu: the multiplier of layer k for block b is
//     beta_{m+64-k} + phi_beta(2b), a general field element).
// The product's values are multiplied pointwise, and E^-1 runs the inverse
// FFT, the inverse encoding (byte tables of the inverse matrix, the 128 bits
// scattered back to stride n) and the inverse BasisCvt of 128 n bits.
//
// BasisCvt on bits.  A division by x^E + x^e (E, e powers of two) of every
// segment of 2E coefficients is two steps, each a XOR of a bit range shifted
// down by D = E - e within the segment: step 1 adds bits [2E-e, 2E) to
// [E, E+e), step 2 adds bits [E, 2E-e) to [e, E) (Alg. 2; the inverse undoes
// step 2, then step 1).  Each step reads bits it does not write, so a
// streaming pass updates words in place.  Levels whose segments fit a tile of
// 2^18 bits run together in shared memory (two-phase: every word's new value
// is computed before any is stored); larger levels stream from HBM, one
// launch per step.
#include <algorithm>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <stdexcept>
#include <tuple>
#include <vector>

#include "../../include/gf2x_gb300.h"
#include "api_internal.h"
#include "kernels.h"
#include "plan.h"
#include "poly_field.h"

namespace gf2x {
namespace {

using poly::H128;

// ---- Host: the encoding matrix and its inverse ---------------------------------

struct FrobHost {
    std::vector<uint4> enc;  // [16][256]: encoding of the column (v << 8p)
    std::vector<uint4> dec;  // [16][256]: column whose encoding is (v << 8p)
};

H128 as_h(const uint4 &x) {
    return H128{(uint64_t)x.x | ((uint64_t)x.y << 32), (uint64_t)x.z | ((uint64_t)x.w << 32)};
}
uint4 as_u4(const H128 &x) {
    return make_uint4((uint32_t)x.lo, (uint32_t)(x.lo >> 32), (uint32_t)x.hi, (uint32_t)(x.hi >> 32));
}
bool hb(const H128 &x, int j) { return ((j < 64 ? x.lo : x.hi) >> (j & 63)) & 1; }
void hf(H128 &x, int j) { (j < 64 ? x.lo : x.hi) ^= 1ull << (j & 63); }
H128 hx(H128 a, H128 b) { return H128{a.lo ^ b.lo, a.hi ^ b.hi}; }

const FrobHost &frob_host() {
    static std::once_flag once;
    static FrobHost F;
    std::call_once(once, [] {
        const std::vector<uint4> &beta = poly::cantor_host();
        H128 w[128];
        for (int j = 0; j < 128; j++) {
            H128 x{1, 0};
            for (int l = 0; l < 7; l++)
                if ((j >> l) & 1) x = poly::hmul(x, as_h(beta[64 - l]));
            w[j] = x;
        }
        // inverse: rows (element, column) with element = sum over the column's
        // bits of w_j, reduced to unit elements by Gauss-Jordan
        H128 el[128], col[128];
        for (int j = 0; j < 128; j++) {
            el[j] = w[j];
            col[j] = H128{0, 0};
            hf(col[j], j);
        }
        for (int t = 0; t < 128; t++) {
            int piv = -1;
            for (int i = t; i < 128; i++)
                if (hb(el[i], t)) {
                    piv = i;
                    break;
                }
            if (piv < 0) throw std::runtime_error("encoding matrix is singular");
            std::swap(el[t], el[piv]);
            std::swap(col[t], col[piv]);
            for (int i = 0; i < 128; i++)
                if (i != t && hb(el[i], t)) {
                    el[i] = hx(el[i], el[t]);
                    col[i] = hx(col[i], col[t]);
                }
        }
        // col[t] is the column whose encoding is the unit element z^t
        F.enc.assign(16 * 256, make_uint4(0, 0, 0, 0));
        F.dec.assign(16 * 256, make_uint4(0, 0, 0, 0));
        for (int p = 0; p < 16; p++)
            for (int v = 0; v < 256; v++) {
                H128 a{0, 0}, b{0, 0};
                for (int q = 0; q < 8; q++)
                    if ((v >> q) & 1) {
                        a = hx(a, w[8 * p + q]);
                        b = hx(b, col[8 * p + q]);
                    }
                F.enc[p * 256 + v] = as_u4(a);
                F.dec[p * 256 + v] = as_u4(b);
            }
    });
    return F;
}

struct FrobDev {
    uint4 *enc = nullptr, *dec = nullptr;
};
std::mutex g_fdev_mu;
std::map<int, FrobDev> g_fdev;

int frob_dev(const FrobDev **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return GF2X_ECUDA;
    }
    const FrobHost &H = frob_host();
    std::lock_guard<std::mutex> lk(g_fdev_mu);
    FrobDev &d = g_fdev[dev];
    if (!d.enc) {
        FrobDev t;
        const size_t b = H.enc.size() * 16;
        if (cudaMalloc(&t.enc, b) != cudaSuccess || cudaMalloc(&t.dec, b) != cudaSuccess ||
            cudaMemcpy(t.enc, H.enc.data(), b, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(t.dec, H.dec.data(), b, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(t.enc);
            cudaFree(t.dec);
            return GF2X_ENOMEM;
        }
        d = t;
    }
    *out = &d;
    return GF2X_OK;
}

// ---- BasisCvt on bits -------------------------------------------------------------

// Bits [lo, hi) of every segment of 2^(logE+1) bits, restricted to word w.
__device__ __forceinline__ uint64_t seg_mask(uint64_t w, int logE, uint64_t lo, uint64_t hi) {
    const uint64_t P = 2ull << logE;
    if (P >= 64) {
        const uint64_t off = (64 * w) & (P - 1);
        const uint64_t a = lo > off ? lo : off, b = hi < off + 64 ? hi : off + 64;
        if (a >= b) return 0;
        const uint64_t n = b - a;
        return (n == 64 ? ~0ull : ((1ull << n) - 1)) << (a - off);
    }
    uint64_t m = ((1ull << (hi - lo)) - 1) << lo;  // one period of P < 64 bits
    for (uint64_t s = P; s < 64; s <<= 1) m |= m << s;
    return m;
}

// 64 bits of f starting at bit position pos (bits past nwords read as 0).
__device__ __forceinline__ uint64_t bits64(const uint64_t *f, uint64_t nwords, uint64_t pos) {
    const uint64_t w = pos >> 6;
    const int sh = (int)(pos & 63);
    const uint64_t lo = w < nwords ? f[w] : 0;
    if (!sh) return lo;
    const uint64_t hi = w + 1 < nwords ? f[w + 1] : 0;
    return (lo >> sh) | (hi << (64 - sh));
}

// The new value of word w after step `step` (1 or 2) of the division by
// x^E + x^e of every 2E-bit segment.
__device__ __forceinline__ uint64_t step_word(const uint64_t *f, uint64_t nwords, uint64_t w,
                                              int logE, int loge, int step) {
    const uint64_t E = 1ull << logE, e = 1ull << loge;
    const uint64_t lo = step == 1 ? E : e, hi = step == 1 ? E + e : E;
    const uint64_t m = seg_mask(w, logE, lo, hi);
    if (!m) return f[w];
    return f[w] ^ (bits64(f, nwords, 64 * w + (E - e)) & m);
}

// One step of one level with segments of at least 128 bits, in place (the
// step reads only bits it does not write).  Only the words holding the step's
// destination bits are visited: per segment of 2E bits, words [0, E/64) for
// step 2 (destination [e, E)) and the words of [E, E + e) for step 1.
__global__ void __launch_bounds__(256) k_bitcvt_step(uint64_t *f, uint64_t nwords, int logE, int loge,
                                                     int step) {
    const uint64_t E = 1ull << logE, e = 1ull << loge, D = E - e;
    const uint64_t seg_words = (2 * E) >> 6;
    const uint64_t first = step == 1 ? (E >> 6) : 0;
    const uint64_t count = step == 1 ? ((E + e + 63) >> 6) - (E >> 6) : (E >> 6);
    const uint64_t lo = step == 1 ? E : e, hi = step == 1 ? E + e : E;
    const uint64_t total = (nwords / seg_words) * count;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t seg = t / count, k = t - seg * count;
        const uint64_t w = seg * seg_words + first + k;
        const uint64_t m = seg_mask(w, logE, lo, hi);
        if (m) f[w] ^= bits64(f, nwords, 64 * w + D) & m;
    }
}

struct BitLevels {
    static constexpr int kMax = 64;
    int n;
    int8_t logE[kMax], loge[kMax];
};

constexpr int kBitTileWordsLog = 12;  // 4096 words = 2^18 bits = 32 KiB
constexpr int kBitTileThreads = 512;

// A run of levels whose segments fit the tile, applied to tiles of
// 2^tile_log words in shared memory; inverse: each level's step 2, then 1.
__global__ void __launch_bounds__(kBitTileThreads) k_bitcvt_tile(uint64_t *f, uint64_t nwords,
                                                                 int tile_log, BitLevels L,
                                                                 int inverse) {
    __shared__ uint64_t s[1 << kBitTileWordsLog];
    const uint64_t tw = 1ull << tile_log;
    constexpr int kPer = (1 << kBitTileWordsLog) / kBitTileThreads;
    for (uint64_t t = blockIdx.x; t * tw < nwords; t += gridDim.x) {
        uint64_t *g = f + t * tw;
        __syncthreads();
        for (uint64_t q = threadIdx.x; q < tw; q += blockDim.x) s[q] = g[q];
        __syncthreads();
        for (int i = 0; i < L.n; i++)
            for (int h = 0; h < 2; h++) {
                const int step = inverse ? 2 - h : 1 + h;
                uint64_t nv[kPer];
#pragma unroll
                for (int k = 0; k < kPer; k++) {
                    const uint64_t q = threadIdx.x + (uint64_t)k * blockDim.x;
                    if (q < tw) nv[k] = step_word(s, tw, q, L.logE[i], L.loge[i], step);
                }
                __syncthreads();
#pragma unroll
                for (int k = 0; k < kPer; k++) {
                    const uint64_t q = threadIdx.x + (uint64_t)k * blockDim.x;
                    if (q < tw) s[q] = nv[k];
                }
                __syncthreads();
            }
        for (uint64_t q = threadIdx.x; q < tw; q += blockDim.x) g[q] = s[q];
    }
}

unsigned grid_of(uint64_t items, unsigned threads, unsigned per_sm = 8) {
    const uint64_t want = (items + threads - 1) / threads;
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)num_sms() * per_sm));
}

// BasisCvt (inverse = 0) or iBasisCvt of 2^L bits at f: the level list of
// Alg. 3 in bit units, runs of tile-sized levels in one tile pass each, the
// others one streaming launch per step.  Returns the launches.
uint64_t run_bit_cvt(uint64_t *f, int L, int inverse, cudaStream_t s) {
    const LevelList lv = basis_cvt_levels(L);
    const uint64_t nwords = L >= 6 ? (1ull << (L - 6)) : 1;
    const int tile_log = std::min<int>(kBitTileWordsLog, L >= 6 ? L - 6 : 0);
    const int tile_bits_log = tile_log + 6;
    uint64_t launches = 0;
    BitLevels run;
    run.n = 0;
    auto flush = [&]() {
        if (!run.n) return;
        const uint64_t tiles = nwords >> tile_log;
        k_bitcvt_tile<<<(unsigned)std::min<uint64_t>(tiles, (uint64_t)num_sms() * 4), kBitTileThreads,
                        0, s>>>(f, nwords, tile_log, run, inverse);
        launches++;
        run.n = 0;
    };
    for (int q = 0; q < lv.n; q++) {
        const Level &l = lv.v[inverse ? lv.n - 1 - q : q];
        if (l.logE + 1 <= tile_bits_log) {
            if (run.n == BitLevels::kMax) flush();
            run.logE[run.n] = l.logE;
            run.loge[run.n] = l.loge;
            run.n++;
            continue;
        }
        flush();
        for (int h = 0; h < 2; h++) {
            const int step = inverse ? 2 - h : 1 + h;
            const uint64_t E = 1ull << l.logE, e = 1ull << l.loge;
            const uint64_t per_seg = step == 1 ? ((E + e + 63) >> 6) - (E >> 6) : (E >> 6);
            const uint64_t items = (nwords / ((2 * E) >> 6)) * per_seg;
            k_bitcvt_step<<<grid_of(items, 256), 256, 0, s>>>(f, nwords, l.logE, l.loge, step);
            launches++;
        }
    }
    flush();
    return launches;
}

// ---- Encoding and its inverse ---------------------------------------------------

__device__ __forceinline__ uint4 x4(uint4 a, uint4 b) {
    return make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w);
}

// XOR over the 16 bytes of v of tab[p * 256 + byte p].
__device__ __forceinline__ uint4 tab16(const uint4 *__restrict__ tab, const uint32_t (&v)[4]) {
    uint4 acc = make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int q = 0; q < 4; q++)
#pragma unroll
        for (int b = 0; b < 4; b++)
            acc = x4(acc, __ldg(tab + (4 * q + b) * 256 + ((v[q] >> (8 * b)) & 255u)));
    return acc;
}

// 32 x 32 bit transpose across a warp: lane l holds row l, and afterwards
// holds column l (bit j = bit l of row j).  Stage s swaps the off-diagonal
// blocks of size s between lanes l and l ^ s.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, unsigned lane) {
    const uint32_t m[5] = {0x55555555u, 0x33333333u, 0x0F0F0F0Fu, 0x00FF00FFu, 0x0000FFFFu};
#pragma unroll
    for (int k = 0; k < 5; k++) {
        const int sh = 1 << k;
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, sh);
        x = (lane & sh) ? ((x & ~m[k]) | ((y & ~m[k]) >> sh)) : ((x & m[k]) | ((y & m[k]) << sh));
    }
    return x;
}

// Element i (i < n) = sum_j g[i + j n] w_j over the bits of the 2^L-bit array
// g (bits at positions >= nbits are zero).  With n >= 32 (a multiple of 32)
// the bits of the warp's 32 consecutive elements in row j are one aligned
// 32-bit word: lane l loads rows l, l+32, l+64, l+96 and a warp transpose
// hands every lane its element's 128-bit column.
__global__ void __launch_bounds__(256) k_encode(const uint64_t *__restrict__ g, uint64_t nbits,
                                                uint64_t n, uint4 *E, const uint4 *__restrict__ enc) {
    const uint64_t rows = std::min<uint64_t>(128, (nbits + n - 1) / n);
    if (n >= 32) {
        const uint32_t *g32 = reinterpret_cast<const uint32_t *>(g);
        const unsigned lane = threadIdx.x & 31;
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
             i += (uint64_t)gridDim.x * blockDim.x) {
            const uint64_t i0 = i - lane;
            uint32_t v[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const uint64_t j = 32 * q + lane;
                const uint64_t pos = j * n + i0;
                const uint32_t row = (j < rows && pos < nbits) ? __ldg(g32 + (pos >> 5)) : 0u;
                v[q] = warp_transpose32(row, lane);
            }
            E[i] = tab16(enc, v);
        }
        return;
    }
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t v[4] = {0, 0, 0, 0};
        for (uint64_t j = 0; j < rows; j++) {
            const uint64_t pos = j * n + i;
            if (pos < nbits) v[j >> 5] |= (uint32_t)((__ldg(g + (pos >> 6)) >> (pos & 63)) & 1u) << (j & 31);
        }
        E[i] = tab16(enc, v);
    }
}

// The inverse: the 128-bit column of element i scattered to bits i + j n of
// the 128 n-bit array c.  With n >= 32 the 32 lanes of a warp hold 32
// consecutive i, so bit j of the warp's columns is one aligned 32-bit word
// (a ballot); smaller n set single bits with atomic ORs into a zeroed c.
__global__ void __launch_bounds__(256) k_decode(const uint4 *__restrict__ E, uint64_t n, uint64_t *c,
                                                const uint4 *__restrict__ dec) {
    const uint64_t total = (n + 31) & ~31ull;
    const unsigned lane = threadIdx.x & 31;
    uint32_t *c32 = reinterpret_cast<uint32_t *>(c);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint4 col = make_uint4(0, 0, 0, 0);
        if (i < n) {
            const uint4 e = E[i];
            const uint32_t v[4] = {e.x, e.y, e.z, e.w};
            col = tab16(dec, v);
        }
        const uint32_t cw[4] = {col.x, col.y, col.z, col.w};
        if (n >= 32) {
            // the warp transpose turns the 32 columns back into rows: lane l
            // stores rows l, l+32, l+64, l+96 of the warp's 32 elements
            const uint64_t i0 = i - lane;
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const uint32_t row = warp_transpose32(cw[q], lane);
                c32[((uint64_t)(32 * q + lane) * n + i0) >> 5] = row;
            }
        } else if (i < n) {
            for (int j = 0; j < 128; j++)
                if ((cw[j >> 5] >> (j & 31)) & 1u) {
                    const uint64_t pos = (uint64_t)j * n + i;
                    atomicOr(reinterpret_cast<unsigned long long *>(c + (pos >> 6)),
                             (unsigned long long)(1ull << (pos & 63)));
                }
        }
    }
}

// The first out_words words of the product's bit array, the last one masked.
__global__ void __launch_bounds__(256) k_copy_out(const uint64_t *__restrict__ c, uint64_t *out,
                                                  uint64_t out_words, uint64_t top_mask) {
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < out_words;
         w += (uint64_t)gridDim.x * blockDim.x)
        out[w] = w == out_words - 1 ? (c[w] & top_mask) : c[w];
}

// ---- Plan and stage order --------------------------------------------------------

struct PlanFrob {
    uint64_t na_bits, nb_bits, na_w, nb_w, out_words, total_bits;
    int m, la, lb;      // n = 2^m points; operands padded to 2^la, 2^lb bits
    uint64_t n, wa, wb;  // words of the padded operands
    // workspace: A bits | B bits | EA (16 n) | EB (16 n) | C bits (2 n words)
    size_t off_a, off_b, off_ea, off_eb, off_c, ws_bytes;
};

constexpr int kMaxFrobLog = 27;  // n <= 2^27 points (products below 2^34 bits)

int plan_frob_init(PlanFrob *p, uint64_t na_bits, uint64_t nb_bits) {
    p->na_bits = na_bits;
    p->nb_bits = nb_bits;
    p->na_w = words_of(na_bits);
    p->nb_w = words_of(nb_bits);
    p->total_bits = na_bits + nb_bits - 1;
    p->out_words = words_of(p->total_bits);
    p->m = log2_ceil((p->total_bits + 127) / 128);
    if (p->m > kMaxFrobLog) return GF2X_EINVAL;
    p->n = 1ull << p->m;
    p->la = log2_ceil(na_bits);
    p->lb = log2_ceil(nb_bits);
    p->wa = p->la >= 6 ? 1ull << (p->la - 6) : 1;
    p->wb = p->lb >= 6 ? 1ull << (p->lb - 6) : 1;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    p->off_a = 0;
    p->off_b = up(8 * p->wa);
    p->off_ea = up(p->off_b + 8 * p->wb);
    p->off_eb = up(p->off_ea + 16 * p->n);
    p->off_c = up(p->off_eb + 16 * p->n);
    p->ws_bytes = up(p->off_c + 16 * p->n);
    return GF2X_OK;
}

int run_frob(const PlanFrob *p, const uint64_t *a, const uint64_t *b, uint64_t *out, void *ws,
             cudaStream_t s, StageHook *hook) {
    const uint4 *beta;
    const FrobDev *D;
    int rc = poly::cantor_dev(&beta);
    if (rc || (rc = frob_dev(&D))) return rc;
    char *base = static_cast<char *>(ws);
    uint64_t *A = reinterpret_cast<uint64_t *>(base + p->off_a);
    uint64_t *B = reinterpret_cast<uint64_t *>(base + p->off_b);
    uint4 *EA = reinterpret_cast<uint4 *>(base + p->off_ea);
    uint4 *EB = reinterpret_cast<uint4 *>(base + p->off_eb);
    uint64_t *C = reinterpret_cast<uint64_t *>(base + p->off_c);
    auto begin = [&](int stage) {
        if (hook) hook->begin(stage);
    };
    auto end = [&](uint64_t k) {
        if (hook) hook->end(k);
    };
    const int alpha_bit = p->m + 64;
    const OperandDesc one[2] = {{a, p->na_w, mask_of_bits(p->na_bits)},
                                {b, p->nb_w, mask_of_bits(p->nb_bits)}};
    uint64_t *X[2] = {A, B};
    uint4 *EX[2] = {EA, EB};
    const uint64_t W[2] = {p->wa, p->wb};
    const int lg[2] = {p->la, p->lb};
    for (int x = 0; x < 2; x++) {
        begin(ST_SPLIT);
        launch_split_pad(one[x], nullptr, 1, X[x], W[x], 0, s);
        end(1);
        begin(ST_BCVT);
        end(run_bit_cvt(X[x], lg[x], 0, s));
        begin(ST_CHREPR);
        k_encode<<<grid_of(p->n, 256), 256, 0, s>>>(X[x], 1ull << lg[x], p->n, EX[x], D->enc);
        end(1);
        begin(x == 0 ? ST_FFT_A : ST_FFT_B);
        end(poly::launch_fft(EX[x], p->m, p->m, 0, 1, 0, alpha_bit, beta, s));
    }
    begin(ST_FUSED);
    poly::launch_gfmul(EA, EB, p->n, s);
    end(1);
    begin(ST_IFFT);
    end(poly::launch_fft(EB, p->m, p->m, 1, 1, 0, alpha_bit, beta, s));
    begin(ST_IBCVT);
    if (p->n < 32) cudaMemsetAsync(C, 0, 16 * p->n, s);
    k_decode<<<grid_of((p->n + 31) & ~31ull, 256), 256, 0, s>>>(EB, p->n, C, D->dec);
    const uint64_t launches = run_bit_cvt(C, p->m + 7, 1, s);
    end(1 + launches + (p->n < 32 ? 1 : 0));
    begin(ST_OUT);
    k_copy_out<<<grid_of(p->out_words, 256), 256, 0, s>>>(C, out, p->out_words,
                                                         mask_of_bits(p->total_bits));
    end(1);
    return cudaGetLastError() == cudaSuccess ? GF2X_OK : GF2X_ECUDA;
}

std::mutex g_fplan_mu;
std::map<std::tuple<int, uint64_t, uint64_t>, std::shared_ptr<PlanFrob>> g_fplans;

int plan_frob_for(uint64_t na_bits, uint64_t nb_bits, std::shared_ptr<PlanFrob> *out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return GF2X_ECUDA;
    }
    const auto key = std::make_tuple(dev, na_bits, nb_bits);
    std::lock_guard<std::mutex> lk(g_fplan_mu);
    auto it = g_fplans.find(key);
    if (it != g_fplans.end()) {
        *out = it->second;
        return GF2X_OK;
    }
    auto p = std::make_shared<PlanFrob>();
    int rc = plan_frob_init(p.get(), na_bits, nb_bits);
    if (rc) return rc;
    if (g_fplans.size() >= 64) g_fplans.clear();
    g_fplans[key] = p;
    *out = p;
    return GF2X_OK;
}

int mul_frob_on_stream(const uint64_t *a, uint64_t na_bits, const uint64_t *b, uint64_t nb_bits,
                       uint64_t *out, cudaStream_t s) {
    std::shared_ptr<PlanFrob> p;
    int rc = plan_frob_for(na_bits, nb_bits, &p);
    if (rc) return rc;
    void *ws = nullptr;
    if ((rc = api::ws_alloc(&ws, p->ws_bytes, s))) return rc;
    std::unique_ptr<StageHook> tm(api::new_timer(s));
    rc = run_frob(p.get(), a, b, out, ws, s, tm.get());
    api::ws_free(ws, s);
    return rc;
}

}  // namespace
}  // namespace gf2x

using namespace gf2x;

extern "C" {

int gf2x_frobenius_points(uint64_t na_bits, uint64_t nb_bits) {
    if (!na_bits || !nb_bits) return -1;
    return log2_ceil((na_bits + nb_bits - 1 + 127) / 128);
}

int gf2x_mul_frobenius_async(const uint64_t *a, uint64_t na_bits, const uint64_t *b,
                             uint64_t nb_bits, uint64_t *out, gf2x_stream_t stream) {
    try {
        if (na_bits > (1ull << 33) || nb_bits > (1ull << 33)) return GF2X_EINVAL;
        int rc = api::check_product_args(a, na_bits, b, nb_bits, out);
        if (rc) return rc;
        if (!na_bits || !nb_bits) return GF2X_OK;
        return mul_frob_on_stream(a, na_bits, b, nb_bits, out, reinterpret_cast<cudaStream_t>(stream));
    } catch (const std::bad_alloc &) {
        return GF2X_ENOMEM;
    } catch (...) {
        return GF2X_ECUDA;
    }
}

int gf2x_mul_frobenius(const uint64_t *a, uint64_t na_bits, const uint64_t *b, uint64_t nb_bits,
                       uint64_t *out) {
    int rc = gf2x_mul_frobenius_async(a, na_bits, b, nb_bits, out, nullptr);
    if (rc) return rc;
    if (cudaStreamSynchronize(0) != cudaSuccess) {
        cudaGetLastError();
        return GF2X_ECUDA;
    }
    return GF2X_OK;
}

int gf2x_stage_bit_basis_cvt(uint64_t *f, int log_bits, int inverse, gf2x_stream_t stream) {
    if (log_bits < 0 || log_bits > 35) return GF2X_EINVAL;
    try {
        run_bit_cvt(f, log_bits, inverse ? 1 : 0, reinterpret_cast<cudaStream_t>(stream));
        return cudaGetLastError() == cudaSuccess ? GF2X_OK : GF2X_ECUDA;
    } catch (...) {
        return GF2X_ECUDA;
    }
}

int gf2x_stage_frobenius_encode(const uint64_t *g, int log_bits, int m, void *E, int decode,
                                gf2x_stream_t stream) {
    if (m < 0 || m > kMaxFrobLog || log_bits < 0 || log_bits > m + 7) return GF2X_EINVAL;
    try {
        const FrobDev *D;
        int rc = frob_dev(&D);
        if (rc) return rc;
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        const uint64_t n = 1ull << m;
        if (!decode) {
            k_encode<<<grid_of(n, 256), 256, 0, s>>>(g, 1ull << log_bits, n, static_cast<uint4 *>(E),
                                                    D->enc);
        } else {
            uint64_t *c = const_cast<uint64_t *>(g);
            if (n < 32) cudaMemsetAsync(c, 0, 16 * n, s);
            k_decode<<<grid_of((n + 31) & ~31ull, 256), 256, 0, s>>>(static_cast<const uint4 *>(E), n,
                                                                    c, D->dec);
        }
        return cudaGetLastError() == cudaSuccess ? GF2X_OK : GF2X_ECUDA;
    } catch (...) {
        return GF2X_ECUDA;
    }
}

int gf2x_stage_fft_frobenius(void *F, int m, int inverse, gf2x_stream_t stream) {
    if (m < 0 || m > kMaxFrobLog) return GF2X_EINVAL;
    try {
        const uint4 *beta;
        int rc = poly::cantor_dev(&beta);
        if (rc) return rc;
        poly::launch_fft(static_cast<uint4 *>(F), m, m, inverse ? 1 : 0, 1, 0, m + 64, beta,
                         reinterpret_cast<cudaStream_t>(stream));
        return cudaGetLastError() == cudaSuccess ? GF2X_OK : GF2X_ECUDA;
    } catch (...) {
        return GF2X_ECUDA;
    }
}

}  // extern "C"
