// GF(2^128) in the polynomial basis of the AES-GCM field, GF(2)[z] /
// (z^128 + z^7 + z^2 + z + 1) (Sec. 2.3), with a Cantor basis (beta_i) of it
// (Sec. 2.4): the field arithmetic and the LCH FFT passes shared by the simple
// form (Alg. 4) and the Frobenius-partition form (Appendix C).
//
// * The Cantor basis: beta_0 = 1 and beta_i the root of y^2 + y = beta_{i-1}
//   whose coefficient at z^0 is 0 (the two roots differ by 1).  In a Cantor
//   basis s_k(phi_beta(j)) = phi_beta(j >> k), so the multiplier of layer k for
//   the butterfly block b (points phi_beta(b 2^(k+1)) + V_{k+1}) is
//   phi_beta(2 b), the XOR of beta_i over the set bits of 2 b: Cantor
//   coordinates switched to the polynomial basis by a linear map (Alg. 4).
//   With an offset alpha = beta_a the multiplier gains s_k(alpha) = beta_{a-k}.
// * GB300 has no carry-less multiply instruction: a 32x32-bit carry-less
//   product is four interleaved integer products per output class (operand
//   bits spaced four apart, so no column sum reaches the next class), 64 and
//   128 bits follow by Karatsuba, and the 256-bit product is reduced with
//   z^128 = z^7 + z^2 + z + 1 (two foldings).  Every product is this general
//   multiply; the butterfly multipliers are general field elements.
#include <algorithm>
#include <map>
#include <mutex>
#include <stdexcept>
#include <vector>

#include "../../include/gf2x_gb300.h"
#include "clmul.cuh"
#include "kernels.h"
#include "poly_field.h"

namespace gf2x {
namespace poly {
namespace {

bool hbit(const H128 &x, int j) { return ((j < 64 ? x.lo : x.hi) >> (j & 63)) & 1; }
void hflip(H128 &x, int j) { (j < 64 ? x.lo : x.hi) ^= 1ull << (j & 63); }

}  // namespace


// Product modulo z^128 + z^7 + z^2 + z + 1, shift-and-add with reduction at
// every step (z * x = x << 1, plus 0x87 when bit 127 falls out).
H128 hmul(H128 a, H128 b) {
    H128 r{0, 0};
    for (int i = 0; i < 128; i++) {
        if (hbit(b, i)) {
            r.lo ^= a.lo;
            r.hi ^= a.hi;
        }
        const bool top = (a.hi >> 63) & 1;
        a.hi = (a.hi << 1) | (a.lo >> 63);
        a.lo <<= 1;
        if (top) a.lo ^= 0x87;
    }
    return r;
}

namespace {

// y with y^2 + y = c and coefficient 0 at z^0 (the map y -> y^2 + y is
// GF(2)-linear with kernel {0, 1}): Gauss-Jordan on the columns L(z^j).
H128 solve_y2_plus_y(H128 c) {
    H128 col[128];
    for (int j = 0; j < 128; j++) {
        H128 e{0, 0};
        hflip(e, j);
        col[j] = hmul(e, e);
        col[j].lo ^= e.lo;
        col[j].hi ^= e.hi;
    }
    // rows[i] = (coefficients of unknown j in equation i, right-hand side)
    std::vector<H128> rows(128);
    std::vector<int> rhs(128);
    for (int i = 0; i < 128; i++) {
        H128 r{0, 0};
        for (int j = 0; j < 128; j++)
            if (hbit(col[j], i)) hflip(r, j);
        rows[i] = r;
        rhs[i] = hbit(c, i);
    }
    std::vector<int> pivot_row(128, -1);
    int rank = 0;
    for (int j = 127; j >= 1; j--) {  // unknown 0 stays free (set to 0)
        int piv = -1;
        for (int i = rank; i < 128; i++)
            if (hbit(rows[i], j)) {
                piv = i;
                break;
            }
        if (piv < 0) continue;
        std::swap(rows[rank], rows[piv]);
        std::swap(rhs[rank], rhs[piv]);
        for (int i = 0; i < 128; i++)
            if (i != rank && hbit(rows[i], j)) {
                rows[i].lo ^= rows[rank].lo;
                rows[i].hi ^= rows[rank].hi;
                rhs[i] ^= rhs[rank];
            }
        pivot_row[j] = rank++;
    }
    // the rows past the rank are zero (column 0 of the map is zero)
    for (int i = rank; i < 128; i++)
        if (rhs[i]) throw std::runtime_error("y^2 + y = c has no root");
    H128 y{0, 0};
    for (int j = 1; j < 128; j++)
        if (pivot_row[j] >= 0 && rhs[pivot_row[j]]) hflip(y, j);
    return y;
}

}  // namespace

// beta_0 .. beta_127 as uint4.
const std::vector<uint4> &cantor_host() {
    static std::once_flag once;
    static std::vector<uint4> B;
    std::call_once(once, [] {
        H128 b{1, 0};
        for (int i = 0; i < 128; i++) {
            if (i) b = solve_y2_plus_y(b);
            B.push_back(make_uint4((uint32_t)b.lo, (uint32_t)(b.lo >> 32), (uint32_t)b.hi,
                                   (uint32_t)(b.hi >> 32)));
        }
    });
    return B;
}

std::mutex g_beta_mu;
std::map<int, uint4 *> g_beta;

int cantor_dev(const uint4 **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return GF2X_ECUDA;
    }
    const std::vector<uint4> &B = cantor_host();
    std::lock_guard<std::mutex> lk(g_beta_mu);
    uint4 *&d = g_beta[dev];
    if (!d) {
        uint4 *t = nullptr;
        if (cudaMalloc(&t, B.size() * 16) != cudaSuccess) {
            cudaGetLastError();
            return GF2X_ENOMEM;
        }
        if (cudaMemcpy(t, B.data(), B.size() * 16, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(t);
            return GF2X_ECUDA;
        }
        d = t;
    }
    *out = d;
    return GF2X_OK;
}

namespace {

// ---- Device: the general GF(2^128) product ---------------------------------

// a * b in GF(2)[z]/(z^128 + z^7 + z^2 + z + 1): 128 x 128 by Karatsuba over
// 64-bit halves, then the high 128 bits H folded twice with z^128 = z^7 + z^2
// + z + 1 (H (1 + z + z^2 + z^7), whose at most 7 overflowing bits are folded
// the same way).
__device__ __forceinline__ uint4 gf128_mul(uint4 a, uint4 b) {
    const uint64_t A0 = (uint64_t)a.x | ((uint64_t)a.y << 32), A1 = (uint64_t)a.z | ((uint64_t)a.w << 32);
    const uint64_t B0 = (uint64_t)b.x | ((uint64_t)b.y << 32), B1 = (uint64_t)b.z | ((uint64_t)b.w << 32);
    uint64_t p0l, p0h, p2l, p2h, pml, pmh;
    clmul64(A0, B0, p0l, p0h);
    clmul64(A1, B1, p2l, p2h);
    clmul64(A0 ^ A1, B0 ^ B1, pml, pmh);
    pml ^= p0l ^ p2l;
    pmh ^= p0h ^ p2h;
    const uint64_t r0 = p0l, r1 = p0h ^ pml, r2 = p2l ^ pmh, r3 = p2h;
    // H = (r2, r3): H z^128 = H + H z + H z^2 + H z^7
    const uint64_t t0 = r2 ^ (r2 << 1) ^ (r2 << 2) ^ (r2 << 7);
    const uint64_t t1 = r3 ^ ((r3 << 1) | (r2 >> 63)) ^ ((r3 << 2) | (r2 >> 62)) ^ ((r3 << 7) | (r2 >> 57));
    const uint64_t x = (r3 >> 63) ^ (r3 >> 62) ^ (r3 >> 57);
    const uint64_t u = x ^ (x << 1) ^ (x << 2) ^ (x << 7);
    const uint64_t lo = r0 ^ t0 ^ u, hi = r1 ^ t1;
    return make_uint4((uint32_t)lo, (uint32_t)(lo >> 32), (uint32_t)hi, (uint32_t)(hi >> 32));
}

__device__ __forceinline__ uint4 xor4s(uint4 a, uint4 b) {
    return make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w);
}

// phi_beta(j): XOR of beta_i over the set bits i of j.
__device__ __forceinline__ uint4 phi_beta(const uint4 *bt, uint32_t j) {
    uint4 r = make_uint4(0, 0, 0, 0);
    while (j) {
        const int i = __ffs(j) - 1;
        r = xor4s(r, bt[i]);
        j &= j - 1;
    }
    return r;
}

// One pass of g layers k_lo .. k_lo+g-1 of FFT_LCH (inverse = 0) or its
// inverse at the points alpha + phi_beta(i), alpha = beta_{alpha_bit} (none if
// alpha_bit < 0; s_k(alpha) = beta_{alpha_bit - k} then adds to every
// multiplier of layer k), on tiles of 2^g rows (index bits k_lo ..) by 2^c consecutive
// elements, for `count` transforms at F + y * strideF of 2^M points each.
// The tile is loaded into shared memory, its layers applied one after another
// (one butterfly per thread per step), and stored back.
__global__ void __launch_bounds__(256) k_fft_poly(uint4 *F, int M, int k_lo, int g, int c,
                                                  int inverse, int count, uint64_t strideF,
                                                  int alpha_bit, const uint4 *__restrict__ beta) {
    extern __shared__ __align__(16) uint4 sm[];
    __shared__ uint4 bt[128];
    for (int i = threadIdx.x; i < 128; i += blockDim.x) bt[i] = beta[i];
    const uint32_t tile = 1u << (g + c), cmask = (1u << c) - 1;
    const int tiles_log = M - g - c, mid_bits = k_lo - c;
    const uint64_t ntiles = (uint64_t)count << tiles_log;
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint64_t y = t >> tiles_log, tt = t & ((1ull << tiles_log) - 1);
        const uint64_t base = ((tt >> mid_bits) << (k_lo + g)) | ((tt & ((1ull << mid_bits) - 1)) << c);
        uint4 *Fy = F + y * strideF;
        auto gidx = [&](uint32_t q) { return base | ((uint64_t)(q >> c) << k_lo) | (q & cmask); };
        __syncthreads();  // bt loaded; the previous tile is stored
        for (uint32_t q = threadIdx.x; q < tile; q += blockDim.x) sm[q] = Fy[gidx(q)];
        __syncthreads();
        for (int step = 0; step < g; step++) {
            const int r = inverse ? step : g - 1 - step;
            const int k = k_lo + r, sh = r + c;
            for (uint32_t w = threadIdx.x; w < tile / 2; w += blockDim.x) {
                const uint32_t qu = ((w >> sh) << (sh + 1)) | (w & ((1u << sh) - 1));
                const uint32_t qv = qu | (1u << sh);
                uint4 cm = phi_beta(bt, (uint32_t)(gidx(qu) >> k) & ~1u);
                if (alpha_bit >= 0) cm = xor4s(cm, bt[alpha_bit - k]);
                uint4 u = sm[qu], v = sm[qv];
                if (!inverse) {
                    u = xor4s(u, gf128_mul(cm, v));
                    v = xor4s(v, u);
                } else {
                    v = xor4s(v, u);
                    u = xor4s(u, gf128_mul(cm, v));
                }
                sm[qu] = u;
                sm[qv] = v;
            }
            __syncthreads();
        }
        for (uint32_t q = threadIdx.x; q < tile; q += blockDim.x) Fy[gidx(q)] = sm[q];
    }
}

__global__ void __launch_bounds__(256) k_gfmul_poly(const uint4 *__restrict__ A, uint4 *B,
                                                      uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        B[i] = gf128_mul(A[i], B[i]);
}

constexpr int kSimpleTileLog = 11;  // 2048 elements, 32 KiB of shared memory
constexpr int kSimpleDepth = 6;     // layers per strided pass (c = 11 - g >= 5)

// The passes of layers [0, L) of a transform of 2^M points: forward from the
// top down (strided passes, then the bottom pass), inverse from the bottom up.
}  // namespace

int launch_fft(uint4 *F, int M, int L, int inverse, int count, uint64_t strideF, int alpha_bit,
               const uint4 *beta, cudaStream_t s) {
    if (L <= 0) return 0;
    struct P3 {
        int k_lo, g, c;
    } ps[8];
    int n = 0;
    const int gb = std::min(L, kSimpleTileLog);
    ps[n++] = P3{0, gb, 0};
    const int rest = L - gb;
    if (rest > 0) {
        const int np = (rest + kSimpleDepth - 1) / kSimpleDepth;
        int k = gb;
        for (int i = 0; i < np; i++) {
            const int g = rest / np + (i < rest % np ? 1 : 0);
            ps[n++] = P3{k, g, kSimpleTileLog - g};
            k += g;
        }
    }
    for (int q = 0; q < n; q++) {
        const P3 &p = inverse ? ps[q] : ps[n - 1 - q];
        const uint64_t tiles = ((uint64_t)count << (M - p.g - p.c));
        const size_t smem = (size_t)16 << (p.g + p.c);
        k_fft_poly<<<(unsigned)std::min<uint64_t>(tiles, (uint64_t)num_sms() * 4), 256, smem, s>>>(
            F, M, p.k_lo, p.g, p.c, inverse, count, strideF, alpha_bit, beta);
    }
    return n;
}

void launch_gfmul(const uint4 *A, uint4 *B, uint64_t n, cudaStream_t s) {
    if (!n) return;
    const uint64_t want = (n + 255) / 256;
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)num_sms() * 8));
    k_gfmul_poly<<<grid, 256, 0, s>>>(A, B, n);
}

}  // namespace poly
}  // namespace gf2x
