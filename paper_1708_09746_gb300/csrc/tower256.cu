// The F~_{2^256} form of Alg. 5 (w = 128, Sec. 4.3 and Table 2): operands in
// 128-bit blocks, each block mapped into F~_{2^256} = F~_{2^128}[x_8] /
// (x_8^2 + x_8 + v_127), the additive FFT over N2 = 2^M2 points of that field.
//
// Layout: an F~_{2^256} element e = lo + x_8 hi is kept as two F~_{2^128}
// halves in two arrays (lo at F[i], hi at F[N2 + i]).  The FFT multipliers
// s_k(alpha) lie in F~_{2^32} (alpha < 2^32), and for c in F~_{2^128}
//   c (lo + x_8 hi) = c lo + x_8 (c hi),
// so one F~_{2^256} transform is two F~_{2^128} transforms with the same
// multipliers: the FFT passes of the 64-bit form (k_fft_pass) run as a batch
// of two "products" at stride N2.  BasisCvt and its inverse only add
// coefficients, so they too act on 128-bit blocks (and on each half of the
// 256-bit coefficients) unchanged.  The new kernels here are changeRepr into
// F~_{2^256}, the generic F~_{2^256} pointmul (Karatsuba over F~_{2^128}), and
// changeRepr^-1 with the recombination of 128-bit limbs.
//
// changeRepr: a 128-bit block p(z) goes to p(r) with r = x_8 = v_128, whose
// minimal polynomial has degree 256 (x_8 is not in F~_{2^128}); chunk
// products have degree <= 254, so changeRepr^-1 (the inverse of the 256 x 256
// matrix [r^0 .. r^255]) recovers them exactly.
#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <stdexcept>
#include <tuple>
#include <vector>

#include "../../include/gf2x_gb300.h"
#include "api_internal.h"
#include "fft_pass.h"
#include "gf2x_mul.cuh"
#include "kernels.h"
#include "plan.h"

namespace gf2x {
namespace {

struct u256 {
    u128 lo, hi;
};

u128 x128(u128 a, u128 b) { return u128{a.lo ^ b.lo, a.hi ^ b.hi}; }

// x_8^2 = x_8 + v_127 (Sec. 3.2): Karatsuba over F~_{2^128}.
u256 tower_mul256(const u256 &a, const u256 &b) {
    const u128 v127{0, 1ull << 63};
    const u128 p0 = tower_mul128(a.lo, b.lo);
    const u128 p1 = tower_mul128(a.hi, b.hi);
    const u128 p2 = tower_mul128(x128(a.lo, a.hi), x128(b.lo, b.hi));
    return u256{x128(p0, tower_mul128(p1, v127)), x128(p2, p0)};
}

bool bit256(const u256 &x, int j) {
    const uint64_t w = j < 64 ? x.lo.lo : j < 128 ? x.lo.hi : j < 192 ? x.hi.lo : x.hi.hi;
    return (w >> (j & 63)) & 1;
}

void flip256(u256 &x, int j) {
    uint64_t *w = j < 64 ? &x.lo.lo : j < 128 ? &x.lo.hi : j < 192 ? &x.hi.lo : &x.hi.hi;
    *w ^= 1ull << (j & 63);
}

u256 x256(const u256 &a, const u256 &b) { return u256{x128(a.lo, b.lo), x128(a.hi, b.hi)}; }

uint4 as_uint4(const u128 &x) {
    return make_uint4((uint32_t)x.lo, (uint32_t)(x.lo >> 32), (uint32_t)x.hi, (uint32_t)(x.hi >> 32));
}

// Byte tables of changeRepr (16 byte positions of a 128-bit block, both halves
// of the image) and of changeRepr^-1 (32 byte positions of a 256-bit element,
// the low and the high 128 bits of the polynomial kept apart).
struct Host256 {
    std::vector<uint4> chr;     // [16][256][2]: (lo, hi) of phi(v << 8p)
    std::vector<uint4> psi_lo;  // [32][256]: bits 0..127 of psi(v << 8p)
    std::vector<uint4> psi_hi;  // [32][256]: bits 128..255 of psi(v << 8p)
};

const Host256 &host256() {
    static std::once_flag once;
    static Host256 H;
    std::call_once(once, [] {
        u256 rp[256];
        rp[0] = u256{u128{1, 0}, u128{0, 0}};
        const u256 r{u128{0, 0}, u128{1, 0}};
        for (int i = 1; i < 256; i++) rp[i] = tower_mul256(rp[i - 1], r);
        H.chr.assign(16 * 256 * 2, make_uint4(0, 0, 0, 0));
        for (int p = 0; p < 16; p++)
            for (int v = 0; v < 256; v++) {
                u256 acc{};
                for (int j = 0; j < 8; j++)
                    if ((v >> j) & 1) acc = x256(acc, rp[8 * p + j]);
                H.chr[(p * 256 + v) * 2] = as_uint4(acc.lo);
                H.chr[(p * 256 + v) * 2 + 1] = as_uint4(acc.hi);
            }
        // inverse of the matrix with columns r^i: rows (element, polynomial)
        // kept so that element = sum over the polynomial's bits of r^i;
        // Gauss-Jordan reduces the elements to the unit vectors v_j
        u256 elem[256], poly[256];
        for (int i = 0; i < 256; i++) {
            elem[i] = rp[i];
            poly[i] = u256{};
            flip256(poly[i], i);
        }
        for (int j = 0; j < 256; j++) {
            int piv = -1;
            for (int i = j; i < 256; i++)
                if (bit256(elem[i], j)) {
                    piv = i;
                    break;
                }
            if (piv < 0) throw std::runtime_error("changeRepr (w = 128) matrix is singular");
            std::swap(elem[j], elem[piv]);
            std::swap(poly[j], poly[piv]);
            for (int i = 0; i < 256; i++)
                if (i != j && bit256(elem[i], j)) {
                    elem[i] = x256(elem[i], elem[j]);
                    poly[i] = x256(poly[i], poly[j]);
                }
        }
        // now poly[j] = psi(v_j)
        H.psi_lo.assign(32 * 256, make_uint4(0, 0, 0, 0));
        H.psi_hi.assign(32 * 256, make_uint4(0, 0, 0, 0));
        for (int p = 0; p < 32; p++)
            for (int v = 0; v < 256; v++) {
                u256 acc{};
                for (int j = 0; j < 8; j++)
                    if ((v >> j) & 1) acc = x256(acc, poly[8 * p + j]);
                H.psi_lo[p * 256 + v] = as_uint4(acc.lo);
                H.psi_hi[p * 256 + v] = as_uint4(acc.hi);
            }
    });
    return H;
}

struct Dev256 {
    uint4 *chr = nullptr, *psi_lo = nullptr, *psi_hi = nullptr;
};

std::mutex g_dev_mu;
std::map<int, Dev256> g_dev;

int dev256(const Dev256 **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return GF2X_ECUDA;
    }
    const Host256 &H = host256();
    std::lock_guard<std::mutex> lk(g_dev_mu);
    Dev256 &d = g_dev[dev];
    if (!d.chr) {
        const size_t bc = H.chr.size() * 16, bp = H.psi_lo.size() * 16;
        Dev256 t;
        if (cudaMalloc(&t.chr, bc) != cudaSuccess || cudaMalloc(&t.psi_lo, bp) != cudaSuccess ||
            cudaMalloc(&t.psi_hi, bp) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(t.chr);
            cudaFree(t.psi_lo);
            cudaFree(t.psi_hi);
            return GF2X_ENOMEM;
        }
        if (cudaMemcpy(t.chr, H.chr.data(), bc, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(t.psi_lo, H.psi_lo.data(), bp, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(t.psi_hi, H.psi_hi.data(), bp, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(t.chr);
            cudaFree(t.psi_lo);
            cudaFree(t.psi_hi);
            return GF2X_ECUDA;
        }
        d = t;
    }
    *out = &d;
    return GF2X_OK;
}

// ---------------------------------------------------------------------------
// Kernels.

// XOR over the 16 bytes of v of tab[(pos0 + p) * stride + byte p] (method of
// four Russians over the bytes of a 128-bit value, tables in global memory).
__device__ __forceinline__ uint4 byte_tab_sum(const uint4 *__restrict__ tab, uint4 v, int pos0,
                                              int stride, int sub) {
    uint4 acc = make_uint4(0, 0, 0, 0);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; q++)
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const uint32_t byte = (w[q] >> (8 * b)) & 255u;
            acc = xor4(acc, __ldg(tab + ((size_t)(pos0 + 4 * q + b) * 256 + byte) * stride + sub));
        }
    return acc;
}

// changeRepr of the P blocks (uint4 each) into both halves of the N2-point
// transform input, with the fan-out of the layers above log2 P: element i
// (i < N2) is phi(block i mod P).  Block j is converted once and written
// N2 / P times.
__global__ void __launch_bounds__(256) k_chrepr256(const uint4 *__restrict__ blocks, uint64_t P,
                                                   uint4 *F, uint64_t N2,
                                                   const uint4 *__restrict__ chr) {
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < P;
         j += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 b = blocks[j];
        const uint4 lo = byte_tab_sum(chr, b, 0, 2, 0), hi = byte_tab_sum(chr, b, 0, 2, 1);
        for (uint64_t i = j; i < N2; i += P) {
            F[i] = lo;
            F[N2 + i] = hi;
        }
    }
}

// pointmul in F~_{2^256}: (a0 + x_8 a1)(b0 + x_8 b1) with x_8^2 = x_8 + v_127:
//   lo = a0 b0 + (a1 b1) v_127,  hi = (a0 + a1)(b0 + b1) + a0 b0,
// the F~_{2^128} products by the F~_{2^8} product table in shared memory.
// The result replaces B.
__global__ void __launch_bounds__(256) k_pointmul256(const uint4 *__restrict__ A, uint4 *B,
                                                     uint64_t N2,
                                                     const DevTables *__restrict__ T) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint8_t *mt = smem;
    uint32_t *lane_tab = reinterpret_cast<uint32_t *>(smem + 65536);
    const uint4 *src = reinterpret_cast<const uint4 *>(T->mul8);
    for (int i = threadIdx.x; i < 4096; i += blockDim.x) reinterpret_cast<uint4 *>(mt)[i] = __ldg(src + i);
    const uint4 *lsrc = reinterpret_cast<const uint4 *>(&T->low_lane[0][0]);
    for (int i = threadIdx.x; i < (int)(kLaneTabBytes / 16); i += blockDim.x)
        reinterpret_cast<uint4 *>(lane_tab)[i] = __ldg(lsrc + i);
    __syncthreads();
    const MtRef M = mt_ref(mt, lane_tab);
    const uint4 v127 = make_uint4(0, 0, 0, 0x80000000u);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N2;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 a0 = A[i], a1 = A[N2 + i], b0 = B[i], b1 = B[N2 + i];
        const uint4 p0 = mt_gmul128(M, a0, b0);
        const uint4 p1 = mt_gmul128(M, a1, b1);
        const uint4 p2 = mt_gmul128(M, xor4(a0, a1), xor4(b0, b1));
        B[i] = xor4(p0, mt_gmul128(M, p1, v127));
        B[N2 + i] = xor4(p2, p0);
    }
}

// changeRepr^-1 and the recombination of 128-bit limbs: output block j (words
// 2j, 2j+1) = bits 0..127 of psi(e_j) XOR bits 128..255 of psi(e_{j-1}), e_j =
// F[j] + x_8 F[N2 + j] (zero for j >= N2).  Words past out_words are not
// written; the last one is masked by top_mask.
__global__ void __launch_bounds__(256) k_ichrepr256_combine(const uint4 *__restrict__ F, uint64_t N2,
                                                            uint64_t *out, uint64_t out_words,
                                                            uint64_t top_mask,
                                                            const uint4 *__restrict__ psi_lo,
                                                            const uint4 *__restrict__ psi_hi) {
    const uint64_t nblk = (out_words + 1) / 2;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < nblk;
         j += (uint64_t)gridDim.x * blockDim.x) {
        uint4 acc = make_uint4(0, 0, 0, 0);
        if (j < N2) {
            acc = xor4(byte_tab_sum(psi_lo, F[j], 0, 1, 0), byte_tab_sum(psi_lo, F[N2 + j], 16, 1, 0));
        }
        if (j >= 1 && j - 1 < N2) {
            acc = xor4(acc, byte_tab_sum(psi_hi, F[j - 1], 0, 1, 0));
            acc = xor4(acc, byte_tab_sum(psi_hi, F[N2 + j - 1], 16, 1, 0));
        }
        uint64_t w0 = (uint64_t)acc.x | ((uint64_t)acc.y << 32);
        uint64_t w1 = (uint64_t)acc.z | ((uint64_t)acc.w << 32);
        if (2 * j == out_words - 1) w0 &= top_mask;
        if (2 * j + 1 == out_words - 1) w1 &= top_mask;
        out[2 * j] = w0;
        if (2 * j + 1 < out_words) out[2 * j + 1] = w1;
    }
}

unsigned grid_for(uint64_t items, unsigned threads) {
    const uint64_t want = (items + threads - 1) / threads;
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)num_sms() * 8));
}

// ---------------------------------------------------------------------------
// Plan and stage order.

struct Plan256 {
    uint64_t na_bits, nb_bits, na_w, nb_w, out_words, total_bits;
    int M2, pa_log, pb_log;
    uint64_t N2, Pa, Pb;  // points; padded 128-bit blocks of a and b
    LevelList lv_a, lv_b, lv_c;
    PassList fft_a, fft_b, ifft;
    // workspace (bytes): FA | FB (2 x 16 N2 each: lo halves, then hi halves)
    // | WA (16 Pa) | WB (16 Pb)
    size_t off_fa, off_fb, off_wa, off_wb, ws_bytes;
};

constexpr int kMaxLogN2 = 27;

int plan256_init(Plan256 *p, uint64_t na_bits, uint64_t nb_bits) {
    p->na_bits = na_bits;
    p->nb_bits = nb_bits;
    p->na_w = words_of(na_bits);
    p->nb_w = words_of(nb_bits);
    p->total_bits = na_bits + nb_bits - 1;
    p->out_words = words_of(p->total_bits);
    const uint64_t na_b = (na_bits + 127) / 128, nb_b = (nb_bits + 127) / 128;
    // N2: the smallest power of two >= the product's number of 128-bit blocks
    p->M2 = log2_ceil(std::max<uint64_t>(2, na_b + nb_b - 1));
    if (p->M2 > kMaxLogN2) return GF2X_EINVAL;
    p->N2 = 1ull << p->M2;
    p->pa_log = log2_ceil(na_b);
    p->pb_log = log2_ceil(nb_b);
    p->Pa = 1ull << p->pa_log;
    p->Pb = 1ull << p->pb_log;
    p->lv_a = basis_cvt_levels(p->pa_log);
    p->lv_b = basis_cvt_levels(p->pb_log);
    p->lv_c = basis_cvt_levels(p->M2);
    if (plan_fft_forward(p->M2, p->pa_log, p->fft_a) || plan_fft_forward(p->M2, p->pb_log, p->fft_b) ||
        plan_fft_inverse(p->M2, p->ifft))
        return GF2X_ECUDA;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    p->off_fa = 0;
    p->off_fb = up(32 * p->N2);
    p->off_wa = up(p->off_fb + 32 * p->N2);
    p->off_wb = up(p->off_wa + 16 * p->Pa);
    p->ws_bytes = up(p->off_wb + 16 * p->Pb);
    return GF2X_OK;
}

// Alg. 5 with w = 128 on stream s.
int run256(const Plan256 *p, const uint64_t *a, const uint64_t *b, uint64_t *out, void *ws,
           cudaStream_t s, int *st, StageHook *hook) {
    const DevTables *T;
    const Dev256 *D;
    int rc = api::tables(&T);
    if (rc || (rc = dev256(&D))) return rc;
    char *base = static_cast<char *>(ws);
    uint4 *FA = reinterpret_cast<uint4 *>(base + p->off_fa);
    uint4 *FB = reinterpret_cast<uint4 *>(base + p->off_fb);
    uint64_t *WA = reinterpret_cast<uint64_t *>(base + p->off_wa);
    uint64_t *WB = reinterpret_cast<uint64_t *>(base + p->off_wb);
    auto begin = [&](int stage) {
        if (hook) hook->begin(stage);
    };
    auto end = [&](uint64_t n) {
        if (hook) hook->end(n);
    };
    const OperandDesc one[2] = {{a, p->na_w, mask_of_bits(p->na_bits)},
                                {b, p->nb_w, mask_of_bits(p->nb_bits)}};
    uint64_t *W[2] = {WA, WB};
    uint4 *F[2] = {FA, FB};
    const uint64_t P[2] = {p->Pa, p->Pb};
    const int lg[2] = {p->pa_log, p->pb_log};
    const LevelList *lv[2] = {&p->lv_a, &p->lv_b};
    const PassList *fw[2] = {&p->fft_a, &p->fft_b};
    for (int x = 0; x < 2; x++) {
        // Split into 2 P 64-bit words = P 128-bit blocks, BasisCvt on the
        // blocks, changeRepr into both halves of the transform input (with
        // the fan-out of the layers above log2 P), the forward layers below
        begin(ST_SPLIT);
        launch_split_pad(one[x], nullptr, 1, W[x], 2 * P[x], 0, s);
        end(1);
        begin(ST_BCVT);
        end(run_basis_cvt<uint4>(reinterpret_cast<uint4 *>(W[x]), lg[x], *lv[x], 0, s));
        begin(ST_CHREPR);
        k_chrepr256<<<grid_for(P[x], 256), 256, 0, s>>>(reinterpret_cast<const uint4 *>(W[x]), P[x],
                                                       F[x], p->N2, D->chr);
        end(1);
        begin(x == 0 ? ST_FFT_A : ST_FFT_B);
        for (int i = 0; i < fw[x]->n; i++)
            launch_fft_pass(fw[x]->v[i], p->M2, F[x], nullptr, P[x], nullptr, T, st, s, 2, p->N2, 0);
        end(fw[x]->n);
    }
    begin(ST_FUSED);
    const int pm_smem = 65536 + (int)kLaneTabBytes;
    ensure_smem_attr(reinterpret_cast<const void *>(k_pointmul256), pm_smem);
    k_pointmul256<<<std::min<unsigned>(grid_for(p->N2, 256), 2 * num_sms()), 256, pm_smem, s>>>(
        FA, FB, p->N2, T);
    end(1);
    begin(ST_IFFT);
    for (int i = 0; i < p->ifft.n; i++)
        launch_fft_pass(p->ifft.v[i], p->M2, FB, nullptr, 0, nullptr, T, st, s, 2, p->N2, 0);
    end(p->ifft.n);
    begin(ST_IBCVT);
    end(run_basis_cvt<uint4>(FB, p->M2, p->lv_c, 1, s, 2, p->N2));
    begin(ST_OUT);
    k_ichrepr256_combine<<<grid_for((p->out_words + 1) / 2, 256), 256, 0, s>>>(
        FB, p->N2, out, p->out_words, mask_of_bits(p->total_bits), D->psi_lo, D->psi_hi);
    end(1);
    return cudaGetLastError() == cudaSuccess ? GF2X_OK : GF2X_ECUDA;
}

std::mutex g_plan_mu;
std::map<std::tuple<int, uint64_t, uint64_t>, std::shared_ptr<Plan256>> g_plans;

int plan256_for(uint64_t na_bits, uint64_t nb_bits, std::shared_ptr<Plan256> *out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return GF2X_ECUDA;
    }
    const auto key = std::make_tuple(dev, na_bits, nb_bits);
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto it = g_plans.find(key);
    if (it != g_plans.end()) {
        *out = it->second;
        return GF2X_OK;
    }
    auto p = std::make_shared<Plan256>();
    int rc = plan256_init(p.get(), na_bits, nb_bits);
    if (rc) return rc;
    if (g_plans.size() >= 64) g_plans.clear();
    g_plans[key] = p;
    *out = p;
    return GF2X_OK;
}

int mul256_on_stream(const uint64_t *a, uint64_t na_bits, const uint64_t *b, uint64_t nb_bits,
                     uint64_t *out, cudaStream_t s, int *st) {
    std::shared_ptr<Plan256> p;
    int rc = plan256_for(na_bits, nb_bits, &p);
    if (rc) return rc;
    void *ws = nullptr;
    if ((rc = api::ws_alloc(&ws, p->ws_bytes, s))) return rc;
    std::unique_ptr<StageHook> tm(api::new_timer(s));
    rc = run256(p.get(), a, b, out, ws, s, st, tm.get());
    api::ws_free(ws, s);
    return rc;
}

int check256(const uint64_t *a, uint64_t na_bits, const uint64_t *b, uint64_t nb_bits,
             const uint64_t *out) {
    if (na_bits > (1ull << 33) || nb_bits > (1ull << 33)) return GF2X_EINVAL;
    return api::check_product_args(a, na_bits, b, nb_bits, out);
}

}  // namespace
}  // namespace gf2x

using namespace gf2x;

extern "C" {

int gf2x_mul_tower256_async(const uint64_t *a, uint64_t na_bits, const uint64_t *b,
                            uint64_t nb_bits, uint64_t *out, gf2x_stream_t stream) {
    try {
        int rc = check256(a, na_bits, b, nb_bits, out);
        if (rc) return rc;
        if (!na_bits || !nb_bits) return GF2X_OK;
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        int *st = api::stream_status(s);
        if (!st) return GF2X_ECUDA;
        return mul256_on_stream(a, na_bits, b, nb_bits, out, s, st);
    } catch (const std::bad_alloc &) {
        return GF2X_ENOMEM;
    } catch (...) {
        return GF2X_ECUDA;
    }
}

int gf2x_mul_tower256(const uint64_t *a, uint64_t na_bits, const uint64_t *b, uint64_t nb_bits,
                      uint64_t *out) {
    try {
        int rc = check256(a, na_bits, b, nb_bits, out);
        if (rc) return rc;
        if (!na_bits || !nb_bits) return GF2X_OK;
        int *st = nullptr;
        if ((rc = api::take_status(&st))) return rc;
        if (cudaMemsetAsync(st, 0, sizeof(int), 0) != cudaSuccess) {
            cudaGetLastError();
            api::give_status(st);
            return GF2X_ECUDA;
        }
        rc = mul256_on_stream(a, na_bits, b, nb_bits, out, nullptr, st);
        if (cudaStreamSynchronize(0) != cudaSuccess) {
            cudaGetLastError();
            rc = GF2X_ECUDA;
        }
        const int ds = api::read_status(st);
        api::give_status(st);
        return rc ? rc : ds;
    } catch (const std::bad_alloc &) {
        return GF2X_ENOMEM;
    } catch (...) {
        return GF2X_ECUDA;
    }
}

uint64_t gf2x_tower256_fft_points(uint64_t na_bits, uint64_t nb_bits) {
    if (!na_bits || !nb_bits) return 0;
    const uint64_t na_b = (na_bits + 127) / 128, nb_b = (nb_bits + 127) / 128;
    return 1ull << log2_ceil(std::max<uint64_t>(2, na_b + nb_b - 1));
}

int gf2x_stage_chrepr256(const void *blocks, uint64_t P, void *F, uint64_t N2,
                         gf2x_stream_t stream) {
    if (!P || (P & (P - 1)) || N2 < P || (N2 & (N2 - 1))) return GF2X_EINVAL;
    try {
        const Dev256 *D;
        int rc = dev256(&D);
        if (rc) return rc;
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        k_chrepr256<<<grid_for(P, 256), 256, 0, s>>>(static_cast<const uint4 *>(blocks), P,
                                                     static_cast<uint4 *>(F), N2, D->chr);
        return cudaGetLastError() == cudaSuccess ? GF2X_OK : GF2X_ECUDA;
    } catch (...) {
        return GF2X_ECUDA;
    }
}

int gf2x_stage_pointmul256(const void *A, void *B, uint64_t N2, gf2x_stream_t stream) {
    if (!N2) return GF2X_OK;
    try {
        const DevTables *T;
        int rc = api::tables(&T);
        if (rc) return rc;
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        const int pm_smem = 65536 + (int)kLaneTabBytes;
        ensure_smem_attr(reinterpret_cast<const void *>(k_pointmul256), pm_smem);
        k_pointmul256<<<std::min<unsigned>(grid_for(N2, 256), 2 * num_sms()), 256, pm_smem, s>>>(
            static_cast<const uint4 *>(A), static_cast<uint4 *>(B), N2, T);
        return cudaGetLastError() == cudaSuccess ? GF2X_OK : GF2X_ECUDA;
    } catch (...) {
        return GF2X_ECUDA;
    }
}

int gf2x_stage_ichrepr256_combine(const void *F, uint64_t N2, uint64_t *out, uint64_t out_words,
                                  uint64_t total_bits, gf2x_stream_t stream) {
    if (!out_words) return GF2X_OK;
    try {
        const Dev256 *D;
        int rc = dev256(&D);
        if (rc) return rc;
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        k_ichrepr256_combine<<<grid_for((out_words + 1) / 2, 256), 256, 0, s>>>(
            static_cast<const uint4 *>(F), N2, out, out_words, mask_of_bits(total_bits), D->psi_lo,
            D->psi_hi);
        return cudaGetLastError() == cudaSuccess ? GF2X_OK : GF2X_ECUDA;
    } catch (...) {
        return GF2X_ECUDA;
    }
}

}  // extern "C"
