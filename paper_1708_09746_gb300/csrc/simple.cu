// The simple form of the product (Alg. 4, Sec. 3.1): the working field stays
// in the polynomial basis of GF(2^128) = GF(2)[z] / (z^128 + z^7 + z^2 + z + 1)
// (the AES-GCM field of Sec. 2.3), the LCH FFT evaluates at the points
// phi_beta(i) of a Cantor basis (beta_i) of that field, and every product --
// in the butterflies and in pointmul -- is a general GF(2^128) product
// (poly_field.cu: field, Cantor basis, emulated carry-less multiply, FFT
// passes).
//
// * A 64-bit block p(z) is already a field element of degree < 64 and two
//   blocks multiply to degree <= 126 without reduction, so the block embeds
//   as itself (no changeRepr) and the interpolated coefficients are the
//   chunk products themselves (no changeRepr^-1).
// * BasisCvt and iBasisCvt are the kernels of the tower form: the novelpoly
//   basis polynomials have coefficients in GF(2) and are the same for every
//   Cantor basis.
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

// ---- Kernels ------------------------------------------------------------------

// The P blocks into the N-point transform input with the fan-out of the layers
// above log2 P: element i = (block i mod P, 0).
__global__ void __launch_bounds__(256) k_embed_simple(const uint64_t *__restrict__ w, uint64_t P,
                                                      uint4 *F, uint64_t N) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t v = w[i & (P - 1)];
        F[i] = make_uint4((uint32_t)v, (uint32_t)(v >> 32), 0u, 0u);
    }
}

// The recombination of Sec. 2.1 on the interpolated chunk products (already
// polynomials of degree <= 126): word j = low half of c_j XOR high half of
// c_{j-1}; words past out_words are not written, the last one is masked.
__global__ void __launch_bounds__(256) k_combine_simple(const uint4 *__restrict__ F, uint64_t N,
                                                        uint64_t *out, uint64_t out_words,
                                                        uint64_t top_mask) {
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < out_words;
         j += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t v = 0;
        if (j < N) {
            const uint4 e = F[j];
            v = (uint64_t)e.x | ((uint64_t)e.y << 32);
        }
        if (j >= 1 && j - 1 < N) {
            const uint4 e = F[j - 1];
            v ^= (uint64_t)e.z | ((uint64_t)e.w << 32);
        }
        if (j == out_words - 1) v &= top_mask;
        out[j] = v;
    }
}

unsigned grid_simple(uint64_t items, unsigned threads, unsigned per_sm = 8) {
    const uint64_t want = (items + threads - 1) / threads;
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)num_sms() * per_sm));
}

// ---- Plan and stage order -----------------------------------------------------

struct PlanSimple {
    uint64_t na_bits, nb_bits, na_w, nb_w, out_words, total_bits;
    int M, pa_log, pb_log;
    uint64_t N, Pa, Pb;
    LevelList lv_a, lv_b, lv_c;
    size_t off_fa, off_fb, off_wa, off_wb, ws_bytes;  // FA | FB (16 N) | WA (8 Pa) | WB (8 Pb)
};

int plan_simple_init(PlanSimple *p, uint64_t na_bits, uint64_t nb_bits) {
    p->na_bits = na_bits;
    p->nb_bits = nb_bits;
    p->na_w = words_of(na_bits);
    p->nb_w = words_of(nb_bits);
    p->total_bits = na_bits + nb_bits - 1;
    p->out_words = words_of(p->total_bits);
    p->M = log2_ceil(std::max<uint64_t>(2, p->na_w + p->nb_w - 1));
    if (p->M > kMaxLogN) return GF2X_EINVAL;
    p->N = 1ull << p->M;
    p->pa_log = log2_ceil(p->na_w);
    p->pb_log = log2_ceil(p->nb_w);
    p->Pa = 1ull << p->pa_log;
    p->Pb = 1ull << p->pb_log;
    p->lv_a = basis_cvt_levels(p->pa_log);
    p->lv_b = basis_cvt_levels(p->pb_log);
    p->lv_c = basis_cvt_levels(p->M);
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    p->off_fa = 0;
    p->off_fb = up(16 * p->N);
    p->off_wa = up(p->off_fb + 16 * p->N);
    p->off_wb = up(p->off_wa + 8 * p->Pa);
    p->ws_bytes = up(p->off_wb + 8 * p->Pb);
    return GF2X_OK;
}

int run_simple(const PlanSimple *p, const uint64_t *a, const uint64_t *b, uint64_t *out, void *ws,
               cudaStream_t s, StageHook *hook) {
    const uint4 *beta;
    int rc = poly::cantor_dev(&beta);
    if (rc) return rc;
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
    for (int x = 0; x < 2; x++) {
        begin(ST_SPLIT);
        launch_split_pad(one[x], nullptr, 1, W[x], P[x], 0, s);
        end(1);
        begin(ST_BCVT);
        end(run_basis_cvt<uint64_t>(W[x], lg[x], *lv[x], 0, s));
        begin(ST_CHREPR);
        k_embed_simple<<<grid_simple(p->N, 256), 256, 0, s>>>(W[x], P[x], F[x], p->N);
        end(1);
        begin(x == 0 ? ST_FFT_A : ST_FFT_B);
        end(poly::launch_fft(F[x], p->M, lg[x], 0, 1, 0, -1, beta, s));
    }
    begin(ST_FUSED);
    poly::launch_gfmul(FA, FB, p->N, s);
    end(1);
    begin(ST_IFFT);
    end(poly::launch_fft(FB, p->M, p->M, 1, 1, 0, -1, beta, s));
    begin(ST_IBCVT);
    end(run_basis_cvt<uint4>(FB, p->M, p->lv_c, 1, s));
    begin(ST_OUT);
    k_combine_simple<<<grid_simple(p->out_words, 256), 256, 0, s>>>(FB, p->N, out, p->out_words,
                                                                   mask_of_bits(p->total_bits));
    end(1);
    return cudaGetLastError() == cudaSuccess ? GF2X_OK : GF2X_ECUDA;
}

std::mutex g_plan_mu;
std::map<std::tuple<int, uint64_t, uint64_t>, std::shared_ptr<PlanSimple>> g_plans;

int plan_simple_for(uint64_t na_bits, uint64_t nb_bits, std::shared_ptr<PlanSimple> *out) {
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
    auto p = std::make_shared<PlanSimple>();
    int rc = plan_simple_init(p.get(), na_bits, nb_bits);
    if (rc) return rc;
    if (g_plans.size() >= 64) g_plans.clear();
    g_plans[key] = p;
    *out = p;
    return GF2X_OK;
}

int mul_simple_on_stream(const uint64_t *a, uint64_t na_bits, const uint64_t *b, uint64_t nb_bits,
                         uint64_t *out, cudaStream_t s) {
    std::shared_ptr<PlanSimple> p;
    int rc = plan_simple_for(na_bits, nb_bits, &p);
    if (rc) return rc;
    void *ws = nullptr;
    if ((rc = api::ws_alloc(&ws, p->ws_bytes, s))) return rc;
    std::unique_ptr<StageHook> tm(api::new_timer(s));
    rc = run_simple(p.get(), a, b, out, ws, s, tm.get());
    api::ws_free(ws, s);
    return rc;
}

int check_simple(const uint64_t *a, uint64_t na_bits, const uint64_t *b, uint64_t nb_bits,
                 const uint64_t *out) {
    if (na_bits > (1ull << 33) || nb_bits > (1ull << 33)) return GF2X_EINVAL;
    return api::check_product_args(a, na_bits, b, nb_bits, out);
}

}  // namespace
}  // namespace gf2x

using namespace gf2x;

extern "C" {

int gf2x_mul_simple_async(const uint64_t *a, uint64_t na_bits, const uint64_t *b, uint64_t nb_bits,
                          uint64_t *out, gf2x_stream_t stream) {
    try {
        int rc = check_simple(a, na_bits, b, nb_bits, out);
        if (rc) return rc;
        if (!na_bits || !nb_bits) return GF2X_OK;
        return mul_simple_on_stream(a, na_bits, b, nb_bits, out, reinterpret_cast<cudaStream_t>(stream));
    } catch (const std::bad_alloc &) {
        return GF2X_ENOMEM;
    } catch (...) {
        return GF2X_ECUDA;
    }
}

int gf2x_mul_simple(const uint64_t *a, uint64_t na_bits, const uint64_t *b, uint64_t nb_bits,
                    uint64_t *out) {
    int rc = gf2x_mul_simple_async(a, na_bits, b, nb_bits, out, nullptr);
    if (rc) return rc;
    if (cudaStreamSynchronize(0) != cudaSuccess) {
        cudaGetLastError();
        return GF2X_ECUDA;
    }
    return GF2X_OK;
}

int gf2x_stage_fft_simple(void *F, int log_n, int layers, int inverse, gf2x_stream_t stream) {
    if (log_n < 0 || log_n > kMaxLogN || layers < 0 || layers > log_n) return GF2X_EINVAL;
    try {
        const uint4 *beta;
        int rc = poly::cantor_dev(&beta);
        if (rc) return rc;
        poly::launch_fft(static_cast<uint4 *>(F), log_n, layers, inverse ? 1 : 0, 1, 0, -1, beta,
                         reinterpret_cast<cudaStream_t>(stream));
        return cudaGetLastError() == cudaSuccess ? GF2X_OK : GF2X_ECUDA;
    } catch (...) {
        return GF2X_ECUDA;
    }
}

int gf2x_stage_gfmul_simple(const void *A, void *B, uint64_t n, gf2x_stream_t stream) {
    if (!n) return GF2X_OK;
    try {
        poly::launch_gfmul(static_cast<const uint4 *>(A), static_cast<uint4 *>(B), n,
                           reinterpret_cast<cudaStream_t>(stream));
        return cudaGetLastError() == cudaSuccess ? GF2X_OK : GF2X_ECUDA;
    } catch (...) {
        return GF2X_ECUDA;
    }
}

}  // extern "C"
