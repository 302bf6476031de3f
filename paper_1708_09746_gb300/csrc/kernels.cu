// CUDA kernels of the product path (Alg. 5) and their host launchers.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "gf2x_dev.cuh"
#include "gf2x_internal.h"
#include "kernels.h"

namespace gf2x {

// ---------------------------------------------------------------------------
// Split (Sec. 2.1): copy the operand's words, clear bits past its length and
// zero-pad to P words.
__global__ void k_split_pad(const uint64_t *__restrict__ a, uint64_t nw, uint64_t last_mask,
                            uint64_t *__restrict__ w, uint64_t P) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < P;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t v = 0;
        if (i < nw) {
            v = a[i];
            if (i == nw - 1) v &= last_mask;
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
__global__ void k_bcvt_level(T *f, uint64_t n_half, int logE, int loge, int inverse) {
    const uint64_t E = 1ull << logE, e = 1ull << loge;
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < n_half;
         w += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t s = w >> logE, t = w & (E - 1);
        if (t >= E - e) continue;
        bcvt_item(f, s << (logE + 1), E, e, t, inverse);
    }
}

template <typename T>
__global__ void k_bcvt_tile(T *f, int tile_log, LevelBatch lb, int inverse) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s = reinterpret_cast<T *>(smem_raw);
    const uint64_t tile = 1ull << tile_log;
    T *g = f + blockIdx.x * tile;
    for (uint64_t i = threadIdx.x; i < tile; i += blockDim.x) s[i] = g[i];
    __syncthreads();
    for (int L = 0; L < lb.count; L++) {
        const int logE = lb.logE[L], loge = lb.loge[L];
        const uint64_t E = 1ull << logE, e = 1ull << loge;
        for (uint64_t w = threadIdx.x; w < tile / 2; w += blockDim.x) {
            uint64_t seg = w >> logE, t = w & (E - 1);
            if (t < E - e) bcvt_item(s, seg << (logE + 1), E, e, t, inverse);
        }
        __syncthreads();
    }
    for (uint64_t i = threadIdx.x; i < tile; i += blockDim.x) g[i] = s[i];
}

// ---------------------------------------------------------------------------
// changeRepr (Sec. 4.3): F[i] = phi(g[i mod P]), phi by 8-bit tables.  The
// periodic copy realises the fan-out of the FFT layers whose upper half is
// zero (Fig. 2).
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

// ---------------------------------------------------------------------------
// changeRepr^-1 and InterleavedCombine (Sec. 2.1): psi(F[j]) is a polynomial
// of degree < 128 in z; z -> x and y -> x^64 add its high word into the next
// output word.
__device__ __forceinline__ uint4 psi(const DevTables *__restrict__ T, uint4 e) {
    uint4 acc = make_uint4(0, 0, 0, 0);
    const uint32_t wv[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
    for (int q = 0; q < 4; q++)
#pragma unroll
        for (int b = 0; b < 4; b++)
            acc = xor4(acc, __ldg(&T->chr_out[4 * q + b][(wv[q] >> (8 * b)) & 255]));
    return acc;
}

__global__ void k_ichrepr_combine(const uint4 *__restrict__ F, uint64_t n, uint64_t *__restrict__ out,
                                  uint64_t out_words, uint64_t last_mask,
                                  const DevTables *__restrict__ T) {
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < out_words;
         j += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t v = 0;
        if (j < n) {
            uint4 c = psi(T, F[j]);
            v ^= (uint64_t)c.x | ((uint64_t)c.y << 32);
        }
        if (j >= 1 && j - 1 < n) {
            uint4 c = psi(T, F[j - 1]);
            v ^= (uint64_t)c.z | ((uint64_t)c.w << 32);
        }
        if (j == out_words - 1) v &= last_mask;
        out[j] = v;
    }
}

// ===========================================================================
// Host launchers.

static inline unsigned grid_for(uint64_t work, unsigned block, unsigned cap = 1u << 20) {
    uint64_t g = (work + block - 1) / block;
    if (g == 0) g = 1;
    return (unsigned)std::min<uint64_t>(g, cap);
}

void launch_split_pad(const uint64_t *a, uint64_t nw, uint64_t last_mask, uint64_t *w, uint64_t P,
                      cudaStream_t s) {
    k_split_pad<<<grid_for(P, 256), 256, 0, s>>>(a, nw, last_mask, w, P);
}

template <typename T>
static int tile_log_for() {
    return sizeof(T) == 8 ? 12 : 11;  // 32 KiB tiles
}

template <typename T>
uint64_t run_basis_cvt(T *f, int m, const std::vector<Level> &fwd, int inverse, cudaStream_t s) {
    uint64_t launches = 0;
    std::vector<Level> lv = fwd;
    if (inverse) std::reverse(lv.begin(), lv.end());
    const int tl = std::min(tile_log_for<T>(), m);
    const uint64_t n = 1ull << m;
    size_t i = 0;
    while (i < lv.size()) {
        if (lv[i].logE + 1 <= tl) {
            LevelBatch lb{};
            lb.count = 0;
            while (i < lv.size() && lv[i].logE + 1 <= tl && lb.count < LevelBatch::kMax) {
                lb.logE[lb.count] = lv[i].logE;
                lb.loge[lb.count] = lv[i].loge;
                lb.count++;
                i++;
            }
            size_t smem = (size_t)sizeof(T) << tl;
            k_bcvt_tile<T><<<(unsigned)(n >> tl), 256, smem, s>>>(f, tl, lb, inverse);
            launches++;
        } else {
            k_bcvt_level<T><<<grid_for(n / 2, 256), 256, 0, s>>>(f, n / 2, lv[i].logE, lv[i].loge,
                                                                 inverse);
            launches++;
            i++;
        }
    }
    return launches;
}

template uint64_t run_basis_cvt<uint64_t>(uint64_t *, int, const std::vector<Level> &, int,
                                          cudaStream_t);
template uint64_t run_basis_cvt<uint4>(uint4 *, int, const std::vector<Level> &, int,
                                       cudaStream_t);

void launch_chrepr(const uint64_t *g, uint64_t P, uint4 *F, uint64_t n, const DevTables *T,
                   cudaStream_t s) {
    k_chrepr<<<grid_for(n, 256), 256, 0, s>>>(g, P - 1, F, n, T);
}

void launch_ichrepr_combine(const uint4 *F, uint64_t n, uint64_t *out, uint64_t out_words,
                            uint64_t last_mask, const DevTables *T, cudaStream_t s) {
    k_ichrepr_combine<<<grid_for(out_words, 256), 256, 0, s>>>(F, n, out, out_words, last_mask, T);
}

}  // namespace gf2x
