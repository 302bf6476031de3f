// Direct products by a short operand (at most kSmallWords words), without a
// transform: c = x y with y short is the sum over y's words y_i of x y_i
// shifted by i words, and each x_q y_i is one 64 x 64 carry-less product
// (clmul.cuh) whose low word lands at q + i and high word at q + i + 1.
//
// Used by the one-shot products for two things:
//  * an operand of at most kSmallWords words: the whole product this way;
//  * the tails split off a product whose word count lies just above a power
//    of two (Sec. 5 on non-power-of-two lengths): with a = a0 + x^(64 A) a1,
//    b = b0 + x^(64 B) b1 and A + B - 1 words fitting half the transform,
//      a b = a0 b0 + x^(64 A) (a1 b) + x^(64 B) (a0 b1),
//    the main product a0 b0 takes a transform of half the length and the two
//    tail products (a1 or b1 of at most kSmallWords words) are added here.
#include <algorithm>

#include "clmul.cuh"
#include "gf2x_dev.cuh"
#include "kernels.h"
#include "launch.h"
#include "small.h"

namespace gf2x {
namespace {

constexpr int kWordsPerThread = 4;

// Product words [j0, j0 + K) per thread: for every word y_i the K + 1 input
// words x_q whose products reach them (q = j0 - i - 1 .. j0 + K - 1 - i).
// out[off + j] receives (or, with `accumulate`, XORs in) word j of x y for
// j < nprod and off + j < out_limit.
__global__ void __launch_bounds__(256) k_mul_small(const uint64_t *__restrict__ x, uint64_t xw,
                                                   uint64_t x_mask, const uint64_t *__restrict__ y,
                                                   int yw, uint64_t y_mask, uint64_t *out,
                                                   uint64_t nprod, uint64_t out_limit, uint64_t off,
                                                   int accumulate) {
    pdl_release();
    pdl_acquire();
    __shared__ uint64_t ys[kSmallWords];
    if ((int)threadIdx.x < yw) {
        uint64_t v = y[threadIdx.x];
        if ((int)threadIdx.x == yw - 1) v &= y_mask;
        ys[threadIdx.x] = v;
    }
    __syncthreads();
    constexpr int K = kWordsPerThread;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t * K < nprod;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t j0 = t * K;
        uint64_t acc[K];
#pragma unroll
        for (int k = 0; k < K; k++) acc[k] = 0;
        for (int i = 0; i < yw; i++) {
            const uint64_t yi = ys[i];
#pragma unroll
            for (int k = -1; k < K; k++) {
                const int64_t q = (int64_t)j0 - i + k;
                if (q < 0 || (uint64_t)q >= xw) continue;
                uint64_t xv = __ldg(x + q);
                if ((uint64_t)q == xw - 1) xv &= x_mask;
                uint64_t lo, hi;
                clmul64(xv, yi, lo, hi);
                if (k >= 0) acc[k] ^= lo;
                if (k + 1 < K) acc[k + 1] ^= hi;
            }
        }
#pragma unroll
        for (int k = 0; k < K; k++) {
            const uint64_t j = j0 + k;
            if (j < nprod && off + j < out_limit) out[off + j] = accumulate ? out[off + j] ^ acc[k] : acc[k];
        }
    }
}

// The same for `count` products of a batch, product y (blockIdx.y) read
// from the descriptors (the shorter operand, at most kSmallWords words,
// multiplies the longer); the output gets dout[y].words words.
__global__ void __launch_bounds__(256) k_mul_small_many(const OperandDesc *__restrict__ da,
                                                        const OperandDesc *__restrict__ db,
                                                        const OutputDesc *__restrict__ dout) {
    __shared__ uint64_t ys[kSmallWords];
    const OperandDesc A = da[blockIdx.y], B = db[blockIdx.y];
    const OutputDesc O = dout[blockIdx.y];
    const bool b_short = B.nw <= A.nw;
    const OperandDesc X = b_short ? A : B, Y = b_short ? B : A;
    const int yw = (int)Y.nw;
    if ((int)threadIdx.x < yw) {
        uint64_t v = Y.src[threadIdx.x];
        if ((int)threadIdx.x == yw - 1) v &= Y.mask;
        ys[threadIdx.x] = v;
    }
    __syncthreads();
    constexpr int K = kWordsPerThread;
    const uint64_t nprod = O.words;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t * K < nprod;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t j0 = t * K;
        uint64_t acc[K];
#pragma unroll
        for (int k = 0; k < K; k++) acc[k] = 0;
        for (int i = 0; i < yw; i++) {
            const uint64_t yi = ys[i];
#pragma unroll
            for (int k = -1; k < K; k++) {
                const int64_t q = (int64_t)j0 - i + k;
                if (q < 0 || (uint64_t)q >= X.nw) continue;
                uint64_t xv = __ldg(X.src + q);
                if ((uint64_t)q == X.nw - 1) xv &= X.mask;
                uint64_t lo, hi;
                clmul64(xv, yi, lo, hi);
                if (k >= 0) acc[k] ^= lo;
                if (k + 1 < K) acc[k + 1] ^= hi;
            }
        }
#pragma unroll
        for (int k = 0; k < K; k++)
            if (j0 + k < nprod) O.out[j0 + k] = acc[k];
    }
}

}  // namespace

void launch_mul_small_many(const OperandDesc *da, const OperandDesc *db, const OutputDesc *dout,
                           int count, uint64_t max_words, cudaStream_t s) {
    if (count <= 0) return;
    const uint64_t threads = (max_words + kWordsPerThread - 1) / kWordsPerThread;
    const unsigned gx = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((threads + 255) / 256, 1024));
    k_mul_small_many<<<dim3(gx, (unsigned)count), 256, 0, s>>>(da, db, dout);
}

void launch_mul_small(const uint64_t *x, uint64_t x_bits, const uint64_t *y, uint64_t y_bits,
                      uint64_t *out, uint64_t out_limit, uint64_t off, bool accumulate,
                      cudaStream_t s) {
    const uint64_t xw = (x_bits + 63) / 64, yw = (y_bits + 63) / 64;
    if (!xw || !yw) return;
    const uint64_t nprod = (x_bits + y_bits - 1 + 63) / 64;
    const uint64_t mx = (x_bits % 64) ? ((1ull << (x_bits % 64)) - 1) : ~0ull;
    const uint64_t my = (y_bits % 64) ? ((1ull << (y_bits % 64)) - 1) : ~0ull;
    const uint64_t threads = (nprod + kWordsPerThread - 1) / kWordsPerThread;
    const unsigned grid = (unsigned)std::max<uint64_t>(
        1, std::min<uint64_t>((threads + 255) / 256, (uint64_t)num_sms() * 16));
    launch_k(k_mul_small, grid, 256, 0, s, x, xw, mx, y, (int)yw, my, out, nprod, out_limit, off,
             accumulate ? 1 : 0);
}

bool tail_split(uint64_t aw, uint64_t bw, uint64_t *A, uint64_t *B) {
    if (!aw || !bw) return false;
    const uint64_t need = aw + bw - 1;
    if (need < 64) return false;  // small transforms: nothing to gain
    uint64_t N = 1;
    while (N < need) N <<= 1;
    const uint64_t X = need - N / 2;  // words past half the transform
    if (X == 0 || X > (uint64_t)kSmallWords) return false;
    // the tail from the longer operand (one tail product), the rest from the
    // other one
    const bool a_long = aw >= bw;
    const uint64_t L = a_long ? aw : bw, S = a_long ? bw : aw;
    const uint64_t tl = std::min<uint64_t>(X, L - 1), ts = X - tl;
    if (ts >= S) return false;
    *A = a_long ? aw - tl : aw - ts;
    *B = a_long ? bw - ts : bw - tl;
    return true;
}

}  // namespace gf2x
