// Direct products by a short operand and the tail split of products just
// above a power-of-two length (small.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace gf2x {

// The longest short operand (in 64-bit words) multiplied without a transform.
constexpr int kSmallWords = 16;

// x * y (y of at most kSmallWords words; bits past x_bits and y_bits ignored)
// into out[off .. off + words of the product), words at or past out_limit not
// written; with `accumulate` XORed into out instead of stored.
void launch_mul_small(const uint64_t *x, uint64_t x_bits, const uint64_t *y, uint64_t y_bits,
                      uint64_t *out, uint64_t out_limit, uint64_t off, bool accumulate,
                      cudaStream_t s);

struct OperandDesc;
struct OutputDesc;

// `count` direct products of a batch (count <= 65535): product y multiplies
// the operands da[y], db[y] (the shorter of at most kSmallWords words) into
// dout[y]; max_words bounds the outputs' lengths.  Device descriptors.
void launch_mul_small_many(const OperandDesc *da, const OperandDesc *db, const OutputDesc *dout,
                           int count, uint64_t max_words, cudaStream_t s);

// For a product of aw x bw words whose N = 2^ceil(log2(aw + bw - 1)) points
// could be halved by cutting at most kSmallWords words off the operands: the
// words A <= aw and B <= bw kept in the main product (A + B - 1 <= N / 2).
bool tail_split(uint64_t aw, uint64_t bw, uint64_t *A, uint64_t *B);

}  // namespace gf2x
