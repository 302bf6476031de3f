// Carry-less products of machine words on the GPU (no carry-less multiply
// instruction on sm_103a): shared by the polynomial-basis field arithmetic and
// the direct products by short operands.
#pragma once
#include <cstdint>

namespace gf2x {

// 32 x 32 -> 64-bit carry-less product: operand bits split into four classes
// by position mod 4; the integer product of two classes has its nonzero
// column sums (at most 8 terms, below 16) in 4-bit fields at the positions of
// class i + j, so its bit there is the column's parity.  The products of one
// output class are XORed and masked to that class.
__device__ __forceinline__ uint64_t clmul32(uint32_t a, uint32_t b) {
    const uint32_t m = 0x11111111u;
    const uint32_t a0 = a & m, a1 = a & (m << 1), a2 = a & (m << 2), a3 = a & (m << 3);
    const uint32_t b0 = b & m, b1 = b & (m << 1), b2 = b & (m << 2), b3 = b & (m << 3);
    auto mw = [](uint32_t x, uint32_t y) { return (uint64_t)x * (uint64_t)y; };
    const uint64_t z0 = mw(a0, b0) ^ mw(a1, b3) ^ mw(a2, b2) ^ mw(a3, b1);
    const uint64_t z1 = mw(a0, b1) ^ mw(a1, b0) ^ mw(a2, b3) ^ mw(a3, b2);
    const uint64_t z2 = mw(a0, b2) ^ mw(a1, b1) ^ mw(a2, b0) ^ mw(a3, b3);
    const uint64_t z3 = mw(a0, b3) ^ mw(a1, b2) ^ mw(a2, b1) ^ mw(a3, b0);
    const uint64_t M = 0x1111111111111111ull;
    return (z0 & M) | (z1 & (M << 1)) | (z2 & (M << 2)) | (z3 & (M << 3));
}

// 64 x 64 -> 128 by Karatsuba over 32-bit halves.
__device__ __forceinline__ void clmul64(uint64_t a, uint64_t b, uint64_t &lo, uint64_t &hi) {
    const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32);
    const uint32_t b0 = (uint32_t)b, b1 = (uint32_t)(b >> 32);
    const uint64_t p0 = clmul32(a0, b0), p2 = clmul32(a1, b1);
    const uint64_t pm = clmul32(a0 ^ a1, b0 ^ b1) ^ p0 ^ p2;
    lo = p0 ^ (pm << 32);
    hi = p2 ^ (pm >> 32);
}

}  // namespace gf2x
