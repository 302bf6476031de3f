// GF(2^128) in the polynomial basis with a Cantor basis (poly_field.cu):
// the field arithmetic and FFT passes of the simple form (Alg. 4) and the
// Frobenius-partition form (Appendix C).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace gf2x {
namespace poly {

// A field element on the host: lo = coefficients of z^0..z^63, hi = z^64..z^127.
struct H128 {
    uint64_t lo, hi;
};

// Product modulo z^128 + z^7 + z^2 + z + 1 (host).
H128 hmul(H128 a, H128 b);

// beta_0 .. beta_127 of the Cantor basis (host), element i as a uint4
// (.x = bits 0..31, ..., .w = bits 96..127).
const std::vector<uint4> &cantor_host();

// The same 128 elements on the current device (uploaded once).
int cantor_dev(const uint4 **beta);

// Layers 0 .. L-1 of FFT_LCH (inverse = 0: from the top layer down, the input
// already repeating its 2^L coefficients periodically) or all L layers of the
// inverse (inverse = 1, from the bottom up) on `count` transforms of 2^M
// elements at F + y * strideF, at the points alpha + phi_beta(i) with alpha =
// beta_{alpha_bit} (alpha = 0 if alpha_bit < 0).  Returns the launches.
int launch_fft(uint4 *F, int M, int L, int inverse, int count, uint64_t strideF, int alpha_bit,
               const uint4 *beta, cudaStream_t s);

// B[i] := A[i] * B[i], i < n.
void launch_gfmul(const uint4 *A, uint4 *B, uint64_t n, cudaStream_t s);

}  // namespace poly
}  // namespace gf2x
