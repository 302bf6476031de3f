// Device-side tables and helpers shared by the kernels.
//
// Elements of F~_{2^128} are uint4: .x = bits 0..31, .y = 32..63,
// .z = 64..95, .w = 96..127.  Each 32-bit limb is a coordinate over the
// subfield F~_{2^32} (Prop. 3.2): a product by a constant c in F~_{2^32} is
// four independent F~_{2^32} products, one per limb (gf2x_mul.cuh).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gf2x {

struct u32x2 {
    uint32_t lo, hi;
};

// Global (device) copy of the size-independent tables.
struct DevTables {
    uint32_t S[32][32];
    uint4 chr_in[8][256];
    uint8_t mul8[65536];
    uint32_t shfl_basis[32][7][32];
    uint32_t shfl_m4r[4][256][7][32];
    // Rows 0-2 of a contiguous FFT tile.  low_lane[x][l]: byte 0 = v_7 x,
    // byte 1 + r = delta_r(l) x with delta_r(l) = s_r(phi(l << 3)), an element
    // of F~_{2^8} (products in F~_{2^8}).  low_shfl[kLowOff[r] + blk * (4 >> r)
    // + h]: the shuffle table of s_r(phi((blk << 8) | (h << (r + 1)))).
    uint32_t low_lane[256][32];
    uint32_t low_shfl[112][7][32];
    // changeRepr^-1 as warp-shuffle tables: psi_shfl[o][q][w][l] = word o of
    // psi(e), e = the element whose word q holds l << 5w (w < 6) or
    // (l & 3) << 30 (w = 6) and is zero elsewhere.
    uint32_t psi_shfl[4][4][7][32];
    // changeRepr the same way: phi_shfl[o][q][w][l] = word o of phi(b), b =
    // the 64-bit block whose 32-bit half q holds l << 5w (w < 6) or
    // (l & 3) << 30 (w = 6) and is zero elsewhere.
    uint32_t phi_shfl[4][2][7][32];
};

constexpr int kLowOff[3] = {0, 64, 96};

// Programmatic dependent launch (kernels launched by launch_k): pdl_release
// lets the next kernel of the stream be scheduled once every CTA of this one
// has started; pdl_acquire returns once the earlier kernels of the stream have
// completed and their writes are visible.  A kernel reads and writes nothing
// that an earlier kernel of the stream touches before its pdl_acquire (only
// constant tables are read before it).  Both are no-ops in a kernel launched
// without the attribute.
__device__ __forceinline__ void pdl_release() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_acquire() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ uint4 xor4(uint4 a, uint4 b) {
    return make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w);
}

// s_k(alpha) for alpha = phi_v(a) (Sec. 4.4): XOR of S[k][t] over set bits t.
__device__ __forceinline__ uint32_t s_k_of(const uint32_t *Sk, uint32_t a) {
    uint32_t c = 0;
    while (a) {
        int t = __ffs(a) - 1;
        c ^= __ldg(Sk + t);
        a &= a - 1;
    }
    return c;
}

}  // namespace gf2x
