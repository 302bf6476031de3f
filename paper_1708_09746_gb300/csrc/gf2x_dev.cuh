// Device-side tower-field arithmetic (Sec. 3.2, Prop. 3.2, Sec. 4.1).
//
// Elements of F~_{2^128} are uint4: .x = bits 0..31, .y = 32..63,
// .z = 64..95, .w = 96..127.  Each 32-bit limb is a coordinate over the
// subfield F~_{2^32} (Prop. 3.2): a product by a constant c in F~_{2^32} is
// four independent F~_{2^32} products, one per limb.
//
// The F~_{2^32} products reduce by Karatsuba through F~_{2^16} to F~_{2^8}
// (x_{k+1}^2 = x_{k+1} + v_{2^k - 1}) and multiply in F~_{2^8} with
// logarithm / exponential tables held in shared memory (the GF(256)
// log/exp method the paper cites for pointmul, Sec. 4.1.3).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gf2x {

// Shared-memory copy of the F~_{2^8} tables (1.8 KiB).
struct SmemGF8 {
    uint16_t log8[256];
    uint8_t exp8[1040];
    uint8_t mul80[256];
};

// Global (device) copy of the size-independent tables.
struct DevTables {
    uint32_t S[32][32];
    uint4 chr_in[8][256];
    uint4 chr_out[16][256];
    SmemGF8 gf8;
};

__device__ __forceinline__ void load_gf8(SmemGF8 &s, const SmemGF8 *g) {
    const uint32_t *src = reinterpret_cast<const uint32_t *>(g);
    uint32_t *dst = reinterpret_cast<uint32_t *>(&s);
    for (int i = threadIdx.x; i < (int)(sizeof(SmemGF8) / 4); i += blockDim.x) dst[i] = src[i];
}

// ---- F~_{2^8} ----------------------------------------------------------------
__device__ __forceinline__ uint32_t gmul8(const SmemGF8 &t, uint32_t a, uint32_t b) {
    return t.exp8[t.log8[a] + t.log8[b]];
}
// a * c where lc = log8[c] (precomputed; 512 for c = 0).
__device__ __forceinline__ uint32_t gmul8_l(const SmemGF8 &t, uint32_t a, uint32_t lc) {
    return t.exp8[t.log8[a] + lc];
}

// ---- F~_{2^16} = F~_{2^8}[x_4], x_4^2 = x_4 + v_7 --------------------------------
__device__ __forceinline__ uint32_t gmul16(const SmemGF8 &t, uint32_t a, uint32_t b) {
    uint32_t a0 = a & 0xff, a1 = a >> 8, b0 = b & 0xff, b1 = b >> 8;
    uint32_t r0 = gmul8(t, a0, b0);
    uint32_t r1 = gmul8(t, a1, t.mul80[b1]);
    uint32_t r2 = gmul8(t, a0 ^ a1, b0 ^ b1);
    return (r0 ^ r1) | ((r2 ^ r0) << 8);
}
// x * v_15 in F~_{2^16} (v_15 = v_7 * x_4).
__device__ __forceinline__ uint32_t gmulP16(const SmemGF8 &t, uint32_t x) {
    uint32_t x0 = x & 0xff, x1 = x >> 8;
    return (uint32_t)t.mul80[t.mul80[x1]] | ((uint32_t)t.mul80[x0 ^ x1] << 8);
}

// ---- F~_{2^32} = F~_{2^16}[x_5], x_5^2 = x_5 + v_15 ------------------------------
__device__ __forceinline__ uint32_t gmul32(const SmemGF8 &t, uint32_t a, uint32_t b) {
    uint32_t a0 = a & 0xffff, a1 = a >> 16, b0 = b & 0xffff, b1 = b >> 16;
    uint32_t r0 = gmul16(t, a0, b0);
    uint32_t r1 = gmul16(t, a1, gmulP16(t, b1));
    uint32_t r2 = gmul16(t, a0 ^ a1, b0 ^ b1);
    return (r0 ^ r1) | ((r2 ^ r0) << 16);
}
// x * v_31 in F~_{2^32} (v_31 = v_15 * x_5).
__device__ __forceinline__ uint32_t gmulP32(const SmemGF8 &t, uint32_t x) {
    uint32_t x0 = x & 0xffff, x1 = x >> 16;
    return gmulP16(t, gmulP16(t, x1)) | (gmulP16(t, x0 ^ x1) << 16);
}

// A multiplier c in F~_{2^32} prepared once for many products: the logs of
// the nine F~_{2^8} Karatsuba leaves of c (the v_7 and v_15 factors of the
// reduction folded into the leaves).
struct MulConst32 {
    uint16_t l[9];
};

__device__ __forceinline__ MulConst32 prep_const32(const SmemGF8 &t, uint32_t c) {
    uint32_t C0 = c & 0xffff, C1 = gmulP16(t, c >> 16), C2 = C0 ^ (c >> 16);
    uint32_t Cs[3] = {C0, C1, C2};
    MulConst32 m;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        uint32_t lo = Cs[i] & 0xff, hi = Cs[i] >> 8;
        m.l[3 * i + 0] = t.log8[lo];
        m.l[3 * i + 1] = t.log8[t.mul80[hi]];
        m.l[3 * i + 2] = t.log8[lo ^ hi];
    }
    return m;
}

// F~_{2^16} product of x by the prepared 16-bit constant with leaf logs l0..l2.
__device__ __forceinline__ uint32_t cmul16(const SmemGF8 &t, uint32_t x, uint32_t l0, uint32_t l1,
                                           uint32_t l2) {
    uint32_t x0 = x & 0xff, x1 = x >> 8;
    uint32_t r0 = gmul8_l(t, x0, l0);
    uint32_t r1 = gmul8_l(t, x1, l1);
    uint32_t r2 = gmul8_l(t, x0 ^ x1, l2);
    return (r0 ^ r1) | ((r2 ^ r0) << 8);
}

__device__ __forceinline__ uint32_t cmul32(const SmemGF8 &t, uint32_t x, const MulConst32 &m) {
    uint32_t X0 = x & 0xffff, X1 = x >> 16;
    uint32_t R0 = cmul16(t, X0, m.l[0], m.l[1], m.l[2]);
    uint32_t R1 = cmul16(t, X1, m.l[3], m.l[4], m.l[5]);
    uint32_t R2 = cmul16(t, X0 ^ X1, m.l[6], m.l[7], m.l[8]);
    return (R0 ^ R1) | ((R2 ^ R0) << 16);
}

// v * c for v in F~_{2^128}, c in F~_{2^32}: limb-wise (Prop. 3.2).
__device__ __forceinline__ uint4 cmul128(const SmemGF8 &t, uint4 v, const MulConst32 &m) {
    return make_uint4(cmul32(t, v.x, m), cmul32(t, v.y, m), cmul32(t, v.z, m), cmul32(t, v.w, m));
}

// ---- F~_{2^64} = F~_{2^32}[x_6] and F~_{2^128} = F~_{2^64}[x_7] ------------------
struct u32x2 {
    uint32_t lo, hi;
};

__device__ __forceinline__ u32x2 gmul64(const SmemGF8 &t, u32x2 a, u32x2 b) {
    uint32_t b1p = gmulP32(t, b.hi);
    uint32_t r0 = gmul32(t, a.lo, b.lo);
    uint32_t r1 = gmul32(t, a.hi, b1p);
    uint32_t r2 = gmul32(t, a.lo ^ a.hi, b.lo ^ b.hi);
    return u32x2{r0 ^ r1, r2 ^ r0};
}
// x * v_63 in F~_{2^64} (v_63 = v_31 * x_6).
__device__ __forceinline__ u32x2 gmulP64(const SmemGF8 &t, u32x2 x) {
    return u32x2{gmulP32(t, gmulP32(t, x.hi)), gmulP32(t, x.lo ^ x.hi)};
}

__device__ __forceinline__ uint4 gmul128(const SmemGF8 &t, uint4 a, uint4 b) {
    u32x2 a0{a.x, a.y}, a1{a.z, a.w}, b0{b.x, b.y}, b1{b.z, b.w};
    u32x2 b1p = gmulP64(t, b1);
    u32x2 r0 = gmul64(t, a0, b0);
    u32x2 r1 = gmul64(t, a1, b1p);
    u32x2 s{a0.lo ^ a1.lo, a0.hi ^ a1.hi}, u{b0.lo ^ b1.lo, b0.hi ^ b1.hi};
    u32x2 r2 = gmul64(t, s, u);
    return make_uint4(r0.lo ^ r1.lo, r0.hi ^ r1.hi, r2.lo ^ r0.lo, r2.hi ^ r0.hi);
}

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
