// Tower-field multiplication kernels' building blocks for the fused passes.
//
// Two ways to multiply a 128-bit element by a multiplier c in F~_{2^32}
// (limb-wise by Prop. 3.2):
//
//  * Warp-shuffle tables, when all 32 lanes of a warp share c: lane l holds
//    T_w[l] = c * (l << 5w) for w < 6 and T_6[l] = c * ((l & 3) << 30), so a
//    limb x is the XOR of seven shuffles indexed by its 5-bit windows (the
//    lane index of a shuffle is taken modulo 32).  This is the method of four
//    Russians of Sec. 4.3/4.4 with the table spread over the warp's registers
//    instead of a cache.  A variant takes the 2-bit window on the integer
//    pipe (six shuffles per limb).
//
//  * The full F~_{2^8} product table (64 KiB in shared memory), when c differs
//    from lane to lane: the F~_{2^32} product is Karatsuba over F~_{2^16} and
//    F~_{2^8} (9 table lookups per limb), the reductions by v_7 and v_15
//    folded into the multiplier's leaves.
#pragma once
#include "gf2x_dev.cuh"

namespace gf2x {

constexpr unsigned kFull = 0xffffffffu;

struct ShflTab {
    uint32_t t[7];
};

__device__ __forceinline__ uint32_t shfl_mul32(uint32_t x, const ShflTab &T) {
    uint32_t r = __shfl_sync(kFull, T.t[0], x);
    r ^= __shfl_sync(kFull, T.t[1], x >> 5);
    r ^= __shfl_sync(kFull, T.t[2], x >> 10);
    r ^= __shfl_sync(kFull, T.t[3], x >> 15);
    r ^= __shfl_sync(kFull, T.t[4], x >> 20);
    r ^= __shfl_sync(kFull, T.t[5], x >> 25);
    r ^= __shfl_sync(kFull, T.t[6], x >> 30);
    return r;
}

__device__ __forceinline__ uint4 shfl_mul128(uint4 v, const ShflTab &T) {
    return make_uint4(shfl_mul32(v.x, T), shfl_mul32(v.y, T), shfl_mul32(v.z, T),
                      shfl_mul32(v.w, T));
}

// The same product with six shuffles per limb: the 2-bit window (bits 30, 31)
// goes through the integer pipe instead, as x_30 c 2^30 + x_31 c 2^31 with the
// two warp-uniform products c1 = c * 2^30, c2 = c * 2^31 masked by the bits.
// The FFT passes run on the shuffle / shared-memory pipe; this moves a
// seventh of their shuffles onto the integer ALU, which has room.
struct ShflTab6 {
    uint32_t t[6];
    uint32_t c1, c2;
};

__device__ __forceinline__ uint32_t shfl6_mul32(uint32_t x, const ShflTab6 &T) {
    uint32_t r = __shfl_sync(kFull, T.t[0], x);
    r ^= __shfl_sync(kFull, T.t[1], x >> 5);
    r ^= __shfl_sync(kFull, T.t[2], x >> 10);
    r ^= __shfl_sync(kFull, T.t[3], x >> 15);
    r ^= __shfl_sync(kFull, T.t[4], x >> 20);
    r ^= __shfl_sync(kFull, T.t[5], x >> 25);
    const uint32_t m31 = (uint32_t)((int32_t)x >> 31);         // all ones iff bit 31
    const uint32_t m30 = (uint32_t)((int32_t)(x << 1) >> 31);  // all ones iff bit 30
    return r ^ (m30 & T.c1) ^ (m31 & T.c2);
}

__device__ __forceinline__ uint4 shfl6_mul128(uint4 v, const ShflTab6 &T) {
    return make_uint4(shfl6_mul32(v.x, T), shfl6_mul32(v.y, T), shfl6_mul32(v.z, T),
                      shfl6_mul32(v.w, T));
}

// The six-shuffle table of c1 + c2 (so of the sum of two multipliers) from two
// seven-word tables laid out [w][32 lanes]: words 0..5 at the calling lane of
// each, and the two constants from lanes 2 and 3 of word 6 (c * 2^31 and
// c * (2^30 + 2^31)), read as one 8-byte broadcast per table.  `a` may be in
// shared or global memory, `b` is read through the read-only path.
__device__ __forceinline__ ShflTab6 shfl6_table_sum(const uint32_t *a, const uint32_t *__restrict__ b,
                                                    int lane) {
    ShflTab6 T;
#pragma unroll
    for (int w = 0; w < 6; w++) T.t[w] = a[32 * w + lane] ^ __ldg(b + 32 * w + lane);
    const uint2 pa = *reinterpret_cast<const uint2 *>(a + 6 * 32 + 2);
    const uint2 pb = __ldg(reinterpret_cast<const uint2 *>(b + 6 * 32 + 2));
    T.c2 = pa.x ^ pb.x;
    T.c1 = pa.y ^ pb.y ^ T.c2;
    return T;
}

// One seven-word table read the same way (global memory, read-only path).
__device__ __forceinline__ ShflTab6 shfl6_table(const uint32_t *__restrict__ b, int lane) {
    ShflTab6 T;
#pragma unroll
    for (int w = 0; w < 6; w++) T.t[w] = __ldg(b + 32 * w + lane);
    const uint2 pb = __ldg(reinterpret_cast<const uint2 *>(b + 6 * 32 + 2));
    T.c2 = pb.x;
    T.c1 = pb.y ^ pb.x;
    return T;
}

// The table of a sum of multipliers is the XOR of their tables.
__device__ __forceinline__ void shfl6_xor(ShflTab6 &T, const ShflTab6 &U) {
#pragma unroll
    for (int w = 0; w < 6; w++) T.t[w] ^= U.t[w];
    T.c1 ^= U.c1;
    T.c2 ^= U.c2;
}

// ---- F~_{2^8} product table: mt[(c << 8) | x] = c * x ----------------------
// The products by the constant v_7 (the reductions X^2 = X + v_{W-1} of every
// tower level end in them) come from a second table with one copy per lane:
// byte 0 of word x * 32 + l is v_7 x for lane l, so the 32 lanes of a warp
// always read 32 different banks (bytes 1..3 hold the per-lane products of the
// lowest FFT rows, DevTables::low_lane).  `v7` points at the calling lane's
// word of entry 0 (table base + 4 * lane).
struct MtRef {
    const uint8_t *mt;
    const uint8_t *v7;
};

constexpr size_t kLaneTabBytes = 256 * 32 * 4;

__device__ __forceinline__ MtRef mt_ref(const uint8_t *mt, const uint32_t *lane_tab) {
    return MtRef{mt, reinterpret_cast<const uint8_t *>(lane_tab + (threadIdx.x & 31))};
}

__device__ __forceinline__ uint32_t mt_v7(const MtRef &M, uint32_t x) {
    return M.v7[x << 7];  // x * v_7
}

__device__ __forceinline__ uint32_t mt_v77(const MtRef &M, uint32_t x) {
    return mt_v7(M, mt_v7(M, x));  // x * v_7^2
}

// x * v_15 in F~_{2^16}
__device__ __forceinline__ uint32_t mt_p16(const MtRef &M, uint32_t x) {
    uint32_t x0 = x & 0xff, x1 = x >> 8;
    return mt_v77(M, x1) | (mt_v7(M, x0 ^ x1) << 8);
}

// A multiplier prepared for the product table: row offsets (leaf << 8) of
// the nine F~_{2^8} Karatsuba leaves.
struct MtConst {
    uint32_t r[9];
};

__device__ __forceinline__ MtConst mt_prep(const MtRef &M, uint32_t c) {
    uint32_t h = c >> 16;
    uint32_t Cs[3] = {c & 0xffff, mt_p16(M, h), (c & 0xffff) ^ h};
    MtConst m;
#pragma unroll
    for (int j = 0; j < 3; j++) {
        uint32_t lo = Cs[j] & 0xff, hi = Cs[j] >> 8;
        m.r[3 * j + 0] = lo << 8;
        m.r[3 * j + 1] = mt_v7(M, hi) << 8;
        m.r[3 * j + 2] = (lo ^ hi) << 8;
    }
    return m;
}

__device__ __forceinline__ uint32_t mt_cmul16(const uint8_t *mt, uint32_t x, uint32_t r0,
                                              uint32_t r1, uint32_t r2) {
    uint32_t x0 = x & 0xff, x1 = x >> 8;
    uint32_t p0 = mt[r0 | x0], p1 = mt[r1 | x1], p2 = mt[r2 | (x0 ^ x1)];
    return (p0 ^ p1) | ((p2 ^ p0) << 8);
}

__device__ __forceinline__ uint32_t mt_cmul32(const uint8_t *mt, uint32_t x, const MtConst &m) {
    uint32_t X0 = x & 0xffff, X1 = x >> 16;
    uint32_t a = mt_cmul16(mt, X0, m.r[0], m.r[1], m.r[2]);
    uint32_t b = mt_cmul16(mt, X1, m.r[3], m.r[4], m.r[5]);
    uint32_t d = mt_cmul16(mt, X0 ^ X1, m.r[6], m.r[7], m.r[8]);
    return (a ^ b) | ((d ^ a) << 16);
}

__device__ __forceinline__ uint4 mt_cmul128(const MtRef &M, uint4 v, const MtConst &m) {
    return make_uint4(mt_cmul32(M.mt, v.x, m), mt_cmul32(M.mt, v.y, m), mt_cmul32(M.mt, v.z, m),
                      mt_cmul32(M.mt, v.w, m));
}

// Generic products (both operands variable) for pointmul.
__device__ __forceinline__ uint32_t mt_gmul16(const MtRef &M, uint32_t a, uint32_t b) {
    uint32_t a0 = a & 0xff, a1 = a >> 8, b0 = b & 0xff, b1 = b >> 8;
    uint32_t p0 = M.mt[(b0 << 8) | a0];
    uint32_t p1 = M.mt[(mt_v7(M, b1) << 8) | a1];
    uint32_t p2 = M.mt[((b0 ^ b1) << 8) | (a0 ^ a1)];
    return (p0 ^ p1) | ((p2 ^ p0) << 8);
}

__device__ __forceinline__ uint32_t mt_gmul32(const MtRef &M, uint32_t a, uint32_t b) {
    uint32_t a0 = a & 0xffff, a1 = a >> 16, b0 = b & 0xffff, b1 = b >> 16;
    uint32_t p0 = mt_gmul16(M, a0, b0);
    uint32_t p1 = mt_gmul16(M, a1, mt_p16(M, b1));
    uint32_t p2 = mt_gmul16(M, a0 ^ a1, b0 ^ b1);
    return (p0 ^ p1) | ((p2 ^ p0) << 16);
}

// x * v_31 in F~_{2^32}
__device__ __forceinline__ uint32_t mt_p32(const MtRef &M, uint32_t x) {
    uint32_t x0 = x & 0xffff, x1 = x >> 16;
    return mt_p16(M, mt_p16(M, x1)) | (mt_p16(M, x0 ^ x1) << 16);
}

__device__ __forceinline__ u32x2 mt_gmul64(const MtRef &M, u32x2 a, u32x2 b) {
    uint32_t p0 = mt_gmul32(M, a.lo, b.lo);
    uint32_t p1 = mt_gmul32(M, a.hi, mt_p32(M, b.hi));
    uint32_t p2 = mt_gmul32(M, a.lo ^ a.hi, b.lo ^ b.hi);
    return u32x2{p0 ^ p1, p2 ^ p0};
}

// x * v_63 in F~_{2^64}
__device__ __forceinline__ u32x2 mt_p64(const MtRef &M, u32x2 x) {
    return u32x2{mt_p32(M, mt_p32(M, x.hi)), mt_p32(M, x.lo ^ x.hi)};
}

__device__ __forceinline__ uint4 mt_gmul128(const MtRef &M, uint4 a, uint4 b) {
    u32x2 a0{a.x, a.y}, a1{a.z, a.w}, b0{b.x, b.y}, b1{b.z, b.w};
    u32x2 p0 = mt_gmul64(M, a0, b0);
    u32x2 p1 = mt_gmul64(M, a1, mt_p64(M, b1));
    u32x2 p2 = mt_gmul64(M, u32x2{a0.lo ^ a1.lo, a0.hi ^ a1.hi}, u32x2{b0.lo ^ b1.lo, b0.hi ^ b1.hi});
    return make_uint4(p0.lo ^ p1.lo, p0.hi ^ p1.hi, p2.lo ^ p0.lo, p2.hi ^ p0.hi);
}

}  // namespace gf2x
