// Bulk asynchronous copies (TMA, cp.async.bulk) between global and shared
// memory, completed on shared-memory mbarriers, for the double-buffered tile
// pipelines of the pass kernels.
//
// A tile is 2^w "rows" (index bits lo .. lo+w-1) of 2^c consecutive elements
// (index bits 0 .. c-1); the other index bits name the tile.  Each row is one
// bulk copy of (2^c << esz_log) bytes (a multiple of 16 bytes, 16-byte
// aligned); when lo == c the rows are adjacent and the tile is one copy.
//
// Every wait is bounded: a wait that runs out reports failure, and the kernel
// records GF2X_ETIMEOUT in its status word and leaves the pipeline.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gf2x {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Default bound of a wait, in try_wait attempts.
constexpr uint32_t kWaitSpins = 1u << 24;

// Bounded wait on the phase with the given parity: false if it ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  uint32_t spins = kWaitSpins) {
    for (uint32_t i = 0; i < spins; i++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                 "r"(smem_u32(src)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Waits until every committed bulk store of this thread has read its source.
__device__ __forceinline__ void bulk_wait_read_all() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// Waits until every committed bulk store of this thread is complete.
__device__ __forceinline__ void bulk_wait_all() {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Orders this thread's generic-proxy shared-memory writes before later
// async-proxy (bulk copy) reads of them.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 16-byte asynchronous copy global -> shared (completed by cp_async_wait_all
// of the issuing thread; both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}

struct TileGeom {
    int c, lo, w;  // columns 2^c, rows 2^w at index bits lo .. lo+w-1
    int esz_log;   // log2 of the element size in bytes (3 or 4)
};

__device__ __forceinline__ uint64_t tile_base(const TileGeom &G, uint64_t t) {
    const int mid_bits = G.lo - G.c;
    const uint64_t mid = t & ((1ull << mid_bits) - 1);
    const uint64_t hi = t >> mid_bits;
    return (hi << (G.lo + G.w)) | (mid << G.c);
}

// Issued by one full warp: lane 0 arms the barrier with the tile's bytes, then
// the lanes issue the row copies.
__device__ __forceinline__ void tile_load_issue(const TileGeom &G, const void *gbase, uint64_t t,
                                                void *sbuf, uint64_t *bar, int lane) {
    const uint32_t row_bytes = (1u << G.c) << G.esz_log;
    const uint32_t tile_bytes = row_bytes << G.w;
    const uint64_t base = tile_base(G, t);
    const char *g = static_cast<const char *>(gbase);
    char *s = static_cast<char *>(sbuf);
    if (lane == 0) mbar_arrive_expect_tx(bar, tile_bytes);
    __syncwarp();
    if (G.lo == G.c) {
        if (lane == 0) bulk_g2s(s, g + (base << G.esz_log), tile_bytes, bar);
    } else {
        for (uint32_t r = lane; r < (1u << G.w); r += 32)
            bulk_g2s(s + (size_t)r * row_bytes, g + ((base | ((uint64_t)r << G.lo)) << G.esz_log),
                     row_bytes, bar);
    }
}

// Issued by one full warp after the tile's shared-memory writes are fenced and
// the CTA has synchronised; each lane commits its own bulk group.
__device__ __forceinline__ void tile_store_issue(const TileGeom &G, void *gbase, uint64_t t,
                                                 const void *sbuf, int lane) {
    const uint32_t row_bytes = (1u << G.c) << G.esz_log;
    const uint64_t base = tile_base(G, t);
    char *g = static_cast<char *>(gbase);
    const char *s = static_cast<const char *>(sbuf);
    if (G.lo == G.c) {
        if (lane == 0) bulk_s2g(g + (base << G.esz_log), s, row_bytes << G.w);
    } else {
        for (uint32_t r = lane; r < (1u << G.w); r += 32)
            bulk_s2g(g + ((base | ((uint64_t)r << G.lo)) << G.esz_log), s + (size_t)r * row_bytes,
                     row_bytes);
    }
    bulk_commit();
}

}  // namespace gf2x
