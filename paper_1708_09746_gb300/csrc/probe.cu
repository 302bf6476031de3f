// Throughput probes of the pipes the product path is bound by: warp shuffles
// (shfl.sync.idx, the four-Russians tables of the butterfly multiply), 32-bit
// XORs on the integer ALU, and conflict-free 32-bit shared-memory loads.
//
// One CTA per SM (its shared-memory request leaves room for no second one),
// 32 warps each; every thread runs a fixed number of
// iterations over eight independent chains (so that latency is hidden) and the
// CTA's first thread records the SM clock before and after (clock64, after a
// barrier).  Rate = warp instructions executed on the SM / elapsed SM cycles,
// averaged over the CTAs.  A data-dependent value is written out at the end so
// that no chain is optimised away.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/gf2x_gb300.h"

namespace {

constexpr int kProbeWarps = 32;
constexpr int kProbeIters = 4096;
constexpr int kChains = 8;
constexpr int kProbeSmem = 160 * 1024;  // dynamic shared memory: one CTA per SM

enum Pipe { PIPE_SHFL = 0, PIPE_XOR = 1, PIPE_LDS = 2 };

template <int P>
__global__ void __launch_bounds__(kProbeWarps * 32, 1)
    k_probe(uint64_t *cycles, uint32_t *sink, uint32_t seed) {
    extern __shared__ uint32_t tab[];  // the first 1024 words are used
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) tab[i] = (uint32_t)i * 2654435761u + seed;
    uint32_t v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) v[c] = seed + (uint32_t)(threadIdx.x * kChains + c);
    __syncthreads();
    uint64_t t0 = clock64();
    for (int it = 0; it < kProbeIters; it++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) {
            if (P == PIPE_SHFL) {
                v[c] = __shfl_sync(0xffffffffu, v[c], v[c] + (uint32_t)c);
            } else if (P == PIPE_XOR) {
                // one three-input XOR (lop3 0x96) per step
                asm("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(v[c]) : "r"(lane), "r"(c * 977 + 1));
            } else {
                // lane l reads word (x * 32 + l): always bank l, conflict-free
                v[c] = tab[((v[c] & 31u) << 5) | (uint32_t)lane];
            }
        }
    }
    __syncthreads();
    uint64_t t1 = clock64();
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < kChains; c++) acc ^= v[c];
    if (acc == 0x9e3779b9u) sink[0] = acc;  // keeps the chains live
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

template <int P>
int run_probe(int sms, double *rate) {
    uint64_t *d_cycles = nullptr;
    uint32_t *d_sink = nullptr;
    if (cudaMalloc(&d_cycles, sizeof(uint64_t) * sms) != cudaSuccess) return GF2X_ENOMEM;
    if (cudaMalloc(&d_sink, sizeof(uint32_t)) != cudaSuccess) {
        cudaFree(d_cycles);
        return GF2X_ENOMEM;
    }
    int rc = GF2X_OK;
    if (cudaFuncSetAttribute(reinterpret_cast<const void *>(k_probe<P>),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kProbeSmem) != cudaSuccess)
        rc = GF2X_ECUDA;
    for (int rep = 0; rep < 2 && rc == GF2X_OK; rep++) {  // the first run warms up
        k_probe<P><<<sms, kProbeWarps * 32, kProbeSmem>>>(d_cycles, d_sink, 12345u + rep);
        if (cudaDeviceSynchronize() != cudaSuccess) rc = GF2X_ECUDA;
    }
    std::vector<uint64_t> cyc(sms);
    if (rc == GF2X_OK &&
        cudaMemcpy(cyc.data(), d_cycles, sizeof(uint64_t) * sms, cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = GF2X_ECUDA;
    cudaFree(d_cycles);
    cudaFree(d_sink);
    if (rc != GF2X_OK) {
        cudaGetLastError();
        return rc;
    }
    double sum = 0;
    for (int i = 0; i < sms; i++) sum += (double)cyc[i];
    const double per_sm = (double)kProbeWarps * kProbeIters * kChains;  // warp instructions
    *rate = sum > 0 ? per_sm / (sum / sms) : 0.0;
    return GF2X_OK;
}

}  // namespace

extern "C" {

int gf2x_probe_pipes(double *shfl_per_clk_sm, double *xor_per_clk_sm, double *lds_per_clk_sm,
                     int *sm_count) {
    if (!shfl_per_clk_sm || !xor_per_clk_sm || !lds_per_clk_sm || !sm_count) return GF2X_EINVAL;
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return GF2X_ECUDA;
    }
    *sm_count = prop.multiProcessorCount;
    int rc = run_probe<PIPE_SHFL>(prop.multiProcessorCount, shfl_per_clk_sm);
    if (rc == GF2X_OK) rc = run_probe<PIPE_XOR>(prop.multiProcessorCount, xor_per_clk_sm);
    if (rc == GF2X_OK) rc = run_probe<PIPE_LDS>(prop.multiProcessorCount, lds_per_clk_sm);
    return rc;
}

}  // extern "C"
