// Fused FFT_LCH passes (fft_pass.cu): configuration and launchers.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "gf2x_dev.cuh"

namespace gf2x {

// One pass: layers k_lo .. k_lo+g-1, tile of 2^g rows x 2^c columns.
struct FftPassCfg {
    int k_lo, g, c;
    int uf;        // tile rows r >= uf have warp-uniform multipliers
    int mode;      // 0 forward, 1 inverse, 2 forward + pointmul + inverse
    int g_f;       // forward layers computed (mode 0/2): rows 0 .. g_f-1
    bool needs_mt; // F~_{2^8} product table in shared memory
    bool low3;     // rows 0-2 in registers with per-lane tables (contiguous
                   // tile of at least 2^8 elements); else product-table layers
    const uint32_t *d_val;   // per-pass multipliers d(k, prefix)
    const uint32_t *d_shfl;  // their warp-shuffle tables (rows r >= uf)
    size_t smem;
    int threads;
    int nbuf;      // tile buffers: 2 (one CTA per SM, next tile loaded while
                   // this one is computed) or 1 (two CTAs per SM take turns)
};

struct FftPassArgs {
    uint4 *F;
    const uint4 *Fsrc;    // non-null: tiles load from Fsrc[idx & pmask] (the fan-out)
    const uint64_t *g64;  // non-null: read changeRepr(g64[idx & pmask]) instead of F
    uint64_t pmask;
    const uint4 *FA;      // mode 2: the other operand's transform
    const DevTables *T;
    const uint32_t *d_val;
    const uint32_t *d_shfl;
    int k_lo, g, c, uf, mode, g_f;
    bool needs_mt, low3;
    int M;        // log2 of the transform length
    int *status;  // device status word (a bounded wait that ran out stores GF2X_ETIMEOUT)
    int count;    // products in the launch: product y at F + y * strideF,
    uint64_t strideF, strideW;  // g64 + y * strideW, FA + y * strideFA
    uint64_t strideFA;          // 0: one transform FA shared by all products
    int nbuf;     // tile buffers (1 or 2)
    uint32_t wait_spins;  // bound of the tile-load waits (try_wait attempts)
};

// A fixed-capacity list of passes (no heap allocation).
struct PassList {
    static constexpr int kMax = 8;
    int n = 0;
    FftPassCfg v[kMax];
};

// Source of the per-pass device tables d(k, prefix) and their shuffle tables
// for a pass (k_lo, g, uf): fills the two device pointers, returns 0 or a
// negative status.  nullptr = the library's own cache (device allocations).
typedef int (*PassTableFn)(int k_lo, int g, int uf, const uint32_t **d_val,
                           const uint32_t **d_shfl);

// Host copy of the tables of pass (k_lo, g, uf): d_val has 2^g - 1 entries,
// d_shfl 224 words per multiplier of the rows r >= uf.
void pass_tables_host(int k_lo, int g, int uf, std::vector<uint32_t> &d_val,
                      std::vector<uint32_t> &d_shfl);
// Words of the two tables of pass (k_lo, g, uf), and a fill into caller
// storage of exactly those sizes (no allocation).
void pass_tables_size(int g, int uf, size_t *n_val, size_t *n_shfl);
void pass_tables_fill(int k_lo, int g, int uf, uint32_t *val, uint32_t *shfl);

// Pass schedules.  Forward: layers [0, log_p) (the layers above log_p are
// fan-outs).  Inverse: all M layers.  Fused: forward of the second operand,
// its bottom pass merged with pointmul and the bottom inverse layers.
// Return 0 or a negative status.
// `depth` = the most layers one strided pass covers (1 .. kFftGlobalMax);
// `nbuf` = tile buffers of the strided passes (1 or 2).
int plan_fft_forward(int M, int log_p, PassList &out, PassTableFn src = nullptr,
                     int depth = 7, int nbuf = 2);
int plan_fft_inverse(int M, PassList &out, PassTableFn src = nullptr, int depth = 7,
                     int nbuf = 2);
int plan_fft_fused(int M, int log_p, PassList &fwd_global, FftPassCfg &local, PassList &inv_global,
                   PassTableFn src = nullptr, int depth = 7, int nbuf = 2);

// Layers of the contiguous bottom pass and of each strided pass.
constexpr int kFftTileLog = 12;
// Dynamic shared memory one CTA may use (227 KiB).
constexpr size_t kMaxPassSmem = 232448;
// First row of a contiguous bottom pass of g layers with warp-uniform
// multipliers: rows 0..2 use the F~_{2^8} product table, rows 3, 4 the
// limb-wise shuffle sub-pass, the rest whole-element shuffle sub-passes.
inline int bottom_uf(int g) { return g >= 5 ? 3 : g; }
constexpr int kFftGlobalMax = 7;  // keeps c = 12 - g >= 5 (warp-uniform multipliers)

int launch_fft_pass(const FftPassCfg &p, int M, uint4 *F, const uint64_t *g64, uint64_t P,
                    const uint4 *FA, const DevTables *T, int *status, cudaStream_t s,
                    int count = 1, uint64_t strideF = 0, uint64_t strideW = 0,
                    const uint4 *Fsrc = nullptr, uint64_t strideFA = ~0ull);

// Bound of the tile-load waits that launches made from now on use, in
// try_wait attempts (negative: the default 2^24; 0: every wait gives up at
// once).  For tests of the timeout path.
void set_wait_spins(int64_t spins);
uint32_t wait_spins();

void launch_pointmul_mt(const uint4 *A, const uint4 *B, uint4 *C, uint64_t n, const DevTables *T,
                        cudaStream_t s);

}  // namespace gf2x
