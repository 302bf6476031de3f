// Host launchers of the CUDA kernels (kernels.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "gf2x_internal.h"

namespace gf2x {

struct DevTables;

// One step of a BasisCvt tile pass, in tile-local index bits:
//  kind 0: a run of G <= 3 divisions (a, a - K), a = a_top .. a_top - G + 1;
//  kind 1: the whole BasisCvt of 2 index bits at scale `a_top` (one division);
//  kind 2: the whole BasisCvt of 4 index bits at scale `a_top` (four divisions).
struct BcvtOp {
    int8_t kind, a_top, K, G;
};

// The steps of one tile pass, in the order they are applied (the inverse
// lists them reversed and applies each one inverted).
struct LevelBatch {
    static constexpr int kMax = 48;
    int count;
    BcvtOp op[kMax];
};

// One operand of a product as Split reads it: nw words, the last one masked.
struct OperandDesc {
    const uint64_t *src;
    uint64_t nw;
    uint64_t mask;
};

// The output of a product as InterleavedCombine writes it.
struct OutputDesc {
    uint64_t *out;
    uint64_t words;
    uint64_t mask;
};

// Raises the dynamic shared-memory limit of `func` to `bytes` once per device
// (the attribute is per device context).
void ensure_smem_attr(const void *func, int bytes);

// Streaming multiprocessors of the current device (grid size of the
// persistent kernels).
unsigned num_sms();

// Sets, for the current device, every kernel attribute the launchers would
// otherwise set on first use (so that later launches allocate nothing).
void prepare_bcvt_attributes();
void prepare_fft_attributes();

// Split of `count` operands: product y reads many[y] (or `one` when many is
// null) and writes P words at w + y * stride.
void launch_split_pad(const OperandDesc &one, const OperandDesc *many, int count, uint64_t *w,
                      uint64_t P, uint64_t stride, cudaStream_t s);

// BasisCvt (inverse = 0) or iBasisCvt (inverse = 1) on 2^m coefficients of
// type T (uint64_t or uint4), with the forward level list `fwd`, for `count`
// arrays at f + y * stride.  Returns the number of kernel launches enqueued.
// Shape of the BasisCvt tile passes: the smallest tile (log2 of its
// elements) and the threads of a CTA whose tile is at most 64 KiB.
struct BcvtTune {
    int tile_min_log = 11;
    int small_threads = 256;
};

// changeRepr fused into the last tile pass of a forward BasisCvt of 64-bit
// blocks: that pass writes phi(block) as a 128-bit element to out + y * stride
// (the staged blocks the first strided FFT pass reads) instead of the block
// back in place.
struct PhiOut {
    uint4 *out = nullptr;
    uint64_t stride = 0;
    const DevTables *T = nullptr;
};

// `phi` (forward, 64-bit blocks only): take changeRepr into the last pass if
// that pass is a tile pass; *phi_done tells whether it was (else the blocks are
// converted in place as usual and changeRepr remains to be done).
template <typename T>
uint64_t run_basis_cvt(T *f, int m, const LevelList &fwd, int inverse, cudaStream_t s,
                       int count = 1, uint64_t stride = 0, const BcvtTune &tune = BcvtTune(),
                       const PhiOut *phi = nullptr, bool *phi_done = nullptr);

// changeRepr of the P blocks of `count` operands (product y at g + y * strideW)
// into F + y * strideF, ahead of their first strided FFT pass.
void launch_chrepr_stage(const uint64_t *g, uint64_t P, uint64_t strideW, uint4 *F,
                         uint64_t strideF, int count, const DevTables *T, cudaStream_t s);

void launch_chrepr(const uint64_t *g, uint64_t P, uint4 *F, uint64_t n, const DevTables *T,
                   cudaStream_t s);

// changeRepr^-1 + InterleavedCombine of `count` products: product y reads n
// elements at F + y * stride and writes many[y] (or `one`); max_words bounds
// the output lengths.  Only output words [j_begin, j_end) are written; with
// `accumulate` they are XORed into the output instead of stored.
void launch_ichrepr_combine(const uint4 *F, uint64_t n, uint64_t stride, const OutputDesc &one,
                            const OutputDesc *many, int count, uint64_t max_words,
                            const DevTables *T, cudaStream_t s, uint64_t j_begin = 0,
                            uint64_t j_end = ~0ull, bool accumulate = false);

// Descriptors of the chunked (unbalanced) product: chunk i of the long operand
// x (xw words, last word masked by x_mask) is x + i * L, min(L, xw - i * L)
// words; its product with the short operand (yw words) lands at out + i * L,
// min(chunk_words, out_words - i * L) words (the last one masked by out_mask).
// dx[i] for every chunk; dout holds the even chunks' outputs, then the odd
// ones'.
void launch_chunk_descs(const uint64_t *x, uint64_t xw, uint64_t x_mask, uint64_t L, uint64_t C,
                        uint64_t *out, uint64_t out_words, uint64_t out_mask,
                        uint64_t chunk_words, OperandDesc *dx, OutputDesc *dout, cudaStream_t s);

}  // namespace gf2x
