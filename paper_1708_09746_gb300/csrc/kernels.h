// Host launchers of the CUDA kernels (kernels.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "gf2x_internal.h"

namespace gf2x {

struct DevTables;

// Consecutive BasisCvt levels applied inside one shared-memory tile, grouped
// into runs: run i is the G[i] levels (a, a - K[i]) for a = a_top[i] down to
// a_top[i] - G[i] + 1 (tile-local index bits), listed in the order they are
// applied (the inverse applies each run's levels bottom-up); G <= 3.
struct LevelBatch {
    static constexpr int kMax = 48;
    int count;
    int8_t a_top[kMax];
    int8_t K[kMax];
    int8_t G[kMax];
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
template <typename T>
uint64_t run_basis_cvt(T *f, int m, const LevelList &fwd, int inverse, cudaStream_t s,
                       int count = 1, uint64_t stride = 0);

void launch_chrepr(const uint64_t *g, uint64_t P, uint4 *F, uint64_t n, const DevTables *T,
                   cudaStream_t s);

// changeRepr^-1 + InterleavedCombine of `count` products: product y reads n
// elements at F + y * stride and writes many[y] (or `one`); max_words bounds
// the output lengths.
void launch_ichrepr_combine(const uint4 *F, uint64_t n, uint64_t stride, const OutputDesc &one,
                            const OutputDesc *many, int count, uint64_t max_words,
                            const DevTables *T, cudaStream_t s);

}  // namespace gf2x
