// Product plans: sizes, BasisCvt level lists, FFT pass schedules, workspace
// layout, and the order of the stages of Alg. 5.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <mutex>

#include "fft_pass.h"
#include "gf2x_dev.cuh"
#include "gf2x_internal.h"
#include "kernels.h"

namespace gf2x {
// Shape parameters of a plan that do not change its results: the FFT fusion
// depth (most layers per strided pass), the strided passes' tile buffering
// and the BasisCvt tile shape.  The
// autotuner (gf2x_autotune) picks them per product shape.
struct PlanTune {
    int fft_depth = 7;
    int fft_nbuf = 2;  // tile buffers of the strided FFT passes (1 or 2)
    BcvtTune bcvt;
};
}  // namespace gf2x

struct gf2x_plan {
    uint64_t na_bits, nb_bits, na_w, nb_w, out_words, total_bits;
    gf2x::PlanTune tune;
    int M, pa_log, pb_log;
    uint64_t N, Pa, Pb;
    gf2x::LevelList lv_a, lv_b, lv_c;
    // FFT pass schedules: forward of a; forward of b whose bottom pass also
    // does pointmul and the bottom inverse layers; the inverse top layers.
    gf2x::PassList fft_a, fft_b, ifft_top;
    gf2x::FftPassCfg fused;
    // workspace layout (bytes): FA | FB | WA | WB | ST (the changeRepr'd blocks
    // of the operand whose first strided pass comes next, max(Pa, Pb) elements,
    // present when a transform has strided passes)
    size_t off_fa, off_fb, off_wa, off_wb, off_st, ws_bytes;
    int device;
    std::mutex mu;
    void *owned_ws = nullptr;
};

namespace gf2x {

constexpr int kMaxLogN = 28;  // FFT points N <= 2^28

// Stage groups timed by the profiling hook (order of gf2x_profile_read).
enum Stage {
    ST_SPLIT, ST_BCVT, ST_CHREPR, ST_FFT_A, ST_FFT_B, ST_FUSED, ST_IFFT, ST_IBCVT, ST_OUT, ST_COUNT
};

struct StageHook {
    virtual void begin(int stage) = 0;
    virtual void end(uint64_t launches) = 0;
    virtual ~StageHook() {}
};

inline uint64_t words_of(uint64_t bits) { return (bits + 63) / 64; }

inline int log2_ceil(uint64_t n) {
    int l = 0;
    while ((1ull << l) < n) l++;
    return l;
}

// Fills *p for operands of na_bits and nb_bits (both > 0).  `src` supplies the
// per-pass device tables (nullptr: the library's cache).  Returns a status.
int plan_init(gf2x_plan *p, uint64_t na_bits, uint64_t nb_bits, PassTableFn src,
              const PlanTune &tune = PlanTune());

// The shape key of a product: (log2 N, log2 Pa, log2 Pb); products with the
// same key share their plan structure and their tuned parameters.
void shape_of(uint64_t na_bits, uint64_t nb_bits, int *M, int *pa_log, int *pb_log);

// Enqueues the whole product on `s` with workspace `ws` (p->ws_bytes bytes,
// 256-byte aligned), tables T and status word `status`; `hook` may be null.
// If b_ready is given, the stages of b start after it (b may still be
// arriving while a is split, converted and transformed).
// If `drain` is given (one product), the output is produced in drain->chunks
// pieces and each piece is copied to drain->host on drain->stream as soon as
// it is written (the copies overlap the rest of the output stage).
struct OutputDrain {
    cudaStream_t stream;
    uint64_t *host;
    int chunks;
    cudaEvent_t *events;  // `chunks` events, owned by the caller
};
int plan_run_core(const gf2x_plan *p, const uint64_t *a, const uint64_t *b, uint64_t *out,
                  void *ws, cudaStream_t s, const DevTables *T, int *status, StageHook *hook,
                  cudaEvent_t b_ready = nullptr, const OutputDrain *drain = nullptr);

// `count` products sharing plan p (same M, log2 Pa, log2 Pb): product y's
// operands and output from many_a[y], many_b[y], many_out[y] (device arrays;
// null = the single `one_*`), its workspace at ws + y * ws_stride;
// max_out_words bounds the outputs' lengths.
int plan_run_batch(const gf2x_plan *p, int count, const OperandDesc *many_a,
                   const OperandDesc *many_b, const OutputDesc *many_out, const OperandDesc &one_a,
                   const OperandDesc &one_b, const OutputDesc &one_out, uint64_t max_out_words,
                   void *ws, size_t ws_stride, cudaStream_t s, const DevTables *T, int *status,
                   StageHook *hook, cudaEvent_t b_ready = nullptr,
                   const OutputDrain *drain = nullptr);

uint64_t mask_of_bits(uint64_t bits);

// The unbalanced product by chunks.  When the long operand x has at least
// four times as many words as the short operand y, x is cut into C chunks of
// L words (L a power of two >= the words of y, at least 512), each chunk is
// multiplied by y with a transform of about 2L points instead of one of about
// xw points, and the chunk products are XORed into the output at i * L.  y is
// converted and transformed once (all layers); every chunk's bottom pass
// multiplies by that one transform.  The chunk plan pc is the plan of y (as
// operand a) times a chunk of 64 L bits (as operand b).
struct ChunkShape {
    uint64_t L = 0, C = 0;
};
bool chunk_shape(uint64_t xw, uint64_t yw, ChunkShape *cs);
size_t chunked_ws_bytes(const gf2x_plan *pc, uint64_t C);
int plan_run_chunked(const gf2x_plan *pc, const ChunkShape &cs, const uint64_t *x,
                     uint64_t x_bits, const uint64_t *y, uint64_t y_bits, uint64_t *out, void *ws,
                     cudaStream_t s, const DevTables *T, int *status, StageHook *hook);

// Host image of the size-independent device tables.
void fill_dev_tables(DevTables *h);

}  // namespace gf2x
