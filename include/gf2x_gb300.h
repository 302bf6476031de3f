/*
 * gf2x_gb300.h -- C ABI of the GB300 (sm_103a) library for products of long
 * binary polynomials with the additive FFT of Lin, Chung and Han over a tower
 * field (Chen, Cheng, Kuo, Li, Yang, "Faster Multiplication for Long Binary
 * Polynomials", arXiv:1708.09746).
 *
 * What is computed (Alg. 5 of the paper, binPolyMul): c(x) = a(x) * b(x) in
 * GF(2)[x].  The library splits each operand into 64-bit blocks (Split,
 * Sec. 2.1), converts them to the novelpoly basis (BasisCvt, Alg. 3),
 * maps each block into the tower field F~_{2^128} (changeRepr, Sec. 4.3),
 * evaluates both at N points with FFT_LCH (Alg. 1), multiplies pointwise
 * (pointmul, Sec. 4.1.3), interpolates (iFFT_LCH), converts back (iBasisCvt,
 * changeRepr^-1) and XOR-folds the overlapping 128-bit limbs
 * (InterleavedCombine, Sec. 2.1).  Every step runs in CUDA kernels of this
 * library; there is no CPU fallback: without a usable GPU every call returns
 * GF2X_ECUDA.
 *
 * Conventions shared by every call:
 *  - Polynomials are arrays of uint64_t words, little-endian: bit i of word j
 *    is the coefficient of x^(64 j + i).  An n-bit operand occupies
 *    ceil(n/64) words; bits at positions >= n are ignored on input.
 *  - The product of an na-bit and an nb-bit operand has na+nb-1 bits and
 *    occupies gf2x_out_words(na, nb) words; output bits at positions
 *    >= na+nb-1 are written as 0.  A zero-length operand gives the empty
 *    product (0 words written).
 *  - Unless stated otherwise, data pointers are DEVICE pointers (cudaMalloc,
 *    cudaMallocAsync or PyTorch CUDA tensors) on the current device.  A host
 *    pointer gives GF2X_EINVAL.  The caller owns all buffers and keeps them
 *    alive until the call (or its stream) completes.
 *  - `out` must not overlap `a` or `b` (GF2X_EINVAL).
 *  - Asynchronous calls enqueue kernels on the caller's stream (0 = the
 *    legacy default stream) and return without waiting.
 *  - Device-side failures: every wait inside a kernel is bounded; a wait that
 *    runs out ends the kernel early and records GF2X_ETIMEOUT in a status word
 *    of the call that launched it (its output is then undefined).  Synchronous
 *    calls return it themselves; the asynchronous calls made on one stream
 *    share that stream's word, which gf2x_stream_status reads; a batch and
 *    each server request have their own (gf2x_batch_status,
 *    gf2x_server_wait).
 *  - Every call returns an int status; no C++ exception crosses this ABI.
 *  - Sizes: operands up to 2^33 bits each (N <= 2^28 FFT points); larger
 *    sizes give GF2X_EINVAL.
 */
#ifndef GF2X_GB300_H
#define GF2X_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GF2X_API __attribute__((visibility("default")))
#else
#define GF2X_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *gf2x_stream_t; /* same handle as cudaStream_t */

enum {
    GF2X_OK = 0,
    GF2X_EINVAL = -1,   /* bad argument (size, null, host pointer, overlap) */
    GF2X_ENOMEM = -2,   /* device or host allocation failed */
    GF2X_ECUDA = -3,    /* a CUDA call or kernel launch failed, or no GPU */
    GF2X_ETIMEOUT = -4, /* a bounded wait ran out (a host wait of the server
                           API, or a device wait inside a kernel) */
    GF2X_EBUSY = -5     /* a resource is in use (server slots / budget) */
};

/* Human-readable text for a status code.  Never NULL. */
GF2X_API const char *gf2x_strerror(int status);

/* Words of the product of an na-bit and an nb-bit operand:
 * ceil((na+nb-1)/64), or 0 if either size is 0. */
GF2X_API uint64_t gf2x_out_words(uint64_t na_bits, uint64_t nb_bits);

/* Number of FFT points N of the product as one transform: the smallest power
 * of two >= na_w + nb_w - 1 (at least 2), na_w = ceil(na/64); 0 if either
 * size is 0.  Plans, batches and the server use it; the one-shot calls use it
 * unless gf2x_chunking reports chunks. */
GF2X_API uint64_t gf2x_fft_points(uint64_t na_bits, uint64_t nb_bits);

/* How gf2x_mul / gf2x_mul_async split unbalanced operands (see below): the
 * chunk length of the longer operand in words, the number of chunks and the
 * transform length of one chunk product; all three 0 when the product runs as
 * one transform of gf2x_fft_points points.  Host-only (no GPU needed);
 * GF2X_EINVAL for a null pointer. */
GF2X_API int gf2x_chunking(uint64_t na_bits, uint64_t nb_bits, uint64_t *chunk_words,
                           uint64_t *chunks, uint64_t *chunk_fft_points);

/* How gf2x_mul / gf2x_mul_async compute a product (host-only, no GPU
 * needed): *path = 0 one transform of gf2x_fft_points points; 1 by chunks of
 * the longer operand (gf2x_chunking); 2 directly, without a transform, when
 * the shorter operand has at most 16 words (each product word is a sum of
 * 64 x 64 carry-less word products); 3 by the tail split: when cutting at
 * most 16 words off the operands halves the transform (a word count just
 * above a power of two), the main product of the first *main_a_words and
 * *main_b_words words takes the half-length transform and the products of
 * the cut-off tails by the other operand are added directly
 * (a b = a0 b0 + x^(64 A) a1 b + x^(64 B) a0 b1).  GF2X_EINVAL for a null
 * pointer. */
GF2X_API int gf2x_product_path(uint64_t na_bits, uint64_t nb_bits, int *path,
                               uint64_t *main_a_words, uint64_t *main_b_words);

/* ---- One-shot products ---------------------------------------------------*/

/* c = a * b (Alg. 5).  Synchronous: enqueues on the legacy default stream,
 * allocates its workspace there (stream-ordered) and waits for completion.
 * Unbalanced operands (the longer at least four chunks of L words, L the
 * shorter's word count rounded up to a power of two, at least 512) are
 * multiplied by chunks: every chunk of the longer operand times one transform
 * of the shorter (transforms of about 2L points), the chunk products XORed
 * into the output at their offsets (distributivity; the same c).  A shorter
 * operand of at most 16 words is multiplied directly, and a product just
 * above a power-of-two length by the tail split (gf2x_product_path).
 * gf2x_mul and gf2x_mul_async do this; plans, batches, the server and the
 * host-buffer call use one transform of the whole product. */
GF2X_API int gf2x_mul(const uint64_t *a, uint64_t na_bits, const uint64_t *b,
             uint64_t nb_bits, uint64_t *out);

/* As gf2x_mul, asynchronous on `stream`.  The workspace is allocated and
 * freed stream-ordered on `stream`, from a per-device pool of the library that
 * keeps its memory mapped between calls (released by gf2x_shutdown). */
GF2X_API int gf2x_mul_async(const uint64_t *a, uint64_t na_bits, const uint64_t *b,
                   uint64_t nb_bits, uint64_t *out, gf2x_stream_t stream);

/* As gf2x_mul with HOST buffers a, b, out (pageable or pinned).  The call
 * copies the operands to the device, runs the product and copies the result
 * back on `stream`, and returns after the result is in `out`.  b is copied on
 * a second stream of the library while a is split, converted and transformed
 * (the copies overlap the work only when the host buffers are pinned). */
GF2X_API int gf2x_mul_host(const uint64_t *a_host, uint64_t na_bits,
                  const uint64_t *b_host, uint64_t nb_bits, uint64_t *out_host,
                  gf2x_stream_t stream);

/* ---- Plans (per-size tables and pass schedule, device resident) ---------*/

typedef struct gf2x_plan gf2x_plan; /* opaque, library-owned */

/* Builds the plan for operands of exactly na_bits and nb_bits: the pass
 * schedule of BasisCvt/FFT, the butterfly multiplier tables s_k(alpha)
 * (Sec. 4.4) and the changeRepr tables (Sec. 4.3), uploaded to the current
 * device.  *p receives the plan; free it with gf2x_plan_destroy. */
GF2X_API int gf2x_plan_create(uint64_t na_bits, uint64_t nb_bits, gf2x_plan **p);

/* Device workspace in bytes that gf2x_plan_execute needs (2 x 16 N bytes of
 * FFT arrays plus the padded operands). */
GF2X_API int gf2x_plan_workspace_bytes(const gf2x_plan *p, size_t *bytes);

/* Runs the product with plan p on `stream`.  workspace: a device buffer of at
 * least gf2x_plan_workspace_bytes bytes, 256-byte aligned, or NULL to use a
 * buffer the plan owns (allocated on first use; executions that share it are
 * then serialised by the caller's stream order).  Asynchronous. */
GF2X_API int gf2x_plan_execute(gf2x_plan *p, const uint64_t *a, const uint64_t *b,
                      uint64_t *out, void *workspace, gf2x_stream_t stream);

GF2X_API int gf2x_plan_destroy(gf2x_plan *p);

/* ---- Autotuning --------------------------------------------------------------
 * Plans of one transform shape (log2 N, log2 Pa, log2 Pb) share parameters
 * that change the speed of a product but never its result: the FFT fusion
 * depth (most butterfly layers one strided pass covers, 1 .. 7), the tile
 * buffers of the strided FFT passes (1 or 2) and the shape of the BasisCvt
 * tile passes (log2 of the smallest tile, 4 .. 14, and the threads of a CTA
 * whose tile is at most 64 KiB, 32 .. 512 in steps of 32).  The defaults are
 * 7, 2, 11 and 256.  The table is process-wide, keyed by shape
 * only (the GPUs of one process are taken to be alike); plans made after a
 * change use the new parameters. */
typedef struct {
    int fft_depth;
    int fft_buffers; /* tile buffers of a strided FFT pass: 2 (one CTA per SM
                        loads the next tile while it computes) or 1 (two CTAs
                        per SM take turns) */
    int bcvt_tile_log;
    int bcvt_threads;
    double ms; /* device time of one product measured by gf2x_autotune, or -1 */
} gf2x_tune_t;

/* Times products of this shape on the current device with candidate
 * parameters (the fusion depths that give distinct pass schedules with one
 * and two tile buffers, then the BasisCvt tile shapes with the best of those), `reps` timed runs each after one
 * warm-up (reps <= 0: 3), on operands of the given sizes in scratch buffers
 * the call allocates and frees.  Stores the fastest parameters for the shape
 * and returns them in *best.  Synchronous. */
GF2X_API int gf2x_autotune(uint64_t na_bits, uint64_t nb_bits, int reps,
                           gf2x_tune_t *best);

/* The parameters plans of this shape use (the defaults, ms = -1, if it was
 * never tuned or set). */
GF2X_API int gf2x_tune_get(uint64_t na_bits, uint64_t nb_bits, gf2x_tune_t *out);

/* Sets the parameters of this shape; GF2X_EINVAL if one is out of range. */
GF2X_API int gf2x_tune_set(uint64_t na_bits, uint64_t nb_bits, const gf2x_tune_t *t);

/* Writes the table to a text file (one shape per line), or reads one back
 * (entries merged into the table).  GF2X_EINVAL on a malformed file. */
GF2X_API int gf2x_tune_save(const char *path);
GF2X_API int gf2x_tune_load(const char *path);

/* ---- Batched products -----------------------------------------------------*/

/* count independent products out[i] = a[i] * b[i], of any (uneven) sizes,
 * enqueued on `stream`.  The arrays a, na_bits, b, nb_bits, out are HOST
 * arrays of `count` entries; a[i], b[i], out[i] are device pointers.  Plans
 * per size are cached and reused; workspaces come from one pooled device
 * allocation.  The shape groups run on eight library-owned streams forked
 * from `stream` and joined back into it.  Asynchronous. */
GF2X_API int gf2x_mul_batched(int count, const uint64_t *const *a,
                     const uint64_t *na_bits, const uint64_t *const *b,
                     const uint64_t *nb_bits, uint64_t *const *out,
                     gf2x_stream_t stream);

/* A reusable batch: the size list fixed at creation, the products grouped by
 * transform shape (log2 N, log2 Pa, log2 Pb) so that each group is one launch
 * per kernel, a device workspace of about mem_budget_bytes (0 = 4 GiB) shared
 * by up to eight graph branches (a group that does not fit a branch's share
 * runs in chunks; at least one product's workspace per branch, and fewer
 * branches where the budget holds fewer such workspaces) and, after the first
 * execution, a CUDA graph of the whole batch that later executions replay: it
 * forks into the eight branches, which take the groups (largest first, each to
 * the least loaded branch) side by side, and joins them.  Host arrays of
 * `count` sizes; zero-length products are skipped.  gf2x_batch_workspace_bytes
 * reports the whole device workspace. */
typedef struct gf2x_batch gf2x_batch; /* opaque, library-owned */
GF2X_API int gf2x_batch_create(int count, const uint64_t *na_bits,
                               const uint64_t *nb_bits, size_t mem_budget_bytes,
                               gf2x_batch **out);
GF2X_API int gf2x_batch_workspace_bytes(const gf2x_batch *batch, size_t *bytes);
/* Runs the batch on `stream` with the products' device pointers (host arrays
 * of `count` pointers, same order as at creation).  Asynchronous; a second
 * execution first waits until the previous one has read its descriptors.
 * Only null pointers are rejected here (pointer kinds are not re-checked). */
GF2X_API int gf2x_batch_execute(gf2x_batch *batch, const uint64_t *const *a,
                                const uint64_t *const *b, uint64_t *const *out,
                                gf2x_stream_t stream);
GF2X_API int gf2x_batch_destroy(gf2x_batch *batch);

/* Tunes the batch in batch context: for every group of products that share a
 * transform shape, times the group's own grouped launch with candidate plan
 * parameters (FFT fusion depth and tile buffering, then the BasisCvt tile
 * shape; the same candidates as gf2x_autotune) and keeps the fastest for that
 * group of this batch only (the process-wide table of gf2x_autotune is not
 * changed).  It runs on the operands and outputs of the batch's last
 * execution, which must still be valid (the outputs are rewritten with the
 * same values); GF2X_EINVAL if the batch was never executed.  *ms_before and
 * *ms_after receive the summed device time of the groups with the previous
 * and the chosen parameters.  The next execution captures the graph again. */
GF2X_API int gf2x_batch_tune(gf2x_batch *batch, int reps, double *ms_before, double *ms_after);

/* Waits for the batch's last execution and returns GF2X_ETIMEOUT if a bounded
 * device wait in it ran out (its outputs are then undefined), else GF2X_OK
 * (GF2X_OK too if it was never executed). */
GF2X_API int gf2x_batch_status(gf2x_batch *batch);

/* ---- Serving ----------------------------------------------------------------
 * A server runs products submitted at any time.  A worker thread admits the
 * queued requests in arrival order as execution slots (CUDA streams, at most
 * max_slots) and workspace memory (one device arena of mem_budget_bytes) free
 * up; up to max_batch queued requests of the same transform shape (1 .. 64)
 * are admitted together as one batched launch; admitted work runs
 * concurrently.  max_slots = max_batch = 1 gives a one-at-a-time server.
 * Latency is measured from submission to the moment the worker sees the
 * result complete. */
typedef struct gf2x_server gf2x_server; /* opaque, library-owned */
GF2X_API int gf2x_server_create(size_t mem_budget_bytes, int max_slots,
                                int max_batch, gf2x_server **out);
/* Queues out = a * b (device pointers, kept alive until the ticket is waited
 * for).  GF2X_EINVAL if its workspace can never fit the arena. */
GF2X_API int gf2x_server_submit(gf2x_server *sv, const uint64_t *a,
                                uint64_t na_bits, const uint64_t *b,
                                uint64_t nb_bits, uint64_t *out,
                                uint64_t *ticket);
/* Waits at most timeout_us for the ticket: its status, or GF2X_ETIMEOUT (the
 * ticket stays valid and can be waited for again).  A completed ticket is
 * consumed by the wait that returns its status. */
GF2X_API int gf2x_server_wait(gf2x_server *sv, uint64_t ticket,
                              uint64_t timeout_us);
/* Latency percentiles (ms) of the completed requests and throughput (requests
 * per second from the first submission to the last completion). */
GF2X_API int gf2x_server_stats(gf2x_server *sv, double *p50_ms, double *p99_ms,
                               double *throughput_per_s, uint64_t *completed);
GF2X_API int gf2x_server_reset_stats(gf2x_server *sv);
/* Finishes the queued and running work, then releases the server. */
GF2X_API int gf2x_server_destroy(gf2x_server *sv);

/* ---- Stage entry points (each one row of the method, for checking and
 * profiling one stage alone; all device pointers, asynchronous) ----------*/

/* BasisCvt (Alg. 3, Appendix B) in place on 2^log_n 64-bit coefficients
 * (inverse = 0) or its inverse iBasisCvt (inverse = 1). */
GF2X_API int gf2x_stage_basis_cvt64(uint64_t *f, int log_n, int inverse,
                           gf2x_stream_t stream);

/* The same on 2^log_n 128-bit coefficients stored as (lo, hi) word pairs. */
GF2X_API int gf2x_stage_basis_cvt128(uint64_t *f, int log_n, int inverse,
                            gf2x_stream_t stream);

/* changeRepr (Sec. 4.3): F[i] = phi(g[i mod p]) for i < n, where phi maps a
 * 64-bit block p(z) to p(r) in F~_{2^128}; F holds n (lo, hi) pairs.  The
 * periodic copy is the fan-out of the FFT layers above log2(p) (Fig. 2). */
GF2X_API int gf2x_stage_chrepr(const uint64_t *g, uint64_t p, uint64_t *F, uint64_t n,
                      gf2x_stream_t stream);

/* FFT_LCH (Alg. 1) in place on 2^log_n elements (lo, hi pairs) at the points
 * \bar{i}, i < 2^log_n; only layers k < log_p are computed (the layers above
 * are fan-outs, already applied by gf2x_stage_chrepr).  inverse = 1 runs
 * iFFT_LCH over all layers (log_p ignored). */
GF2X_API int gf2x_stage_fft(uint64_t *F, int log_n, int log_p, int inverse,
                   gf2x_stream_t stream);

/* pointmul: C[i] = A[i] * B[i] in F~_{2^128} for i < n (C may equal B). */
GF2X_API int gf2x_stage_pointmul(const uint64_t *A, const uint64_t *B, uint64_t *C,
                        uint64_t n, gf2x_stream_t stream);

/* changeRepr^-1 and InterleavedCombine: out[j] = lo(psi(F[j])) ^
 * hi(psi(F[j-1])) for j < ceil(total_bits/64), bits >= total_bits cleared;
 * F holds n (lo, hi) pairs (entries past n read as 0). */
GF2X_API int gf2x_stage_ichrepr_combine(const uint64_t *F, uint64_t n, uint64_t *out,
                               uint64_t total_bits, gf2x_stream_t stream);

/* ---- Per-stage timing (the component profile of the paper's Table 4) ----*/

/* on = 1: every later product records a CUDA event before and after each of
 * its stage groups on the stream it runs on: split, basis_cvt, chrepr
 * (changeRepr of the blocks of a transform with strided passes; a transform
 * without them converts in its bottom pass), fft_a (FFT_LCH of a), fft_b (top
 * FFT_LCH layers of b), fft_pointmul_ifft_bottom (bottom FFT layers of b +
 * pointmul + bottom iFFT layers), ifft_top, ibasis_cvt, ichrepr_combine.
 * on = 0 stops. */
GF2X_API int gf2x_profile_enable(int on);

/* Drops recorded events and zeroes the sums. */
GF2X_API int gf2x_profile_reset(void);

/* Waits for the recorded events, then returns for stage index `stage`
 * (0 .. 8, order above) the summed elapsed milliseconds, the number of
 * kernel launches in those stages and the number of stage executions. */
GF2X_API int gf2x_profile_read(int stage, double *ms, uint64_t *launches,
                               uint64_t *calls);

/* Name of stage index `stage`, or "" if out of range. */
GF2X_API const char *gf2x_profile_stage_name(int stage);

/* ---- Pipe throughput probe ------------------------------------------------*/

/* Measures, on the current device, the issue rate of the three instruction
 * kinds the product path is bound by, in warp instructions per SM clock:
 * shfl.sync.idx (the shuffle tables of the butterfly multiply), three-input
 * XOR (lop3) and conflict-free 32-bit shared-memory loads.  One CTA of 32 warps
 * per SM runs eight independent chains of each kind; cycles come from the SM
 * clock.  *sm_count receives the SM count.  Takes a few milliseconds; returns a
 * status. */
GF2X_API int gf2x_probe_pipes(double *shfl_per_clk_sm, double *xor_per_clk_sm,
                              double *lds_per_clk_sm, int *sm_count);

/* ---- Allocation-free product --------------------------------------------*/

/* Scratch the allocation-free product keeps in a static device array on every
 * GPU that loads this library (until the process exits), and the largest
 * transform it accepts: N <= 2^18 points, i.e. na_w + nb_w - 1 <= 2^18 words
 * (for example two operands of 2^23 bits each). */
#define GF2X_NOALLOC_SCRATCH_BYTES (16ull << 20)
#define GF2X_NOALLOC_MAX_FFT_POINTS (1ull << 18)

/* c = a * b, the same result as gf2x_mul, without allocating any device
 * memory: for callers that cannot call cudaMalloc or any other allocator
 * while they multiply (a service whose device memory is all handed to its own
 * pool, a plugin whose host owns every allocation, a latency path on which an
 * allocation would synchronise the device).  The paper has no counterpart;
 * this is a library convenience.  a, b, out: device pointers as for gf2x_mul.
 * The work runs on `stream` and the call waits for that stream before it
 * returns.  The scratch lives in one file-scope device array shared by every
 * call; calls that overlapped on the GPU would race on it, so the library
 * runs them one at a time under a process-wide lock.  The first call on each
 * device looks the static arrays up and copies the tables in with synchronous
 * copies: make it before any stream capture.  Products needing more than
 * GF2X_NOALLOC_MAX_FFT_POINTS points give GF2X_EINVAL; a bounded device wait
 * that ran out gives GF2X_ETIMEOUT. */
GF2X_API int gf2x_mul_noalloc(const uint64_t *a, uint64_t na_bits,
                              const uint64_t *b, uint64_t nb_bits,
                              uint64_t *out, gf2x_stream_t stream);

/* ---- The F~_{2^256} form (w = 128) ----------------------------------------
 * Sec. 4.3 and the F~_{2^256} row of Table 2: the operands are cut into
 * 128-bit blocks, BasisCvt converts the blocks, changeRepr maps each block
 * p(z) into F~_{2^256} = F~_{2^128}[x_8]/(x_8^2 + x_8 + v_127) as p(x_8), the
 * additive FFT runs over N2 = gf2x_tower256_fft_points points of that field
 * (half as many as the F~_{2^128} form), pointmul multiplies general
 * F~_{2^256} elements, and changeRepr^-1 plus the recombination of 128-bit
 * limbs gives the same product c = a * b.  Elements are held as two
 * F~_{2^128} halves (lo, the x_8 coefficient) in two arrays of N2 entries. */

/* N2: the smallest power of two >= the product's number of 128-bit blocks
 * ceil(na/128) + ceil(nb/128) - 1 (at least 2); 0 if either size is 0. */
GF2X_API uint64_t gf2x_tower256_fft_points(uint64_t na_bits, uint64_t nb_bits);

/* c = a * b by the F~_{2^256} form, synchronous on the legacy default stream
 * (same conventions and result as gf2x_mul; N2 <= 2^27, operands up to 2^33
 * bits).  The workspace (4 x 16 N2 bytes plus the padded blocks) comes from
 * the library's stream-ordered pool. */
GF2X_API int gf2x_mul_tower256(const uint64_t *a, uint64_t na_bits, const uint64_t *b,
                               uint64_t nb_bits, uint64_t *out);

/* As gf2x_mul_tower256, asynchronous on `stream` (device-side failures are
 * reported by gf2x_stream_status). */
GF2X_API int gf2x_mul_tower256_async(const uint64_t *a, uint64_t na_bits, const uint64_t *b,
                                     uint64_t nb_bits, uint64_t *out, gf2x_stream_t stream);

/* Stage entry points of the F~_{2^256} form (asynchronous on `stream`, device
 * pointers), for stage-by-stage checks:
 *  - changeRepr: `blocks` holds P 128-bit blocks (P a power of two, 16 bytes
 *    each, little-endian); F receives 2 N2 elements of 16 bytes: F[i] and
 *    F[N2 + i] are the low half and the x_8 coefficient of p_{i mod P}(x_8)
 *    (N2 >= P a power of two: the fan-out of the FFT layers above log2 P).
 *  - pointmul: B[i] := A[i] * B[i] for i < N2, elements split as above.
 *  - changeRepr^-1 + recombination: out receives out_words words of
 *    sum_j psi(e_j) z^(128 j), e_j = F[j] + x_8 F[N2 + j], bits at positions
 *    >= total_bits cleared. */
GF2X_API int gf2x_stage_chrepr256(const void *blocks, uint64_t P, void *F, uint64_t N2,
                                  gf2x_stream_t stream);
GF2X_API int gf2x_stage_pointmul256(const void *A, void *B, uint64_t N2, gf2x_stream_t stream);
GF2X_API int gf2x_stage_ichrepr256_combine(const void *F, uint64_t N2, uint64_t *out,
                                           uint64_t out_words, uint64_t total_bits,
                                           gf2x_stream_t stream);

/* ---- The simple polynomial-basis form (Alg. 4) ---------------------------
 * Sec. 3.1: the working field is the polynomial basis of the AES-GCM field
 * GF(2)[z]/(z^128 + z^7 + z^2 + z + 1), the LCH FFT evaluates at the points
 * phi_beta(i) of a Cantor basis (beta_0 = 1, beta_i^2 + beta_i = beta_{i-1},
 * each beta_i the root with coefficient 0 at z^0), the butterfly multipliers
 * s_k(alpha) = phi_beta(2b) are general field elements, and a 64-bit block is
 * a field element as it stands (no changeRepr).  Every multiplication is a
 * general GF(2^128) product (emulated carry-less multiply and reduction); the
 * form exists to be compared with the tower form, whose butterfly
 * multipliers lie in a small subfield.  Same result as gf2x_mul. */

/* c = a * b by the simple form, synchronous on the legacy default stream
 * (same conventions as gf2x_mul; N <= 2^28 points). */
GF2X_API int gf2x_mul_simple(const uint64_t *a, uint64_t na_bits, const uint64_t *b,
                             uint64_t nb_bits, uint64_t *out);

/* As gf2x_mul_simple, asynchronous on `stream`. */
GF2X_API int gf2x_mul_simple_async(const uint64_t *a, uint64_t na_bits, const uint64_t *b,
                                   uint64_t nb_bits, uint64_t *out, gf2x_stream_t stream);

/* Stage entry points of the simple form (asynchronous, device pointers):
 *  - FFT_LCH (inverse = 0) or its inverse over GF(2^128) in the polynomial
 *    basis on 2^log_n elements of 16 bytes (element i = (lo, hi) 64-bit
 *    words), layers 0 .. layers-1 only (the forward transform of a
 *    polynomial of 2^layers coefficients whose input already repeats them
 *    periodically; layers = log_n for the whole transform);
 *  - the general product B[i] := A[i] * B[i] for i < n. */
GF2X_API int gf2x_stage_fft_simple(void *F, int log_n, int layers, int inverse,
                                   gf2x_stream_t stream);
GF2X_API int gf2x_stage_gfmul_simple(const void *A, void *B, uint64_t n, gf2x_stream_t stream);

/* ---- The Frobenius-partition form (Appendix C) ---------------------------
 * No Kronecker segmentation: a polynomial of degree < 128 n (n = 2^m) is
 * evaluated, its coefficients taken as elements of GF(2^128) (the polynomial
 * basis of the simple form), at the n points beta_{m+64} + V_m of the Cantor
 * basis; this map is a bijection onto GF(2^128)^n (Proposition C.1), so
 * c = a b needs n = 2^m points with 128 n >= na + nb - 1: half as many as the
 * 64-bit Kronecker forms.  The map is a truncated additive FFT: BasisCvt of
 * the one-bit coefficients, an "encoding" of the 128 bits at stride n into one
 * element (the seven truncated layers), and an m-layer FFT whose multipliers
 * are general field elements.  Same result as gf2x_mul. */

/* m, the log2 of the number of points of the product (-1 if a size is 0). */
GF2X_API int gf2x_frobenius_points(uint64_t na_bits, uint64_t nb_bits);

/* c = a * b by the Frobenius-partition form, synchronous on the legacy
 * default stream (same conventions as gf2x_mul; n <= 2^27 points). */
GF2X_API int gf2x_mul_frobenius(const uint64_t *a, uint64_t na_bits, const uint64_t *b,
                                uint64_t nb_bits, uint64_t *out);

/* As gf2x_mul_frobenius, asynchronous on `stream`. */
GF2X_API int gf2x_mul_frobenius_async(const uint64_t *a, uint64_t na_bits, const uint64_t *b,
                                      uint64_t nb_bits, uint64_t *out, gf2x_stream_t stream);

/* Stage entry points of the Frobenius form (asynchronous, device pointers):
 *  - BasisCvt (inverse = 0) or iBasisCvt of 2^log_bits one-bit coefficients
 *    packed little-endian in max(1, 2^(log_bits-6)) words, in place;
 *  - the encoding (decode = 0): E[i] = sum_j g[i + j 2^m] w_j, i < 2^m, over
 *    the 2^log_bits bits of g (log_bits <= m + 7); or its inverse (decode = 1):
 *    the 128 2^m bits of g (written) from the 2^m elements E;
 *  - FFT_LCH (inverse = 0) or its inverse over the 2^m points
 *    beta_{m+64} + phi_beta(i), in place on 2^m elements of 16 bytes. */
GF2X_API int gf2x_stage_bit_basis_cvt(uint64_t *f, int log_bits, int inverse,
                                      gf2x_stream_t stream);
GF2X_API int gf2x_stage_frobenius_encode(const uint64_t *g, int log_bits, int m, void *E,
                                         int decode, gf2x_stream_t stream);
GF2X_API int gf2x_stage_fft_frobenius(void *F, int m, int inverse, gf2x_stream_t stream);

/* ---- Device-side failures ------------------------------------------------*/

/* Waits for `stream` and returns the status of the asynchronous calls made
 * on it since the last gf2x_stream_status of that stream (gf2x_mul_async,
 * gf2x_plan_execute, gf2x_mul_batched): GF2X_ETIMEOUT if a bounded device wait
 * in one of them ran out, else GF2X_OK; the stream's status is then cleared.
 * The library keeps one status word per stream it has seen (up to 512 per
 * device; the calls on further streams share word 0 of the device). */
GF2X_API int gf2x_stream_status(gf2x_stream_t stream);

/* For tests of the timeout path: every bounded device wait of the kernels
 * launched from now on gives up after `spins` attempts (0: at once, without
 * waiting); a negative value restores the default bound (2^24 attempts).  The
 * kernels still let every copy they started land before they exit.  Process-
 * wide; not for production use. */
GF2X_API int gf2x_debug_set_wait_spins(int64_t spins);

/* Releases the per-device tables and cached plans of this library. */
GF2X_API int gf2x_shutdown(void);

#ifdef __cplusplus
}
#endif

#endif /* GF2X_GB300_H */
