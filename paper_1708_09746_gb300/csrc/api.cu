// The C ABI (include/gf2x_gb300.h): argument checks, per-device tables,
// plans and the order of the stages of Alg. 5.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/gf2x_gb300.h"
#include "gf2x_dev.cuh"
#include "gf2x_internal.h"
#include "fft_pass.h"
#include "kernels.h"
#include "api_internal.h"
#include "plan.h"
#include "small.h"

using namespace gf2x;

namespace {

// ---- Per-device context: the size-independent tables, uploaded once. ------
//
// Status words: a kernel that gives up a bounded wait writes GF2X_ETIMEOUT to
// the status word it was launched with.  Each device has one array of
// kStatusWords such words: word 0 belongs to the stage entry points; a
// synchronous call (gf2x_mul, gf2x_mul_host) takes a free word for its own
// duration; the asynchronous calls made on one stream share a word of that
// stream (read and cleared by gf2x_stream_status); each server slot owns one.
// So a timeout is reported to the call, stream or request that caused it.
constexpr int kStatusWords = 1024;

struct DeviceCtx {
    DevTables *tables = nullptr;
    int *status = nullptr;  // kStatusWords device status words
    std::vector<int> free_words;                // unused word indices (>= 1)
    std::map<cudaStream_t, int> stream_words;   // stream -> its word
    // Workspace pool: keeps its memory mapped between products (release
    // threshold at the maximum), so that a product does not map and unmap the
    // pages of its workspace every time.
    cudaMemPool_t pool = nullptr;
    cudaStream_t copy_stream = nullptr;  // second operand's upload in gf2x_mul_host
};

std::mutex g_ctx_mu;
std::map<int, DeviceCtx> g_ctx;

int current_device(int *dev) {
    cudaError_t e = cudaGetDevice(dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GF2X_ECUDA;
    }
    return GF2X_OK;
}

int get_tables(const DevTables **out) {
    int dev;
    int rc = current_device(&dev);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_ctx_mu);
    DeviceCtx &c = g_ctx[dev];
    if (!c.tables) {
        std::unique_ptr<DevTables> h(new (std::nothrow) DevTables);
        if (!h) return GF2X_ENOMEM;
        fill_dev_tables(h.get());
        DevTables *d = nullptr;
        if (cudaMalloc(&d, sizeof(DevTables)) != cudaSuccess) {
            cudaGetLastError();
            return GF2X_ENOMEM;
        }
        if (cudaMemcpy(d, h.get(), sizeof(DevTables), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(d);
            return GF2X_ECUDA;
        }
        int *st = nullptr;
        if (cudaMalloc(&st, kStatusWords * sizeof(int)) != cudaSuccess ||
            cudaMemset(st, 0, kStatusWords * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(d);
            if (st) cudaFree(st);
            return GF2X_ENOMEM;
        }
        c.tables = d;
        c.status = st;
        c.free_words.clear();
        for (int i = kStatusWords - 1; i >= 1; i--) c.free_words.push_back(i);
        c.stream_words.clear();
    }
    *out = c.tables;
    return GF2X_OK;
}

// The workspace pool and the copy stream of the current device, created on
// first use.
int device_pool(cudaMemPool_t *pool, cudaStream_t *copy_stream) {
    int dev;
    int rc = current_device(&dev);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_ctx_mu);
    DeviceCtx &c = g_ctx[dev];
    if (!c.pool) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pl = nullptr;
        if (cudaMemPoolCreate(&pl, &props) != cudaSuccess) {
            cudaGetLastError();
            return GF2X_ECUDA;
        }
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(pl, cudaMemPoolAttrReleaseThreshold, &keep);
        cudaStream_t cs = nullptr;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            cudaMemPoolDestroy(pl);
            return GF2X_ECUDA;
        }
        c.pool = pl;
        c.copy_stream = cs;
    }
    if (pool) *pool = c.pool;
    if (copy_stream) *copy_stream = c.copy_stream;
    return GF2X_OK;
}

// Stream-ordered workspace from the device's pool.
int ws_alloc(void **p, size_t bytes, cudaStream_t s) {
    cudaMemPool_t pool;
    int rc = device_pool(&pool, nullptr);
    if (rc) return rc;
    if (cudaMallocFromPoolAsync(p, bytes ? bytes : 256, pool, s) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return GF2X_ENOMEM;
    }
    return GF2X_OK;
}

void ws_free(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

// Word 0 of the current device: the stage entry points' status word (valid
// after get_tables).
int *device_status() {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_ctx_mu);
    return g_ctx[dev].status;
}

// Reads and clears one status word.  The caller has waited for the work that
// writes it.
int read_clear_status(int *st) {
    if (!st) return GF2X_OK;
    int v = 0;
    if (cudaMemcpy(&v, st, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return GF2X_ECUDA;
    }
    if (v && cudaMemset(st, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return GF2X_ECUDA;
    }
    return v;
}

// Reads and clears word 0 after the whole device has finished.
int take_device_status() {
    int *st = device_status();
    if (!st) return GF2X_OK;
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return GF2X_ECUDA;
    }
    return read_clear_status(st);
}

// A free status word of the current device for one call (GF2X_EBUSY when all
// are in use); give it back with give_status_word once its work has finished.
int take_status_word(int **w) {
    const DevTables *T;
    int rc = get_tables(&T);
    if (rc) return rc;
    int dev = 0;
    if ((rc = current_device(&dev))) return rc;
    std::lock_guard<std::mutex> lk(g_ctx_mu);
    DeviceCtx &c = g_ctx[dev];
    if (c.free_words.empty()) return GF2X_EBUSY;
    *w = c.status + c.free_words.back();
    c.free_words.pop_back();
    return GF2X_OK;
}

void give_status_word(int *w) {
    if (!w) return;
    std::lock_guard<std::mutex> lk(g_ctx_mu);
    for (auto &kv : g_ctx) {
        DeviceCtx &c = kv.second;
        if (c.status && w > c.status && w < c.status + kStatusWords) {
            c.free_words.push_back((int)(w - c.status));
            return;
        }
    }
}

// The status word of the asynchronous calls on stream s of the current device
// (taken on first use and kept; when no word is free, word 0).
int *stream_status_word(cudaStream_t s) {
    const DevTables *T;
    if (get_tables(&T)) return nullptr;
    int dev = 0;
    if (current_device(&dev)) return nullptr;
    std::lock_guard<std::mutex> lk(g_ctx_mu);
    DeviceCtx &c = g_ctx[dev];
    auto it = c.stream_words.find(s);
    if (it != c.stream_words.end()) return c.status + it->second;
    // keep half the words for the synchronous calls and the server slots
    if ((int)c.stream_words.size() >= kStatusWords / 2 || c.free_words.empty()) return c.status;
    const int i = c.free_words.back();
    c.free_words.pop_back();
    c.stream_words[s] = i;
    return c.status + i;
}

int check_launch() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GF2X_OK : GF2X_ECUDA;
}

// Device memory of the current device, or managed memory?  A null pointer is
// accepted only for size 0.
int check_dev_ptr(const void *p, size_t bytes) {
    if (bytes == 0) return GF2X_OK;
    if (!p) return GF2X_EINVAL;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GF2X_EINVAL;
    }
    if (at.type == cudaMemoryTypeManaged) return GF2X_OK;
    if (at.type != cudaMemoryTypeDevice) return GF2X_EINVAL;
    // device memory of another GPU: the kernels run on the current device and
    // would reach it only through peer access, so it is refused
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return GF2X_ECUDA;
    }
    return at.device == dev ? GF2X_OK : GF2X_EINVAL;
}

bool overlap(const void *a, size_t na, const void *b, size_t nb) {
    if (!na || !nb) return false;
    auto x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}


// ---- Per-stage timing (the component profile of Table 4) -------------------
// When enabled, plan_run records a CUDA event before and after each stage on
// the stream it runs on; gf2x_profile_read waits for the events and sums the
// elapsed times per stage.
const char *kStageNames[ST_COUNT] = {"split",      "basis_cvt", "chrepr",
                                     "fft_a",      "fft_b",     "fft_pointmul_ifft_bottom",
                                     "ifft_top",   "ibasis_cvt", "ichrepr_combine"};

struct ProfRec {
    int stage;
    cudaEvent_t a, b;
    uint64_t launches;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof_pending;
double g_prof_ms[ST_COUNT];
uint64_t g_prof_launches[ST_COUNT];
uint64_t g_prof_calls[ST_COUNT];

struct StageTimer : StageHook {
    cudaStream_t s;
    bool on;
    int stage = -1;
    cudaEvent_t a = nullptr;
    explicit StageTimer(cudaStream_t s_) : s(s_) {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        on = g_prof_on;
    }
    void begin(int st) override {
        if (!on) return;
        stage = st;
        cudaEventCreate(&a);
        cudaEventRecord(a, s);
    }
    void end(uint64_t launches) override {
        if (!on || stage < 0) return;
        cudaEvent_t b;
        cudaEventCreate(&b);
        cudaEventRecord(b, s);
        std::lock_guard<std::mutex> lk(g_prof_mu);
        g_prof_pending.push_back(ProfRec{stage, a, b, launches});
        stage = -1;
    }
};

}  // namespace

// ---- Plans ------------------------------------------------------------------
namespace {

// ---- Tuning table: shape (log2 N, log2 Pa, log2 Pb) -> plan parameters ------
struct TuneEntry {
    PlanTune t;
    double ms = -1;
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, TuneEntry> g_tune;

std::tuple<int, int, int> shape_key(uint64_t na_bits, uint64_t nb_bits) {
    int M, pa, pb;
    shape_of(na_bits, nb_bits, &M, &pa, &pb);
    return std::make_tuple(M, pa, pb);
}

TuneEntry tune_for(uint64_t na_bits, uint64_t nb_bits) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(shape_key(na_bits, nb_bits));
    return it == g_tune.end() ? TuneEntry() : it->second;
}

bool tune_valid(const gf2x_tune_t &t) {
    return t.fft_depth >= 1 && t.fft_depth <= kFftGlobalMax && (t.fft_buffers == 1 || t.fft_buffers == 2) &&
           t.bcvt_tile_log >= 4 &&
           t.bcvt_tile_log <= 14 && t.bcvt_threads >= 32 && t.bcvt_threads <= 512 &&
           t.bcvt_threads % 32 == 0;
}

PlanTune from_abi(const gf2x_tune_t &t) {
    PlanTune p;
    p.fft_depth = t.fft_depth;
    p.fft_nbuf = t.fft_buffers;
    p.bcvt.tile_min_log = t.bcvt_tile_log;
    p.bcvt.small_threads = t.bcvt_threads;
    return p;
}

gf2x_tune_t to_abi(const TuneEntry &e) {
    gf2x_tune_t t;
    t.fft_depth = e.t.fft_depth;
    t.fft_buffers = e.t.fft_nbuf;
    t.bcvt_tile_log = e.t.bcvt.tile_min_log;
    t.bcvt_threads = e.t.bcvt.small_threads;
    t.ms = e.ms;
    return t;
}

void drop_cached_plans_of(const std::tuple<int, int, int> &key);

void tune_store(const std::tuple<int, int, int> &key, const TuneEntry &e) {
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = e;
    }
    drop_cached_plans_of(key);
}

int plan_init(gf2x_plan *p, uint64_t na_bits, uint64_t nb_bits, const PlanTune *tune = nullptr) {
    const PlanTune t = tune ? *tune : tune_for(na_bits, nb_bits).t;
    int rc = gf2x::plan_init(p, na_bits, nb_bits, nullptr, t);
    if (rc == -1) return GF2X_EINVAL;
    if (rc == -2) return GF2X_ENOMEM;
    return rc ? GF2X_ECUDA : GF2X_OK;
}

// Alg. 5, stage after stage, on `s`, with the library's tables.
int plan_run(const gf2x_plan *p, const uint64_t *a, const uint64_t *b, uint64_t *out, void *ws,
             cudaStream_t s, int *st, cudaEvent_t b_ready = nullptr,
             const OutputDrain *drain = nullptr) {
    const DevTables *T;
    int rc = get_tables(&T);
    if (rc) return rc;
    StageTimer tm(s);
    rc = plan_run_core(p, a, b, out, ws, s, T, st, &tm, b_ready, drain);
    return rc ? GF2X_ECUDA : GF2X_OK;
}

// Plan cache for the one-shot calls, keyed by (device, sizes).
std::mutex g_cache_mu;
std::map<std::tuple<int, uint64_t, uint64_t>, std::shared_ptr<gf2x_plan>> g_cache;

void drop_cached_plans_of(const std::tuple<int, int, int> &key) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    for (auto it = g_cache.begin(); it != g_cache.end();) {
        if (shape_key(std::get<1>(it->first), std::get<2>(it->first)) == key)
            it = g_cache.erase(it);
        else
            ++it;
    }
}

int cached_plan(uint64_t na_bits, uint64_t nb_bits, std::shared_ptr<gf2x_plan> *out) {
    int dev;
    int rc = current_device(&dev);
    if (rc) return rc;
    auto key = std::make_tuple(dev, na_bits, nb_bits);
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
        *out = it->second;
        return GF2X_OK;
    }
    auto p = std::make_shared<gf2x_plan>();
    rc = plan_init(p.get(), na_bits, nb_bits);
    if (rc) return rc;
    if (g_cache.size() >= 256) g_cache.clear();
    g_cache[key] = p;
    *out = p;
    return GF2X_OK;
}

int check_sizes(uint64_t na_bits, uint64_t nb_bits) {
    if (na_bits > (1ull << 33) || nb_bits > (1ull << 33)) return GF2X_EINVAL;
    return GF2X_OK;
}

int check_operands(const uint64_t *a, uint64_t na_bits, const uint64_t *b, uint64_t nb_bits,
                   const uint64_t *out) {
    int rc = check_sizes(na_bits, nb_bits);
    if (rc) return rc;
    size_t ba = 8 * words_of(na_bits), bb = 8 * words_of(nb_bits);
    size_t bo = 8 * gf2x_out_words(na_bits, nb_bits);
    if ((rc = check_dev_ptr(a, ba))) return rc;
    if ((rc = check_dev_ptr(b, bb))) return rc;
    if ((rc = check_dev_ptr(out, bo))) return rc;
    if (overlap(out, bo, a, ba) || overlap(out, bo, b, bb)) return GF2X_EINVAL;
    return GF2X_OK;
}

// Unbalanced operands: the product by chunks of the long operand against one
// transform of the short one (plan_run_chunked).
int mul_chunked(const uint64_t *x, uint64_t x_bits, const uint64_t *y, uint64_t y_bits,
                uint64_t *out, const ChunkShape &cs, cudaStream_t s, int *st) {
    std::shared_ptr<gf2x_plan> pc;
    int rc = cached_plan(y_bits, 64 * cs.L, &pc);
    if (rc) return rc;
    const DevTables *T;
    if ((rc = get_tables(&T))) return rc;
    void *ws = nullptr;
    if ((rc = ws_alloc(&ws, chunked_ws_bytes(pc.get(), cs.C), s))) return rc;
    StageTimer tm(s);
    rc = plan_run_chunked(pc.get(), cs, x, x_bits, y, y_bits, out, ws, s, T, st, &tm);
    ws_free(ws, s);
    if (rc) return GF2X_ECUDA;
    return check_launch();
}

// A product just above a power-of-two word count: a0 b0 with half the
// transform, plus the tail products by the direct kernel (small.cu).
int mul_tails(const uint64_t *a, uint64_t na_bits, const uint64_t *b, uint64_t nb_bits,
              uint64_t *out, uint64_t A, uint64_t B, cudaStream_t s, int *st) {
    const uint64_t aw = words_of(na_bits), bw = words_of(nb_bits);
    const uint64_t a0_bits = A < aw ? 64 * A : na_bits, b0_bits = B < bw ? 64 * B : nb_bits;
    const uint64_t ow = gf2x_out_words(na_bits, nb_bits), mw = gf2x_out_words(a0_bits, b0_bits);
    std::shared_ptr<gf2x_plan> p;
    int rc = cached_plan(a0_bits, b0_bits, &p);
    if (rc) return rc;
    void *ws = nullptr;
    if ((rc = ws_alloc(&ws, p->ws_bytes, s))) return rc;
    rc = plan_run(p.get(), a, b, out, ws, s, st);
    ws_free(ws, s);
    if (rc) return rc;
    if (ow > mw && cudaMemsetAsync(out + mw, 0, 8 * (ow - mw), s) != cudaSuccess) {
        cudaGetLastError();
        return GF2X_ECUDA;
    }
    // a1 b at word A, a0 b1 at word B
    if (A < aw) launch_mul_small(b, nb_bits, a + A, na_bits - 64 * A, out, ow, A, true, s);
    if (B < bw) launch_mul_small(a, a0_bits, b + B, nb_bits - 64 * B, out, ow, B, true, s);
    return check_launch();
}

// Which way the one-shot calls compute a product: 0 one transform, 1 chunks
// of the longer operand, 2 direct (a short operand), 3 tail split.
int product_path(uint64_t na_bits, uint64_t nb_bits, ChunkShape *cs, uint64_t *A, uint64_t *B) {
    const uint64_t aw = words_of(na_bits), bw = words_of(nb_bits);
    if (std::min(aw, bw) <= (uint64_t)kSmallWords) return 2;
    if (chunk_shape(aw, bw, cs) || chunk_shape(bw, aw, cs)) return 1;
    if (tail_split(aw, bw, A, B)) return 3;
    return 0;
}

int mul_on_stream(const uint64_t *a, uint64_t na_bits, const uint64_t *b, uint64_t nb_bits,
                  uint64_t *out, cudaStream_t s, int *st) {
    {
        const uint64_t aw = words_of(na_bits), bw = words_of(nb_bits);
        if (std::min(aw, bw) <= (uint64_t)kSmallWords) {
            const uint64_t ow = gf2x_out_words(na_bits, nb_bits);
            if (bw <= aw)
                launch_mul_small(a, na_bits, b, nb_bits, out, ow, 0, false, s);
            else
                launch_mul_small(b, nb_bits, a, na_bits, out, ow, 0, false, s);
            return check_launch();
        }
    }
    ChunkShape cs;
    if (chunk_shape(words_of(na_bits), words_of(nb_bits), &cs))
        return mul_chunked(a, na_bits, b, nb_bits, out, cs, s, st);
    if (chunk_shape(words_of(nb_bits), words_of(na_bits), &cs))
        return mul_chunked(b, nb_bits, a, na_bits, out, cs, s, st);
    uint64_t A = 0, B = 0;
    if (tail_split(words_of(na_bits), words_of(nb_bits), &A, &B))
        return mul_tails(a, na_bits, b, nb_bits, out, A, B, s, st);
    std::shared_ptr<gf2x_plan> p;
    int rc = cached_plan(na_bits, nb_bits, &p);
    if (rc) return rc;
    void *ws = nullptr;
    if ((rc = ws_alloc(&ws, p->ws_bytes, s))) return rc;
    rc = plan_run(p.get(), a, b, out, ws, s, st);
    ws_free(ws, s);
    if (rc == GF2X_OK) rc = check_launch();
    return rc;
}

}  // namespace

// Entry points shared with the batch and server modules.
namespace gf2x {
namespace api {
int tables(const DevTables **T) { return get_tables(T); }
int *stream_status(cudaStream_t s) { return stream_status_word(s); }
int take_status(int **w) { return take_status_word(w); }
void give_status(int *w) { give_status_word(w); }
int read_status(int *w) { return read_clear_status(w); }
int plan_for(uint64_t na_bits, uint64_t nb_bits, std::shared_ptr<gf2x_plan> *p) {
    return cached_plan(na_bits, nb_bits, p);
}
int check_product_args(const uint64_t *a, uint64_t na_bits, const uint64_t *b, uint64_t nb_bits,
                       const uint64_t *out) {
    return check_operands(a, na_bits, b, nb_bits, out);
}
StageHook *new_timer(cudaStream_t s) { return new StageTimer(s); }
int ws_alloc(void **p, size_t bytes, cudaStream_t s) { return ::ws_alloc(p, bytes, s); }
void ws_free(void *p, cudaStream_t s) { ::ws_free(p, s); }
int make_plan(uint64_t na_bits, uint64_t nb_bits, const PlanTune &t,
              std::shared_ptr<gf2x_plan> *out) {
    auto p = std::make_shared<gf2x_plan>();
    int rc = ::plan_init(p.get(), na_bits, nb_bits, &t);
    if (rc) return rc;
    *out = p;
    return GF2X_OK;
}
int run_one(const gf2x_plan *p, const uint64_t *a, const uint64_t *b, uint64_t *out, void *ws,
            cudaStream_t s) {
    return plan_run(p, a, b, out, ws, s, stream_status_word(s));
}
}  // namespace api
}  // namespace gf2x

extern "C" {

const char *gf2x_strerror(int status) {
    switch (status) {
        case GF2X_OK: return "ok";
        case GF2X_EINVAL: return "invalid argument";
        case GF2X_ENOMEM: return "out of memory";
        case GF2X_ECUDA: return "CUDA error (or no usable GPU)";
        case GF2X_ETIMEOUT: return "timed out";
        case GF2X_EBUSY: return "busy";
        default: return "unknown status";
    }
}

uint64_t gf2x_out_words(uint64_t na_bits, uint64_t nb_bits) {
    if (!na_bits || !nb_bits) return 0;
    return words_of(na_bits + nb_bits - 1);
}

uint64_t gf2x_fft_points(uint64_t na_bits, uint64_t nb_bits) {
    if (!na_bits || !nb_bits) return 0;
    uint64_t need = std::max<uint64_t>(2, words_of(na_bits) + words_of(nb_bits) - 1);
    return 1ull << log2_ceil(need);
}

int gf2x_chunking(uint64_t na_bits, uint64_t nb_bits, uint64_t *chunk_words, uint64_t *chunks,
                  uint64_t *chunk_fft_points) {
    if (!chunk_words || !chunks || !chunk_fft_points) return GF2X_EINVAL;
    *chunk_words = *chunks = *chunk_fft_points = 0;
    if (!na_bits || !nb_bits) return GF2X_OK;
    const uint64_t na_w = words_of(na_bits), nb_w = words_of(nb_bits);
    if (std::min(na_w, nb_w) <= (uint64_t)kSmallWords) return GF2X_OK;  // direct product
    ChunkShape cs;
    uint64_t yw;
    if (chunk_shape(na_w, nb_w, &cs))
        yw = nb_w;
    else if (chunk_shape(nb_w, na_w, &cs))
        yw = na_w;
    else
        return GF2X_OK;
    *chunk_words = cs.L;
    *chunks = cs.C;
    *chunk_fft_points = 1ull << log2_ceil(std::max<uint64_t>(2, yw + cs.L - 1));
    return GF2X_OK;
}

int gf2x_product_path(uint64_t na_bits, uint64_t nb_bits, int *path, uint64_t *main_a_words,
                      uint64_t *main_b_words) {
    if (!path || !main_a_words || !main_b_words) return GF2X_EINVAL;
    *path = 0;
    *main_a_words = words_of(na_bits);
    *main_b_words = words_of(nb_bits);
    if (!na_bits || !nb_bits) return GF2X_OK;
    ChunkShape cs;
    uint64_t A = 0, B = 0;
    *path = product_path(na_bits, nb_bits, &cs, &A, &B);
    if (*path == 3) {
        *main_a_words = A;
        *main_b_words = B;
    }
    return GF2X_OK;
}

int gf2x_mul_async(const uint64_t *a, uint64_t na_bits, const uint64_t *b, uint64_t nb_bits,
                   uint64_t *out, gf2x_stream_t stream) {
    try {
        int rc = check_operands(a, na_bits, b, nb_bits, out);
        if (rc) return rc;
        if (!na_bits || !nb_bits) return GF2X_OK;
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        int *st = stream_status_word(s);
        if (!st) return GF2X_ECUDA;
        return mul_on_stream(a, na_bits, b, nb_bits, out, s, st);
    } catch (const std::bad_alloc &) {
        return GF2X_ENOMEM;
    } catch (...) {
        return GF2X_ECUDA;
    }
}

int gf2x_mul(const uint64_t *a, uint64_t na_bits, const uint64_t *b, uint64_t nb_bits,
             uint64_t *out) {
    try {
        int rc = check_operands(a, na_bits, b, nb_bits, out);
        if (rc) return rc;
        if (!na_bits || !nb_bits) return GF2X_OK;
        // a status word of this call's own, so that a timeout is reported
        // here and nowhere else
        int *st = nullptr;
        if ((rc = take_status_word(&st))) return rc;
        if (cudaMemsetAsync(st, 0, sizeof(int), 0) != cudaSuccess) {
            cudaGetLastError();
            give_status_word(st);
            return GF2X_ECUDA;
        }
        rc = mul_on_stream(a, na_bits, b, nb_bits, out, nullptr, st);
        if (cudaStreamSynchronize(0) != cudaSuccess) {
            cudaGetLastError();
            rc = GF2X_ECUDA;
        }
        const int ds = read_clear_status(st);
        give_status_word(st);
        return rc ? rc : ds;
    } catch (const std::bad_alloc &) {
        return GF2X_ENOMEM;
    } catch (...) {
        return GF2X_ECUDA;
    }
}

// Pieces of the product copied back while the rest is computed: the copy of
// piece i starts as soon as the recombination has written it.
#ifndef GF2X_HOST_PIECES
#define GF2X_HOST_PIECES 4
#endif

int gf2x_mul_host(const uint64_t *a_host, uint64_t na_bits, const uint64_t *b_host,
                  uint64_t nb_bits, uint64_t *out_host, gf2x_stream_t stream) {
    try {
        int rc = check_sizes(na_bits, nb_bits);
        if (rc) return rc;
        if (!na_bits || !nb_bits) return GF2X_OK;
        if (!a_host || !b_host || !out_host) return GF2X_EINVAL;
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        size_t ba = 8 * words_of(na_bits), bb = 8 * words_of(nb_bits);
        size_t bo = 8 * gf2x_out_words(na_bits, nb_bits);
        if (overlap(out_host, bo, a_host, ba) || overlap(out_host, bo, b_host, bb)) return GF2X_EINVAL;
        std::shared_ptr<gf2x_plan> p;
        if ((rc = cached_plan(na_bits, nb_bits, &p))) return rc;
        cudaStream_t cs;
        if ((rc = device_pool(nullptr, &cs))) return rc;
        char *buf = nullptr;
        size_t total = p->ws_bytes + ((ba + 255) & ~255ull) + ((bb + 255) & ~255ull) + bo;
        if ((rc = ws_alloc(reinterpret_cast<void **>(&buf), total, s))) return rc;
        uint64_t *da = reinterpret_cast<uint64_t *>(buf + p->ws_bytes);
        uint64_t *db = reinterpret_cast<uint64_t *>(buf + p->ws_bytes + ((ba + 255) & ~255ull));
        uint64_t *dout = reinterpret_cast<uint64_t *>(buf + p->ws_bytes + ((ba + 255) & ~255ull) +
                                                      ((bb + 255) & ~255ull));
        // b is uploaded on the copy stream while a is split, converted and
        // transformed on s; the product path waits for it before Split(b).
        // The output is written in pieces, each copied back on the copy
        // stream while the next one is computed.
        constexpr int kPieces = GF2X_HOST_PIECES;
        cudaEvent_t ev[kPieces + 3] = {};
        bool ev_ok = true;
        for (auto &e : ev) ev_ok = ev_ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
        if (!ev_ok) {
            cudaGetLastError();
            for (auto &e : ev)
                if (e) cudaEventDestroy(e);
            ws_free(buf, s);
            return GF2X_ECUDA;
        }
        cudaEvent_t alloc_done = ev[kPieces], b_ready = ev[kPieces + 1], drained = ev[kPieces + 2];
        int *st = nullptr;
        if ((rc = take_status_word(&st))) {
            for (auto &x : ev) cudaEventDestroy(x);
            ws_free(buf, s);
            return rc;
        }
        cudaMemsetAsync(st, 0, sizeof(int), s);
        // a first, alone on the link; b after it, while a is being processed
        cudaMemcpyAsync(da, a_host, ba, cudaMemcpyHostToDevice, s);
        cudaEventRecord(alloc_done, s);
        cudaStreamWaitEvent(cs, alloc_done, 0);
        cudaMemcpyAsync(db, b_host, bb, cudaMemcpyHostToDevice, cs);
        cudaEventRecord(b_ready, cs);
        const OutputDrain drain{cs, out_host, kPieces, ev};
        rc = plan_run(p.get(), da, db, dout, buf, s, st, b_ready, &drain);
        cudaEventRecord(drained, cs);
        cudaStreamWaitEvent(s, drained, 0);  // the copies have read the buffer
        ws_free(buf, s);
        cudaError_t e = cudaStreamSynchronize(s);
        for (auto &x : ev) cudaEventDestroy(x);
        const int ds = e == cudaSuccess ? read_clear_status(st) : GF2X_ECUDA;
        give_status_word(st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return GF2X_ECUDA;
        }
        return rc ? rc : ds;
    } catch (const std::bad_alloc &) {
        return GF2X_ENOMEM;
    } catch (...) {
        return GF2X_ECUDA;
    }
}

int gf2x_plan_create(uint64_t na_bits, uint64_t nb_bits, gf2x_plan **out) {
    if (!out) return GF2X_EINVAL;
    *out = nullptr;
    try {
        int rc = check_sizes(na_bits, nb_bits);
        if (rc) return rc;
        if (!na_bits || !nb_bits) return GF2X_EINVAL;
        const DevTables *T;
        if ((rc = get_tables(&T))) return rc;
        gf2x_plan *p = new (std::nothrow) gf2x_plan();
        if (!p) return GF2X_ENOMEM;
        rc = plan_init(p, na_bits, nb_bits);
        if (rc) {
            delete p;
            return rc;
        }
        *out = p;
        return GF2X_OK;
    } catch (const std::bad_alloc &) {
        return GF2X_ENOMEM;
    } catch (...) {
        return GF2X_ECUDA;
    }
}

int gf2x_plan_workspace_bytes(const gf2x_plan *p, size_t *bytes) {
    if (!p || !bytes) return GF2X_EINVAL;
    *bytes = p->ws_bytes;
    return GF2X_OK;
}

int gf2x_plan_execute(gf2x_plan *p, const uint64_t *a, const uint64_t *b, uint64_t *out,
                      void *workspace, gf2x_stream_t stream) {
    if (!p) return GF2X_EINVAL;
    try {
        int rc = check_operands(a, p->na_bits, b, p->nb_bits, out);
        if (rc) return rc;
        int dev;
        if ((rc = current_device(&dev))) return rc;
        if (dev != p->device) return GF2X_EINVAL;
        void *ws = workspace;
        if (ws) {
            if (reinterpret_cast<uintptr_t>(ws) & 255) return GF2X_EINVAL;
            if ((rc = check_dev_ptr(ws, p->ws_bytes))) return rc;
        } else {
            std::lock_guard<std::mutex> lk(p->mu);
            if (!p->owned_ws) {
                if (cudaMalloc(&p->owned_ws, p->ws_bytes) != cudaSuccess) {
                    cudaGetLastError();
                    p->owned_ws = nullptr;
                    return GF2X_ENOMEM;
                }
            }
            ws = p->owned_ws;
        }
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        int *st = stream_status_word(s);
        if (!st) return GF2X_ECUDA;
        return plan_run(p, a, b, out, ws, s, st);
    } catch (...) {
        return GF2X_ECUDA;
    }
}

int gf2x_plan_destroy(gf2x_plan *p) {
    if (!p) return GF2X_EINVAL;
    if (p->owned_ws) {
        cudaDeviceSynchronize();
        cudaFree(p->owned_ws);
    }
    delete p;
    return GF2X_OK;
}

// ---- Stage entry points -------------------------------------------------------

int gf2x_stage_basis_cvt64(uint64_t *f, int log_n, int inverse, gf2x_stream_t stream) {
    if (log_n < 0 || log_n > kMaxLogN + 1) return GF2X_EINVAL;
    int rc = check_dev_ptr(f, 8ull << log_n);
    if (rc) return rc;
    try {
        run_basis_cvt<uint64_t>(f, log_n, basis_cvt_levels(log_n), inverse ? 1 : 0,
                                reinterpret_cast<cudaStream_t>(stream));
    } catch (...) {
        return GF2X_ECUDA;
    }
    return check_launch();
}

int gf2x_stage_basis_cvt128(uint64_t *f, int log_n, int inverse, gf2x_stream_t stream) {
    if (log_n < 0 || log_n > kMaxLogN) return GF2X_EINVAL;
    int rc = check_dev_ptr(f, 16ull << log_n);
    if (rc) return rc;
    if (reinterpret_cast<uintptr_t>(f) & 15) return GF2X_EINVAL;
    try {
        run_basis_cvt<uint4>(reinterpret_cast<uint4 *>(f), log_n, basis_cvt_levels(log_n),
                             inverse ? 1 : 0, reinterpret_cast<cudaStream_t>(stream));
    } catch (...) {
        return GF2X_ECUDA;
    }
    return check_launch();
}

int gf2x_stage_chrepr(const uint64_t *g, uint64_t p, uint64_t *F, uint64_t n,
                      gf2x_stream_t stream) {
    if (p == 0 || (p & (p - 1)) || n == 0 || (n & (n - 1)) || p > n || n > (1ull << kMaxLogN))
        return GF2X_EINVAL;
    int rc;
    if ((rc = check_dev_ptr(g, 8 * p)) || (rc = check_dev_ptr(F, 16 * n))) return rc;
    if (reinterpret_cast<uintptr_t>(F) & 15) return GF2X_EINVAL;
    const DevTables *T;
    if ((rc = get_tables(&T))) return rc;
    launch_chrepr(g, p, reinterpret_cast<uint4 *>(F), n, T, reinterpret_cast<cudaStream_t>(stream));
    return check_launch();
}

int gf2x_stage_fft(uint64_t *F, int log_n, int log_p, int inverse, gf2x_stream_t stream) {
    if (log_n < 0 || log_n > kMaxLogN || log_p < 0 || log_p > log_n) return GF2X_EINVAL;
    int rc = check_dev_ptr(F, 16ull << log_n);
    if (rc) return rc;
    if (reinterpret_cast<uintptr_t>(F) & 15) return GF2X_EINVAL;
    const DevTables *T;
    if ((rc = get_tables(&T))) return rc;
    try {
        PassList passes;
        rc = inverse ? plan_fft_inverse(log_n, passes) : plan_fft_forward(log_n, log_p, passes);
        if (rc) return rc == -2 ? GF2X_ENOMEM : GF2X_ECUDA;
        for (int i = 0; i < passes.n; i++)
            launch_fft_pass(passes.v[i], log_n, reinterpret_cast<uint4 *>(F), nullptr, 0, nullptr,
                            T, device_status(), reinterpret_cast<cudaStream_t>(stream));
    } catch (...) {
        return GF2X_ECUDA;
    }
    return check_launch();
}

int gf2x_stage_pointmul(const uint64_t *A, const uint64_t *B, uint64_t *C, uint64_t n,
                        gf2x_stream_t stream) {
    if (n > (1ull << kMaxLogN)) return GF2X_EINVAL;
    int rc;
    if ((rc = check_dev_ptr(A, 16 * n)) || (rc = check_dev_ptr(B, 16 * n)) ||
        (rc = check_dev_ptr(C, 16 * n)))
        return rc;
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B) |
         reinterpret_cast<uintptr_t>(C)) & 15)
        return GF2X_EINVAL;
    if (n == 0) return GF2X_OK;
    const DevTables *T;
    if ((rc = get_tables(&T))) return rc;
    launch_pointmul_mt(reinterpret_cast<const uint4 *>(A), reinterpret_cast<const uint4 *>(B),
                       reinterpret_cast<uint4 *>(C), n, T, reinterpret_cast<cudaStream_t>(stream));
    return check_launch();
}

int gf2x_stage_ichrepr_combine(const uint64_t *F, uint64_t n, uint64_t *out, uint64_t total_bits,
                               gf2x_stream_t stream) {
    if (n > (1ull << kMaxLogN)) return GF2X_EINVAL;
    uint64_t ow = words_of(total_bits);
    int rc;
    if ((rc = check_dev_ptr(F, 16 * n)) || (rc = check_dev_ptr(out, 8 * ow))) return rc;
    if (reinterpret_cast<uintptr_t>(F) & 15) return GF2X_EINVAL;
    if (overlap(out, 8 * ow, F, 16 * n)) return GF2X_EINVAL;
    if (ow == 0) return GF2X_OK;
    const DevTables *T;
    if ((rc = get_tables(&T))) return rc;
    const OutputDesc d{out, ow, mask_of_bits(total_bits)};
    launch_ichrepr_combine(reinterpret_cast<const uint4 *>(F), n, 0, d, nullptr, 1, ow, T,
                           reinterpret_cast<cudaStream_t>(stream));
    return check_launch();
}

int gf2x_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on != 0;
    return GF2X_OK;
}

int gf2x_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &r : g_prof_pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_prof_pending.clear();
    for (int i = 0; i < ST_COUNT; i++) {
        g_prof_ms[i] = 0;
        g_prof_launches[i] = 0;
        g_prof_calls[i] = 0;
    }
    cudaGetLastError();
    return GF2X_OK;
}

int gf2x_profile_read(int stage, double *ms, uint64_t *launches, uint64_t *calls) {
    if (stage < 0 || stage >= ST_COUNT || !ms || !launches || !calls) return GF2X_EINVAL;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    int rc = GF2X_OK;
    for (auto &r : g_prof_pending) {
        float t = 0;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess)
            rc = GF2X_ECUDA;
        g_prof_ms[r.stage] += t;
        g_prof_launches[r.stage] += r.launches;
        g_prof_calls[r.stage] += 1;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_prof_pending.clear();
    cudaGetLastError();
    *ms = g_prof_ms[stage];
    *launches = g_prof_launches[stage];
    *calls = g_prof_calls[stage];
    return rc;
}

const char *gf2x_profile_stage_name(int stage) {
    if (stage < 0 || stage >= ST_COUNT) return "";
    return kStageNames[stage];
}

// ---- Autotuning -------------------------------------------------------------

int gf2x_autotune(uint64_t na_bits, uint64_t nb_bits, int reps, gf2x_tune_t *best) {
    if (!best) return GF2X_EINVAL;
    try {
        int rc = check_sizes(na_bits, nb_bits);
        if (rc) return rc;
        if (!na_bits || !nb_bits) return GF2X_EINVAL;
        const DevTables *T;
        if ((rc = get_tables(&T))) return rc;
        if (reps <= 0) reps = 3;
        int M, pa, pb;
        shape_of(na_bits, nb_bits, &M, &pa, &pb);
        if (M > kMaxLogN) return GF2X_EINVAL;
        // scratch operands (the timing does not depend on the bits), output, workspace
        const size_t ba = 8 * words_of(na_bits), bb = 8 * words_of(nb_bits);
        const size_t bo = 8 * gf2x_out_words(na_bits, nb_bits);
        std::unique_ptr<gf2x_plan> probe(new gf2x_plan());
        if ((rc = plan_init(probe.get(), na_bits, nb_bits))) return rc;
        char *buf = nullptr;
        const size_t total = probe->ws_bytes + ((ba + 255) & ~255ull) + ((bb + 255) & ~255ull) + bo;
        if (cudaMalloc(reinterpret_cast<void **>(&buf), total) != cudaSuccess) {
            cudaGetLastError();
            return GF2X_ENOMEM;
        }
        uint64_t *da = reinterpret_cast<uint64_t *>(buf + probe->ws_bytes);
        uint64_t *db = reinterpret_cast<uint64_t *>(buf + probe->ws_bytes + ((ba + 255) & ~255ull));
        uint64_t *dout = reinterpret_cast<uint64_t *>(buf + probe->ws_bytes + ((ba + 255) & ~255ull) +
                                                      ((bb + 255) & ~255ull));
        cudaMemset(da, 0x5a, ba);
        cudaMemset(db, 0xa5, bb);
        cudaStream_t s = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        int *st = nullptr;
        if ((rc = take_status_word(&st))) {
            cudaFree(buf);
            return rc;
        }
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        cudaMemsetAsync(st, 0, sizeof(int), s);
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        auto trial = [&](const PlanTune &t, double *ms) -> int {
            std::unique_ptr<gf2x_plan> pl(new gf2x_plan());
            int r = plan_init(pl.get(), na_bits, nb_bits, &t);
            if (r) return r;
            if ((r = plan_run_core(pl.get(), da, db, dout, buf, s, T, st, nullptr)))
                return GF2X_ECUDA;
            cudaEventRecord(e0, s);
            for (int i = 0; i < reps; i++)
                if (plan_run_core(pl.get(), da, db, dout, buf, s, T, st, nullptr))
                    return GF2X_ECUDA;
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                cudaGetLastError();
                return GF2X_ECUDA;
            }
            float f = 0;
            cudaEventElapsedTime(&f, e0, e1);
            *ms = f / reps;
            return GF2X_OK;
        };
        // 1. fusion depth: the depths that give distinct strided-pass counts
        TuneEntry bestE;
        bestE.ms = 1e30;
        int seen[3][8];
        int nseen = 0;
        for (int d = kFftGlobalMax; d >= 4 && rc == GF2X_OK; d--) {
            auto npass = [&](int top) { return top > kFftTileLog ? (top - kFftTileLog + d - 1) / d : 0; };
            const int sig[3] = {npass(pa), npass(pb), npass(M)};
            bool dup = false;
            for (int q = 0; q < nseen; q++)
                dup = dup || (seen[0][q] == sig[0] && seen[1][q] == sig[1] && seen[2][q] == sig[2]);
            if (dup) continue;
            for (int q = 0; q < 3; q++) seen[q][nseen] = sig[q];
            nseen++;
            const bool strided = sig[0] + sig[1] + sig[2] > 0;
            for (int nb = 2; nb >= (strided ? 1 : 2) && rc == GF2X_OK; nb--) {
                PlanTune t;
                t.fft_depth = d;
                t.fft_nbuf = nb;
                double ms;
                if ((rc = trial(t, &ms))) break;
                if (ms < bestE.ms) {
                    bestE.t = t;
                    bestE.ms = ms;
                }
            }
        }
        // 2. BasisCvt tile shape with that depth
        const int tiles[4] = {10, 11, 12, 13}, threads[3] = {128, 256, 512};
        for (int i = 0; i < 4 && rc == GF2X_OK; i++)
            for (int j = 0; j < 3 && rc == GF2X_OK; j++) {
                PlanTune t = bestE.t;
                t.bcvt.tile_min_log = tiles[i];
                t.bcvt.small_threads = threads[j];
                if (t.bcvt.tile_min_log == bestE.t.bcvt.tile_min_log &&
                    t.bcvt.small_threads == bestE.t.bcvt.small_threads)
                    continue;
                double ms;
                if ((rc = trial(t, &ms))) break;
                if (ms < bestE.ms) {
                    bestE.t = t;
                    bestE.ms = ms;
                }
            }
        cudaStreamSynchronize(s);
        const int ds = read_clear_status(st);
        give_status_word(st);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaStreamDestroy(s);
        cudaFree(buf);
        if (rc == GF2X_OK) rc = ds;
        if (rc) return rc;
        tune_store(shape_key(na_bits, nb_bits), bestE);
        *best = to_abi(bestE);
        return GF2X_OK;
    } catch (const std::bad_alloc &) {
        return GF2X_ENOMEM;
    } catch (...) {
        return GF2X_ECUDA;
    }
}

int gf2x_tune_get(uint64_t na_bits, uint64_t nb_bits, gf2x_tune_t *out) {
    if (!out || !na_bits || !nb_bits || check_sizes(na_bits, nb_bits)) return GF2X_EINVAL;
    *out = to_abi(tune_for(na_bits, nb_bits));
    return GF2X_OK;
}

int gf2x_tune_set(uint64_t na_bits, uint64_t nb_bits, const gf2x_tune_t *t) {
    if (!t || !na_bits || !nb_bits || check_sizes(na_bits, nb_bits) || !tune_valid(*t))
        return GF2X_EINVAL;
    TuneEntry e;
    e.t = from_abi(*t);
    e.ms = t->ms;
    tune_store(shape_key(na_bits, nb_bits), e);
    return GF2X_OK;
}

int gf2x_tune_save(const char *path) {
    if (!path) return GF2X_EINVAL;
    FILE *f = std::fopen(path, "w");
    if (!f) return GF2X_EINVAL;
    std::fprintf(f, "gf2x-tune 1\n");
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (const auto &kv : g_tune)
            std::fprintf(f, "%d %d %d %d %d %d %d %.6f\n", std::get<0>(kv.first),
                         std::get<1>(kv.first), std::get<2>(kv.first), kv.second.t.fft_depth,
                         kv.second.t.fft_nbuf, kv.second.t.bcvt.tile_min_log,
                         kv.second.t.bcvt.small_threads, kv.second.ms);
    }
    const bool ok = std::fclose(f) == 0;
    return ok ? GF2X_OK : GF2X_EINVAL;
}

int gf2x_tune_load(const char *path) {
    if (!path) return GF2X_EINVAL;
    FILE *f = std::fopen(path, "r");
    if (!f) return GF2X_EINVAL;
    char magic[16] = {0};
    int version = 0;
    if (std::fscanf(f, "%15s %d", magic, &version) != 2 || std::strcmp(magic, "gf2x-tune") != 0 ||
        version != 1) {
        std::fclose(f);
        return GF2X_EINVAL;
    }
    std::vector<std::pair<std::tuple<int, int, int>, TuneEntry>> rows;
    int M, pa, pb;
    gf2x_tune_t t;
    int got;
    while ((got = std::fscanf(f, "%d %d %d %d %d %d %d %lf", &M, &pa, &pb, &t.fft_depth,
                              &t.fft_buffers, &t.bcvt_tile_log, &t.bcvt_threads, &t.ms)) == 8) {
        if (M < 1 || M > kMaxLogN || pa < 0 || pa > M || pb < 0 || pb > M || !tune_valid(t)) {
            std::fclose(f);
            return GF2X_EINVAL;
        }
        TuneEntry e;
        e.t = from_abi(t);
        e.ms = t.ms;
        rows.emplace_back(std::make_tuple(M, pa, pb), e);
    }
    const bool clean = got == EOF;
    std::fclose(f);
    if (!clean) return GF2X_EINVAL;
    for (const auto &r : rows) tune_store(r.first, r.second);
    return GF2X_OK;
}

int gf2x_stream_status(gf2x_stream_t stream) {
    try {
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            return GF2X_ECUDA;
        }
        int *st = stream_status_word(s);
        if (!st) return GF2X_ECUDA;
        return read_clear_status(st);
    } catch (...) {
        return GF2X_ECUDA;
    }
}

int gf2x_debug_set_wait_spins(int64_t spins) {
    set_wait_spins(spins);
    return GF2X_OK;
}

int gf2x_shutdown(void) {
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        g_cache.clear();
    }
    std::lock_guard<std::mutex> lk(g_ctx_mu);
    int cur = -1;
    cudaGetDevice(&cur);
    for (auto &kv : g_ctx) {
        if (kv.second.tables) {
            cudaSetDevice(kv.first);
            cudaDeviceSynchronize();
            cudaFree(kv.second.tables);
            kv.second.tables = nullptr;
        }
        if (kv.second.status) {
            cudaSetDevice(kv.first);
            cudaFree(kv.second.status);
            kv.second.status = nullptr;
            kv.second.free_words.clear();
            kv.second.stream_words.clear();
        }
        if (kv.second.pool) {
            cudaSetDevice(kv.first);
            cudaDeviceSynchronize();
            cudaStreamDestroy(kv.second.copy_stream);
            cudaMemPoolDestroy(kv.second.pool);
            kv.second.pool = nullptr;
            kv.second.copy_stream = nullptr;
        }
    }
    if (cur >= 0) cudaSetDevice(cur);
    cudaGetLastError();
    return GF2X_OK;
}

}  // extern "C"
