// The C ABI (include/gf2x_gb300.h): argument checks, per-device tables,
// plans and the order of the stages of Alg. 5.
#include <algorithm>
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

using namespace gf2x;

namespace {

// ---- Per-device context: the size-independent tables, uploaded once. ------
struct DeviceCtx {
    DevTables *tables = nullptr;
    int *status = nullptr;  // device status word of the pipelined kernels
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
        if (cudaMalloc(&st, sizeof(int)) != cudaSuccess || cudaMemset(st, 0, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(d);
            if (st) cudaFree(st);
            return GF2X_ENOMEM;
        }
        c.tables = d;
        c.status = st;
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

// Device status word of the current device (valid after get_tables).
int *device_status() {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_ctx_mu);
    return g_ctx[dev].status;
}

// Reads and clears the device status word (synchronises the device).
int take_device_status() {
    int *st = device_status();
    if (!st) return GF2X_OK;
    int v = 0;
    if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpy(&v, st, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return GF2X_ECUDA;
    }
    if (v) cudaMemset(st, 0, sizeof(int));
    return v;
}

int check_launch() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GF2X_OK : GF2X_ECUDA;
}

// Device (or managed) memory?  A null pointer is accepted only for size 0.
int check_dev_ptr(const void *p, size_t bytes) {
    if (bytes == 0) return GF2X_OK;
    if (!p) return GF2X_EINVAL;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GF2X_EINVAL;
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return GF2X_EINVAL;
    return GF2X_OK;
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
const char *kStageNames[ST_COUNT] = {"split",        "basis_cvt",      "chrepr_fft_a",
                                     "chrepr_fft_b", "fft_pointmul_ifft_bottom", "ifft_top",
                                     "ibasis_cvt",   "ichrepr_combine"};

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

int plan_init(gf2x_plan *p, uint64_t na_bits, uint64_t nb_bits) {
    int rc = gf2x::plan_init(p, na_bits, nb_bits, nullptr);
    if (rc == -1) return GF2X_EINVAL;
    if (rc == -2) return GF2X_ENOMEM;
    return rc ? GF2X_ECUDA : GF2X_OK;
}

// Alg. 5, stage after stage, on `s`, with the library's tables.
int plan_run(const gf2x_plan *p, const uint64_t *a, const uint64_t *b, uint64_t *out, void *ws,
             cudaStream_t s, cudaEvent_t b_ready = nullptr) {
    const DevTables *T;
    int rc = get_tables(&T);
    if (rc) return rc;
    StageTimer tm(s);
    rc = plan_run_core(p, a, b, out, ws, s, T, device_status(), &tm, b_ready);
    return rc ? GF2X_ECUDA : GF2X_OK;
}

// Plan cache for the one-shot calls, keyed by (device, sizes).
std::mutex g_cache_mu;
std::map<std::tuple<int, uint64_t, uint64_t>, std::shared_ptr<gf2x_plan>> g_cache;

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

int mul_on_stream(const uint64_t *a, uint64_t na_bits, const uint64_t *b, uint64_t nb_bits,
                  uint64_t *out, cudaStream_t s) {
    std::shared_ptr<gf2x_plan> p;
    int rc = cached_plan(na_bits, nb_bits, &p);
    if (rc) return rc;
    void *ws = nullptr;
    if ((rc = ws_alloc(&ws, p->ws_bytes, s))) return rc;
    rc = plan_run(p.get(), a, b, out, ws, s);
    ws_free(ws, s);
    if (rc == GF2X_OK) rc = check_launch();
    return rc;
}

}  // namespace

// Entry points shared with the batch and server modules.
namespace gf2x {
namespace api {
int tables(const DevTables **T) { return get_tables(T); }
int *status_word() { return device_status(); }
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
int run_one(const gf2x_plan *p, const uint64_t *a, const uint64_t *b, uint64_t *out, void *ws,
            cudaStream_t s) {
    return plan_run(p, a, b, out, ws, s);
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

int gf2x_mul_async(const uint64_t *a, uint64_t na_bits, const uint64_t *b, uint64_t nb_bits,
                   uint64_t *out, gf2x_stream_t stream) {
    try {
        int rc = check_operands(a, na_bits, b, nb_bits, out);
        if (rc) return rc;
        if (!na_bits || !nb_bits) return GF2X_OK;
        return mul_on_stream(a, na_bits, b, nb_bits, out, reinterpret_cast<cudaStream_t>(stream));
    } catch (const std::bad_alloc &) {
        return GF2X_ENOMEM;
    } catch (...) {
        return GF2X_ECUDA;
    }
}

int gf2x_mul(const uint64_t *a, uint64_t na_bits, const uint64_t *b, uint64_t nb_bits,
             uint64_t *out) {
    int rc = gf2x_mul_async(a, na_bits, b, nb_bits, out, nullptr);
    if (rc) return rc;
    if (cudaStreamSynchronize(0) != cudaSuccess) {
        cudaGetLastError();
        return GF2X_ECUDA;
    }
    return take_device_status();
}

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
        cudaEvent_t alloc_done = nullptr, b_ready = nullptr;
        if (cudaEventCreateWithFlags(&alloc_done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&b_ready, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            if (alloc_done) cudaEventDestroy(alloc_done);
            ws_free(buf, s);
            return GF2X_ECUDA;
        }
        cudaEventRecord(alloc_done, s);
        cudaMemcpyAsync(da, a_host, ba, cudaMemcpyHostToDevice, s);
        cudaStreamWaitEvent(cs, alloc_done, 0);
        cudaMemcpyAsync(db, b_host, bb, cudaMemcpyHostToDevice, cs);
        cudaEventRecord(b_ready, cs);
        rc = plan_run(p.get(), da, db, dout, buf, s, b_ready);
        cudaMemcpyAsync(out_host, dout, bo, cudaMemcpyDeviceToHost, s);
        ws_free(buf, s);
        cudaError_t e = cudaStreamSynchronize(s);
        cudaEventDestroy(alloc_done);
        cudaEventDestroy(b_ready);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return GF2X_ECUDA;
        }
        return rc;
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
        return plan_run(p, a, b, out, ws, reinterpret_cast<cudaStream_t>(stream));
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
