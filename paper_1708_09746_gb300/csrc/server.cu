// Serving loop: requests arrive at any time; a worker thread admits them as
// device memory and execution slots free up, batches the queued requests that
// share a transform shape into one launch, runs admitted work concurrently on
// its slots' streams, and records arrival -> result-ready latency.
//
// Memory admission: the server owns one device arena of `mem_budget` bytes
// (first-fit over offsets); a request (or batch) is admitted only when its
// workspace fits.  Plans and tables stay resident (the library's caches).
// Waits are bounded: gf2x_server_wait returns GF2X_ETIMEOUT when its limit
// runs out; the worker polls completion events and never blocks on the GPU.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "../../include/gf2x_gb300.h"
#include "api_internal.h"
#include "kernels.h"
#include "plan.h"
#include "small.h"

using namespace gf2x;

namespace {

using Clock = std::chrono::steady_clock;

// How a request is computed: one transform, grouped with the queued requests
// of the same transform shape (kGroup); by chunks of the longer operand
// against one transform of the shorter (kChunked, alone); directly without a
// transform when the shorter operand has at most kSmallWords words (kDirect,
// grouped with the other direct requests).
enum Path { kGroup = 0, kChunked = 1, kDirect = 2 };

struct Request {
    uint64_t ticket;
    const uint64_t *a, *b;
    uint64_t *out;
    uint64_t na, nb;
    std::tuple<int, int, int> shape;
    Clock::time_point t_submit;
    int path = kGroup;
    bool swap = false;  // kChunked: the chunks are cut from b (x = b, y = a)
    ChunkShape cs;
    std::shared_ptr<gf2x_plan> cplan;  // kChunked: the chunk plan
};

// First-fit allocator over [0, size) of a device arena (offsets 256-aligned).
struct Arena {
    size_t size = 0;
    std::map<size_t, size_t> free_;  // offset -> length
    void init(size_t n) {
        size = n;
        free_.clear();
        free_[0] = n;
    }
    bool alloc(size_t n, size_t *off) {
        n = (n + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n, at = it->first + n;
                free_.erase(it);
                if (rest) free_[at] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = (n + 255) & ~(size_t)255;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

constexpr int kMaxBatch = 64;

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<Request> reqs;
    size_t off = 0, bytes = 0;
    OperandDesc *d_a = nullptr, *d_b = nullptr;  // device descriptors (kMaxBatch)
    OutputDesc *d_out = nullptr;
    OperandDesc *h_a = nullptr, *h_b = nullptr;  // pinned mirrors
    OutputDesc *h_out = nullptr;
    int *d_st = nullptr;  // this slot's device status word (a library word)
    int *h_st = nullptr;  // pinned copy, written at the end of each batch
};

}  // namespace

struct gf2x_server {
    int device = 0;
    int max_batch = kMaxBatch;
    char *arena_base = nullptr;
    Arena arena;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> queue;
    std::unordered_map<uint64_t, int> status;  // ticket -> 1 running/queued, 0 done, <0 error
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    // statistics
    std::vector<double> lat_ms;
    Clock::time_point t_first{}, t_last{};
    uint64_t completed = 0;
    bool any = false;
};

namespace {

void worker_main(gf2x_server *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        bool progressed = false;
        // 1. completions (non-blocking event queries)
        for (auto &sl : S->slots) {
            if (!sl.busy) continue;
            cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            // the slot's own status word, copied back before `done`: a bounded
            // device wait that ran out is reported to this batch's requests
            const int st = (q == cudaSuccess) ? (*sl.h_st ? *sl.h_st : GF2X_OK) : GF2X_ECUDA;
            if (q != cudaSuccess) cudaGetLastError();
            const auto now = Clock::now();
            for (auto &r : sl.reqs) {
                S->status[r.ticket] = st;
                S->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r.t_submit).count());
                S->completed++;
            }
            S->t_last = now;
            S->arena.release(sl.off, sl.bytes);
            sl.reqs.clear();
            sl.busy = false;
            progressed = true;
        }
        if (progressed) S->cv_done.notify_all();
        // 2. admission: head of the queue plus queued requests of the same shape
        while (!S->queue.empty()) {
            Slot *free_slot = nullptr;
            for (auto &sl : S->slots)
                if (!sl.busy) {
                    free_slot = &sl;
                    break;
                }
            if (!free_slot) break;
            const Request head = S->queue.front();
            std::shared_ptr<gf2x_plan> plan;
            int rc = head.path == kGroup ? api::plan_for(head.na, head.nb, &plan) : GF2X_OK;
            if (rc) {
                S->status[head.ticket] = rc;
                S->queue.pop_front();
                S->cv_done.notify_all();
                continue;
            }
            // workspace per request of the group: the plan's, the chunked
            // product's, or none for direct products (one arena unit)
            const size_t per_req = head.path == kGroup ? plan->ws_bytes
                                   : head.path == kChunked ? chunked_ws_bytes(head.cplan.get(), head.cs.C)
                                                           : 256;
            std::vector<size_t> take{0};
            if (head.path != kChunked)
                for (size_t q = 1; q < S->queue.size() && take.size() < (size_t)S->max_batch; q++)
                    if (S->queue[q].shape == head.shape) take.push_back(q);
            // largest batch whose workspace fits the free arena memory now
            size_t off = 0;
            size_t k = take.size();
            while (k > 0 && !S->arena.alloc(k * per_req, &off)) k = k > 1 ? k / 2 : 0;
            if (k == 0) break;  // wait for memory (head-of-line order kept)
            take.resize(k);
            Slot &sl = *free_slot;
            sl.reqs.clear();
            for (size_t q : take) sl.reqs.push_back(S->queue[q]);
            for (size_t q = take.size(); q-- > 0;) S->queue.erase(S->queue.begin() + take[q]);
            sl.off = off;
            sl.bytes = k * per_req;
            uint64_t max_words = 0;
            for (size_t q = 0; q < k; q++) {
                const Request &r = sl.reqs[q];
                sl.h_a[q] = OperandDesc{r.a, words_of(r.na), mask_of_bits(r.na)};
                sl.h_b[q] = OperandDesc{r.b, words_of(r.nb), mask_of_bits(r.nb)};
                const uint64_t tot = r.na + r.nb - 1;
                sl.h_out[q] = OutputDesc{r.out, words_of(tot), mask_of_bits(tot)};
                max_words = std::max(max_words, words_of(tot));
            }
            const DevTables *T;
            rc = api::tables(&T);
            if (!rc) {
                *sl.h_st = 0;
                cudaMemsetAsync(sl.d_st, 0, sizeof(int), sl.stream);
                cudaMemcpyAsync(sl.d_a, sl.h_a, k * sizeof(OperandDesc), cudaMemcpyHostToDevice, sl.stream);
                cudaMemcpyAsync(sl.d_b, sl.h_b, k * sizeof(OperandDesc), cudaMemcpyHostToDevice, sl.stream);
                cudaMemcpyAsync(sl.d_out, sl.h_out, k * sizeof(OutputDesc), cudaMemcpyHostToDevice,
                                sl.stream);
                const OperandDesc none_in{nullptr, 0, 0};
                const OutputDesc none_out{nullptr, 0, 0};
                if (head.path == kGroup) {
                    rc = plan_run_batch(plan.get(), (int)k, sl.d_a, sl.d_b, sl.d_out, none_in,
                                        none_in, none_out, max_words, S->arena_base + off,
                                        plan->ws_bytes, sl.stream, T, sl.d_st, nullptr)
                             ? GF2X_ECUDA
                             : GF2X_OK;
                } else if (head.path == kChunked) {
                    const Request &r = sl.reqs[0];
                    const uint64_t *x = r.swap ? r.b : r.a, *y = r.swap ? r.a : r.b;
                    const uint64_t xb = r.swap ? r.nb : r.na, yb = r.swap ? r.na : r.nb;
                    rc = plan_run_chunked(r.cplan.get(), r.cs, x, xb, y, yb, r.out,
                                          S->arena_base + off, sl.stream, T, sl.d_st, nullptr)
                             ? GF2X_ECUDA
                             : GF2X_OK;
                } else {
                    for (const Request &r : sl.reqs) {
                        const uint64_t ow = gf2x_out_words(r.na, r.nb);
                        if (words_of(r.nb) <= words_of(r.na))
                            launch_mul_small(r.a, r.na, r.b, r.nb, r.out, ow, 0, false, sl.stream);
                        else
                            launch_mul_small(r.b, r.nb, r.a, r.na, r.out, ow, 0, false, sl.stream);
                    }
                    rc = cudaGetLastError() == cudaSuccess ? GF2X_OK : GF2X_ECUDA;
                }
                if (!rc)
                    cudaMemcpyAsync(sl.h_st, sl.d_st, sizeof(int), cudaMemcpyDeviceToHost, sl.stream);
            }
            if (!rc && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) rc = GF2X_ECUDA;
            if (rc) {
                cudaGetLastError();
                for (auto &r : sl.reqs) S->status[r.ticket] = rc;
                S->arena.release(sl.off, sl.bytes);
                sl.reqs.clear();
                S->cv_done.notify_all();
                continue;
            }
            sl.busy = true;
        }
        bool busy = false;
        for (auto &sl : S->slots) busy |= sl.busy;
        if (S->stop && !busy && S->queue.empty()) break;
        // sleep until new work arrives, or poll again shortly while work runs
        S->cv_work.wait_for(lk, std::chrono::microseconds(busy ? 20 : 2000));
    }
}

}  // namespace

extern "C" {

int gf2x_server_create(size_t mem_budget_bytes, int max_slots, int max_batch,
                       gf2x_server **out) {
    if (!out || max_slots <= 0 || max_slots > 256 || mem_budget_bytes < 4096 || max_batch < 1 ||
        max_batch > kMaxBatch)
        return GF2X_EINVAL;
    *out = nullptr;
    try {
        std::unique_ptr<gf2x_server> S(new gf2x_server());
        S->max_batch = max_batch;
        if (cudaGetDevice(&S->device) != cudaSuccess) {
            cudaGetLastError();
            return GF2X_ECUDA;
        }
        const DevTables *T;
        int rc = api::tables(&T);
        if (rc) return rc;
        if (cudaMalloc(reinterpret_cast<void **>(&S->arena_base), mem_budget_bytes) != cudaSuccess) {
            cudaGetLastError();
            return GF2X_ENOMEM;
        }
        S->arena.init(mem_budget_bytes);
        S->slots.resize(max_slots);
        for (auto &sl : S->slots) {
            bool ok = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess &&
                      cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess &&
                      cudaMalloc(&sl.d_a, kMaxBatch * sizeof(OperandDesc)) == cudaSuccess &&
                      cudaMalloc(&sl.d_b, kMaxBatch * sizeof(OperandDesc)) == cudaSuccess &&
                      cudaMalloc(&sl.d_out, kMaxBatch * sizeof(OutputDesc)) == cudaSuccess &&
                      cudaMallocHost(&sl.h_a, kMaxBatch * sizeof(OperandDesc)) == cudaSuccess &&
                      cudaMallocHost(&sl.h_b, kMaxBatch * sizeof(OperandDesc)) == cudaSuccess &&
                      cudaMallocHost(&sl.h_out, kMaxBatch * sizeof(OutputDesc)) == cudaSuccess &&
                      cudaMallocHost(&sl.h_st, sizeof(int)) == cudaSuccess;
            if (ok) {
                *sl.h_st = 0;
                rc = api::take_status(&sl.d_st);
                if (rc) {
                    gf2x_server_destroy(S.release());
                    return rc;
                }
            }
            if (!ok) {
                cudaGetLastError();
                gf2x_server_destroy(S.release());
                return GF2X_ENOMEM;
            }
        }
        prepare_bcvt_attributes();
        prepare_fft_attributes();
        gf2x_server *raw = S.get();
        S->worker = std::thread(worker_main, raw);
        *out = S.release();
        return GF2X_OK;
    } catch (const std::bad_alloc &) {
        return GF2X_ENOMEM;
    } catch (...) {
        return GF2X_ECUDA;
    }
}

int gf2x_server_submit(gf2x_server *S, const uint64_t *a, uint64_t na_bits, const uint64_t *b,
                       uint64_t nb_bits, uint64_t *out, uint64_t *ticket) {
    if (!S || !ticket) return GF2X_EINVAL;
    try {
        int rc = api::check_product_args(a, na_bits, b, nb_bits, out);
        if (rc) return rc;
        Request r;
        r.a = a;
        r.b = b;
        r.out = out;
        r.na = na_bits;
        r.nb = nb_bits;
        r.t_submit = Clock::now();
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) return GF2X_EBUSY;
        r.ticket = S->next_ticket++;
        *ticket = r.ticket;
        if (!na_bits || !nb_bits) {
            S->status[r.ticket] = GF2X_OK;
            return GF2X_OK;
        }
        const uint64_t na_w = words_of(na_bits), nb_w = words_of(nb_bits);
        const int M = log2_ceil(std::max<uint64_t>(2, na_w + nb_w - 1));
        size_t need = 0;
        if (std::min(na_w, nb_w) <= (uint64_t)kSmallWords) {
            r.path = kDirect;
            r.shape = std::make_tuple(-2, 0, 0);
            need = 256;
        } else if (chunk_shape(na_w, nb_w, &r.cs) || (r.swap = chunk_shape(nb_w, na_w, &r.cs))) {
            r.path = kChunked;
            const uint64_t y_bits = r.swap ? na_bits : nb_bits;
            if ((rc = api::plan_for(y_bits, 64 * r.cs.L, &r.cplan))) return rc;
            r.shape = std::make_tuple(-1, M, 0);
            need = chunked_ws_bytes(r.cplan.get(), r.cs.C);
        } else {
            r.shape = std::make_tuple(M, log2_ceil(na_w), log2_ceil(nb_w));
            std::shared_ptr<gf2x_plan> plan;
            if ((rc = api::plan_for(na_bits, nb_bits, &plan))) return rc;
            need = plan->ws_bytes;
        }
        if (need > S->arena.size) return GF2X_EINVAL;  // could never be admitted
        if (!S->any) {
            S->t_first = r.t_submit;
            S->any = true;
        }
        S->status[r.ticket] = 1;
        S->queue.push_back(r);
        S->cv_work.notify_one();
        return GF2X_OK;
    } catch (const std::bad_alloc &) {
        return GF2X_ENOMEM;
    } catch (...) {
        return GF2X_ECUDA;
    }
}

int gf2x_server_wait(gf2x_server *S, uint64_t ticket, uint64_t timeout_us) {
    if (!S) return GF2X_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->status.find(ticket);
    if (it == S->status.end()) return GF2X_EINVAL;
    const auto deadline = Clock::now() + std::chrono::microseconds(timeout_us);
    while (S->status[ticket] == 1) {
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout &&
            S->status[ticket] == 1)
            return GF2X_ETIMEOUT;
    }
    const int st = S->status[ticket];
    S->status.erase(ticket);
    return st;
}

int gf2x_server_stats(gf2x_server *S, double *p50_ms, double *p99_ms, double *throughput_per_s,
                      uint64_t *completed) {
    if (!S || !p50_ms || !p99_ms || !throughput_per_s || !completed) return GF2X_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    std::vector<double> v = S->lat_ms;
    *completed = S->completed;
    if (v.empty()) {
        *p50_ms = *p99_ms = *throughput_per_s = 0;
        return GF2X_OK;
    }
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) {
        size_t i = (size_t)std::min<double>(v.size() - 1, std::max(0.0, p * (v.size() - 1)));
        return v[i];
    };
    *p50_ms = pct(0.50);
    *p99_ms = pct(0.99);
    const double span = std::chrono::duration<double>(S->t_last - S->t_first).count();
    *throughput_per_s = span > 0 ? (double)S->completed / span : 0.0;
    return GF2X_OK;
}

int gf2x_server_reset_stats(gf2x_server *S) {
    if (!S) return GF2X_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    S->lat_ms.clear();
    S->completed = 0;
    S->any = false;
    return GF2X_OK;
}

int gf2x_server_destroy(gf2x_server *S) {
    if (!S) return GF2X_EINVAL;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (auto &sl : S->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        cudaFree(sl.d_a);
        cudaFree(sl.d_b);
        cudaFree(sl.d_out);
        cudaFreeHost(sl.h_a);
        cudaFreeHost(sl.h_b);
        cudaFreeHost(sl.h_out);
        cudaFreeHost(sl.h_st);
        api::give_status(sl.d_st);
    }
    cudaFree(S->arena_base);
    cudaGetLastError();
    delete S;
    return GF2X_OK;
}

}  // extern "C"
