// Batched products: many products of uneven sizes in few launches.
//
// Products whose transforms have the same shape (log2 N, log2 Pa, log2 Pb)
// run the same kernels with the same pass schedule; only their operand
// lengths, masks and output lengths differ.  A batch groups its products by
// shape; each group (in chunks that fit the memory budget) is one launch per
// kernel, blockIdx.y (or the high bits of the persistent kernels' tile index)
// selecting the product, whose workspace sits at a fixed stride.  Per-product
// operand/output descriptors live in a device array.
//
// gf2x_batch_execute captures the whole batch once into a CUDA graph (the
// descriptor upload from a pinned host mirror plus every launch) and replays
// it on later calls, rewriting only the pinned descriptors.  The graph forks
// into kBatchBranches streams with a workspace each; the groups go to the
// branches largest first, each to the least loaded one, so that the many small
// groups' launches overlap instead of leaving the GPU mostly idle one after
// another (4096 uneven products: 79 k/s on one branch, 99 k with two, 111 k
// with four, 117 k with eight).
#include <algorithm>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "../../include/gf2x_gb300.h"
#include "api_internal.h"
#include "kernels.h"
#include "plan.h"
#include "small.h"

using namespace gf2x;

// Branches of a batch's CUDA graph: the shape groups are independent, so the
// graph forks into this many streams (each with its own workspace) and joins
// at the end, letting small groups' launches run side by side.
#ifndef GF2X_BATCH_BRANCHES
#define GF2X_BATCH_BRANCHES 8
#endif
constexpr int kBatchBranches = GF2X_BATCH_BRANCHES;

struct gf2x_batch {
    struct Chunk {
        std::shared_ptr<gf2x_plan> plan;  // null: direct products (short operand)
        int first, count;  // range in the grouped order
        uint64_t max_out_words;
    };
    int count = 0, device = 0;
    std::vector<uint64_t> na, nb;
    std::vector<int> order;  // grouped order -> product index
    std::vector<Chunk> chunks;
    size_t ws_bytes = 0;  // per branch, shared by its chunks (run one after another)
    int nbr = 1;          // branches used: at most kBatchBranches, fewer where the
                          // budget holds fewer branch workspaces
    void *ws = nullptr;   // nbr regions of ws_bytes (rounded to 256)
    cudaStream_t branch[kBatchBranches] = {};
    cudaEvent_t fork = nullptr, join[kBatchBranches] = {};
    OperandDesc *d_a = nullptr, *d_b = nullptr;
    OutputDesc *d_out = nullptr;
    OperandDesc *h_a = nullptr, *h_b = nullptr;  // pinned mirrors
    OutputDesc *h_out = nullptr;
    cudaStream_t cap = nullptr;  // private stream for capture
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    int *st = nullptr;  // the batch's own status word (a library word)
    bool launched = false;
    std::mutex mu;
};

namespace {

// `branches`: workspaces the budget is shared among (one per graph branch).
int batch_build(gf2x_batch *B, int count, const uint64_t *na_bits, const uint64_t *nb_bits,
                size_t mem_budget, int branches) {
    B->count = count;
    B->na.assign(na_bits, na_bits + count);
    B->nb.assign(nb_bits, nb_bits + count);
    // group by transform shape; products with a short operand (at most
    // kSmallWords words) go to one launch of direct products
    std::map<std::tuple<int, int, int>, std::vector<int>> groups;
    std::vector<int> direct;
    for (int i = 0; i < count; i++) {
        if (!na_bits[i] || !nb_bits[i]) continue;
        if (na_bits[i] > (1ull << 33) || nb_bits[i] > (1ull << 33)) return GF2X_EINVAL;
        const uint64_t na_w = words_of(na_bits[i]), nb_w = words_of(nb_bits[i]);
        if (std::min(na_w, nb_w) <= (uint64_t)kSmallWords) {
            direct.push_back(i);
            continue;
        }
        const int M = log2_ceil(std::max<uint64_t>(2, na_w + nb_w - 1));
        if (M > kMaxLogN) return GF2X_EINVAL;
        groups[std::make_tuple(M, log2_ceil(na_w), log2_ceil(nb_w))].push_back(i);
    }
    size_t max_group_bytes = 0, max_one = 0;
    for (auto &kv : groups) {
        std::shared_ptr<gf2x_plan> p;
        int rc = api::plan_for(B->na[kv.second[0]], B->nb[kv.second[0]], &p);
        if (rc) return rc;
        max_one = std::max(max_one, p->ws_bytes);
        max_group_bytes = std::max(max_group_bytes, p->ws_bytes * kv.second.size());
    }
    branches = std::max(1, branches);
    B->ws_bytes = std::max(max_one, std::min(max_group_bytes, mem_budget / branches));
    // a product whose workspace alone exceeds a branch's share: fewer branches
    // (at least one), so that the batch stays within its budget where it can
    B->nbr = (int)std::max<size_t>(
        1, std::min<size_t>(branches, mem_budget / std::max<size_t>(1, B->ws_bytes)));
    for (auto &kv : groups) {
        std::shared_ptr<gf2x_plan> p;
        api::plan_for(B->na[kv.second[0]], B->nb[kv.second[0]], &p);
        const int per = (int)std::max<size_t>(
            1, std::min<size_t>(B->ws_bytes / p->ws_bytes, 65535));
        const std::vector<int> &idx = kv.second;
        for (size_t c0 = 0; c0 < idx.size(); c0 += per) {
            gf2x_batch::Chunk ch;
            ch.plan = p;
            ch.first = (int)B->order.size();
            ch.count = (int)std::min<size_t>(per, idx.size() - c0);
            ch.max_out_words = 0;
            for (int q = 0; q < ch.count; q++) {
                const int i = idx[c0 + q];
                B->order.push_back(i);
                ch.max_out_words = std::max(ch.max_out_words, gf2x_out_words(B->na[i], B->nb[i]));
            }
            B->chunks.push_back(ch);
        }
    }
    for (size_t c0 = 0; c0 < direct.size(); c0 += 65535) {
        gf2x_batch::Chunk ch;
        ch.first = (int)B->order.size();
        ch.count = (int)std::min<size_t>(65535, direct.size() - c0);
        ch.max_out_words = 0;
        for (int q = 0; q < ch.count; q++) {
            const int i = direct[c0 + q];
            B->order.push_back(i);
            ch.max_out_words = std::max(ch.max_out_words, gf2x_out_words(B->na[i], B->nb[i]));
        }
        B->chunks.push_back(ch);
    }
    return GF2X_OK;
}

void fill_descs(const gf2x_batch *B, const uint64_t *const *a, const uint64_t *const *b,
                uint64_t *const *out, OperandDesc *ha, OperandDesc *hb, OutputDesc *ho) {
    for (size_t k = 0; k < B->order.size(); k++) {
        const int i = B->order[k];
        ha[k] = OperandDesc{a[i], words_of(B->na[i]), mask_of_bits(B->na[i])};
        hb[k] = OperandDesc{b[i], words_of(B->nb[i]), mask_of_bits(B->nb[i])};
        const uint64_t tot = B->na[i] + B->nb[i] - 1;
        ho[k] = OutputDesc{out[i], words_of(tot), mask_of_bits(tot)};
    }
}

// Device work of a chunk, for balancing the branches: products times
// N log2 N of their transforms (direct products: their output words).
double chunk_cost(const gf2x_batch::Chunk &ch) {
    if (!ch.plan) return (double)ch.count * (double)ch.max_out_words;
    const double N = (double)ch.plan->N;
    return (double)ch.count * N * (double)(ch.plan->M + 1);
}

size_t branch_stride(const gf2x_batch *B) { return (B->ws_bytes + 255) & ~(size_t)255; }

// The chunks on kBatchBranches streams forked from s and joined back into it
// (longest chunks first, each to the least loaded branch), branch k on its own
// workspace region.
int enqueue_branches(gf2x_batch *B, cudaStream_t s) {
    const DevTables *T;
    int rc = api::tables(&T);
    if (rc) return rc;
    const OperandDesc none_in{nullptr, 0, 0};
    const OutputDesc none_out{nullptr, 0, 0};
    std::vector<int> ord(B->chunks.size());
    for (size_t i = 0; i < ord.size(); i++) ord[i] = (int)i;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
        return chunk_cost(B->chunks[x]) > chunk_cost(B->chunks[y]);
    });
    const int nbr = std::max(1, std::min(B->nbr, kBatchBranches));
    double load[kBatchBranches] = {};
    std::vector<int> to(B->chunks.size(), 0);
    for (int c : ord) {
        int k = 0;
        for (int q = 1; q < nbr; q++)
            if (load[q] < load[k]) k = q;
        to[c] = k;
        load[k] += chunk_cost(B->chunks[c]);
    }
    if (cudaEventRecord(B->fork, s) != cudaSuccess) return GF2X_ECUDA;
    for (int k = 0; k < nbr; k++)
        if (cudaStreamWaitEvent(B->branch[k], B->fork, 0) != cudaSuccess) return GF2X_ECUDA;
    for (size_t c = 0; c < B->chunks.size(); c++) {
        const auto &ch = B->chunks[c];
        cudaStream_t bs = B->branch[to[c]];
        void *ws = static_cast<char *>(B->ws) + (size_t)to[c] * branch_stride(B);
        if (!ch.plan) {
            launch_mul_small_many(B->d_a + ch.first, B->d_b + ch.first, B->d_out + ch.first,
                                  ch.count, ch.max_out_words, bs);
            continue;
        }
        if (plan_run_batch(ch.plan.get(), ch.count, B->d_a + ch.first, B->d_b + ch.first,
                           B->d_out + ch.first, none_in, none_in, none_out, ch.max_out_words, ws,
                           ch.plan->ws_bytes, bs, T, B->st, nullptr))
            return GF2X_ECUDA;
    }
    for (int k = 0; k < nbr; k++) {
        if (cudaEventRecord(B->join[k], B->branch[k]) != cudaSuccess) return GF2X_ECUDA;
        if (cudaStreamWaitEvent(s, B->join[k], 0) != cudaSuccess) return GF2X_ECUDA;
    }
    return GF2X_OK;
}

// Branch streams of one-shot batches (gf2x_mul_batched): created once per
// device and reused by every call.
int branch_streams(cudaStream_t (&out)[kBatchBranches]) {
    static std::mutex mu;
    static std::map<int, std::vector<cudaStream_t>> pool;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return GF2X_ECUDA;
    }
    std::lock_guard<std::mutex> lk(mu);
    std::vector<cudaStream_t> &v = pool[dev];
    while ((int)v.size() < kBatchBranches) {
        cudaStream_t x = nullptr;
        if (cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return GF2X_ECUDA;
        }
        v.push_back(x);
    }
    for (int k = 0; k < kBatchBranches; k++) out[k] = v[k];
    return GF2X_OK;
}

int check_all(int count, const uint64_t *const *a, const uint64_t *na_bits,
              const uint64_t *const *b, const uint64_t *nb_bits, uint64_t *const *out) {
    for (int i = 0; i < count; i++) {
        int rc = api::check_product_args(a[i], na_bits[i], b[i], nb_bits[i], out[i]);
        if (rc) return rc;
    }
    return GF2X_OK;
}

}  // namespace

extern "C" {

int gf2x_mul_batched(int count, const uint64_t *const *a, const uint64_t *na_bits,
                     const uint64_t *const *b, const uint64_t *nb_bits, uint64_t *const *out,
                     gf2x_stream_t stream) {
    if (count < 0) return GF2X_EINVAL;
    if (count == 0) return GF2X_OK;
    if (!a || !na_bits || !b || !nb_bits || !out) return GF2X_EINVAL;
    try {
        int rc = check_all(count, a, na_bits, b, nb_bits, out);
        if (rc) return rc;
        gf2x_batch B;
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        if ((rc = batch_build(&B, count, na_bits, nb_bits, free_b / 2, kBatchBranches))) return rc;
        if (B.order.empty()) return GF2X_OK;
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        const size_t n = B.order.size();
        std::vector<OperandDesc> ha(n), hb(n);
        std::vector<OutputDesc> ho(n);
        fill_descs(&B, a, b, out, ha.data(), hb.data(), ho.data());
        if ((rc = branch_streams(B.branch))) return rc;
        char *mem = nullptr;
        const size_t dbytes = n * (2 * sizeof(OperandDesc) + sizeof(OutputDesc));
        const size_t ws_off = (dbytes + 255) & ~(size_t)255;
        if ((rc = api::ws_alloc(reinterpret_cast<void **>(&mem),
                                ws_off + (size_t)B.nbr * branch_stride(&B), s)))
            return rc;
        OperandDesc *da = reinterpret_cast<OperandDesc *>(mem);
        OperandDesc *db = da + n;
        OutputDesc *dout = reinterpret_cast<OutputDesc *>(db + n);
        // pageable sources: each copy has read its source when the call returns
        cudaMemcpyAsync(da, ha.data(), n * sizeof(OperandDesc), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(db, hb.data(), n * sizeof(OperandDesc), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(dout, ho.data(), n * sizeof(OutputDesc), cudaMemcpyHostToDevice, s);
        // the groups on the branch streams, forked from s and joined back into it
        bool ev_ok = cudaEventCreateWithFlags(&B.fork, cudaEventDisableTiming) == cudaSuccess;
        for (int k = 0; ev_ok && k < kBatchBranches; k++)
            ev_ok = cudaEventCreateWithFlags(&B.join[k], cudaEventDisableTiming) == cudaSuccess;
        B.ws = mem + ws_off;
        B.d_a = da;
        B.d_b = db;
        B.d_out = dout;
        B.st = api::stream_status(s);
        rc = !ev_ok ? GF2X_ECUDA : (!B.st ? GF2X_ECUDA : enqueue_branches(&B, s));
        if (B.fork) cudaEventDestroy(B.fork);
        for (int k = 0; k < kBatchBranches; k++)
            if (B.join[k]) cudaEventDestroy(B.join[k]);
        api::ws_free(mem, s);
        if (rc == GF2X_OK && cudaGetLastError() != cudaSuccess) rc = GF2X_ECUDA;
        return rc;
    } catch (const std::bad_alloc &) {
        return GF2X_ENOMEM;
    } catch (...) {
        return GF2X_ECUDA;
    }
}

int gf2x_batch_create(int count, const uint64_t *na_bits, const uint64_t *nb_bits,
                      size_t mem_budget_bytes, gf2x_batch **out) {
    if (!out) return GF2X_EINVAL;
    *out = nullptr;
    if (count <= 0 || !na_bits || !nb_bits) return GF2X_EINVAL;
    try {
        std::unique_ptr<gf2x_batch> B(new gf2x_batch());
        if (cudaGetDevice(&B->device) != cudaSuccess) {
            cudaGetLastError();
            return GF2X_ECUDA;
        }
        if (!mem_budget_bytes) mem_budget_bytes = (size_t)1 << 32;
        int rc = batch_build(B.get(), count, na_bits, nb_bits, mem_budget_bytes, kBatchBranches);
        if (rc) return rc;
        const size_t n = std::max<size_t>(1, B->order.size());
        bool ok = cudaMalloc(&B->ws, (size_t)B->nbr * std::max<size_t>(256, branch_stride(B.get()))) ==
                      cudaSuccess &&
                  cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) == cudaSuccess &&
                  cudaMalloc(&B->d_a, n * sizeof(OperandDesc)) == cudaSuccess &&
                  cudaMalloc(&B->d_b, n * sizeof(OperandDesc)) == cudaSuccess &&
                  cudaMalloc(&B->d_out, n * sizeof(OutputDesc)) == cudaSuccess &&
                  cudaMallocHost(&B->h_a, n * sizeof(OperandDesc)) == cudaSuccess &&
                  cudaMallocHost(&B->h_b, n * sizeof(OperandDesc)) == cudaSuccess &&
                  cudaMallocHost(&B->h_out, n * sizeof(OutputDesc)) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&B->done, cudaEventDisableTiming) == cudaSuccess;
        for (int k = 0; ok && k < kBatchBranches; k++)
            ok = cudaStreamCreateWithFlags(&B->branch[k], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&B->join[k], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            gf2x_batch_destroy(B.release());
            return GF2X_ENOMEM;
        }
        if ((rc = api::take_status(&B->st))) {
            gf2x_batch_destroy(B.release());
            return rc;
        }
        *out = B.release();
        return GF2X_OK;
    } catch (const std::bad_alloc &) {
        return GF2X_ENOMEM;
    } catch (...) {
        return GF2X_ECUDA;
    }
}

int gf2x_batch_workspace_bytes(const gf2x_batch *B, size_t *bytes) {
    if (!B || !bytes) return GF2X_EINVAL;
    *bytes = (size_t)B->nbr * branch_stride(B);
    return GF2X_OK;
}

int gf2x_batch_execute(gf2x_batch *B, const uint64_t *const *a, const uint64_t *const *b,
                       uint64_t *const *out, gf2x_stream_t stream) {
    if (!B || !a || !b || !out) return GF2X_EINVAL;
    try {
        std::lock_guard<std::mutex> lk(B->mu);
        int dev = -1;
        cudaGetDevice(&dev);
        if (dev != B->device) return GF2X_EINVAL;
        // pointer kinds are not re-checked here (the graph path stays cheap)
        for (size_t k = 0; k < B->order.size(); k++) {
            const int i = B->order[k];
            if (!a[i] || !b[i] || !out[i]) return GF2X_EINVAL;
        }
        int rc;
        if (B->order.empty()) return GF2X_OK;
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        // the previous replay has read the pinned descriptors
        if (B->launched && cudaEventSynchronize(B->done) != cudaSuccess) {
            cudaGetLastError();
            return GF2X_ECUDA;
        }
        fill_descs(B, a, b, out, B->h_a, B->h_b, B->h_out);
        if (!B->exec) {
            const DevTables *T;
            if ((rc = api::tables(&T))) return rc;
            prepare_bcvt_attributes();
            prepare_fft_attributes();
            const size_t n = B->order.size();
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                cudaGetLastError();
                return GF2X_ECUDA;
            }
            cudaMemsetAsync(B->st, 0, sizeof(int), B->cap);
            cudaMemcpyAsync(B->d_a, B->h_a, n * sizeof(OperandDesc), cudaMemcpyHostToDevice, B->cap);
            cudaMemcpyAsync(B->d_b, B->h_b, n * sizeof(OperandDesc), cudaMemcpyHostToDevice, B->cap);
            cudaMemcpyAsync(B->d_out, B->h_out, n * sizeof(OutputDesc), cudaMemcpyHostToDevice,
                            B->cap);
            rc = enqueue_branches(B, B->cap);
            cudaError_t e = cudaStreamEndCapture(B->cap, &g);
            if (rc || e != cudaSuccess || !g) {
                cudaGetLastError();
                if (g) cudaGraphDestroy(g);
                return rc ? rc : GF2X_ECUDA;
            }
            e = cudaGraphInstantiate(&B->exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                cudaGetLastError();
                B->exec = nullptr;
                return GF2X_ECUDA;
            }
        }
        if (cudaGraphLaunch(B->exec, s) != cudaSuccess || cudaEventRecord(B->done, s) != cudaSuccess) {
            cudaGetLastError();
            return GF2X_ECUDA;
        }
        B->launched = true;
        return GF2X_OK;
    } catch (...) {
        return GF2X_ECUDA;
    }
}

int gf2x_batch_destroy(gf2x_batch *B) {
    if (!B) return GF2X_EINVAL;
    if (B->launched) cudaEventSynchronize(B->done);
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->done) cudaEventDestroy(B->done);
    if (B->cap) cudaStreamDestroy(B->cap);
    if (B->fork) cudaEventDestroy(B->fork);
    for (int k = 0; k < kBatchBranches; k++) {
        if (B->join[k]) cudaEventDestroy(B->join[k]);
        if (B->branch[k]) cudaStreamDestroy(B->branch[k]);
    }
    cudaFree(B->ws);
    cudaFree(B->d_a);
    cudaFree(B->d_b);
    cudaFree(B->d_out);
    cudaFreeHost(B->h_a);
    cudaFreeHost(B->h_b);
    cudaFreeHost(B->h_out);
    api::give_status(B->st);
    cudaGetLastError();
    delete B;
    return GF2X_OK;
}

int gf2x_batch_tune(gf2x_batch *B, int reps, double *ms_before, double *ms_after) {
    if (!B || !ms_before || !ms_after) return GF2X_EINVAL;
    if (reps <= 0) reps = 2;
    try {
        std::lock_guard<std::mutex> lk(B->mu);
        if (!B->launched) return GF2X_EINVAL;  // the descriptors come from an execution
        if (cudaEventSynchronize(B->done) != cudaSuccess) {
            cudaGetLastError();
            return GF2X_ECUDA;
        }
        const DevTables *T;
        int rc = api::tables(&T);
        if (rc) return rc;
        int *st = nullptr;
        if ((rc = api::take_status(&st))) return rc;
        cudaStream_t s = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaMemsetAsync(st, 0, sizeof(int), s);
        const OperandDesc none_in{nullptr, 0, 0};
        const OutputDesc none_out{nullptr, 0, 0};
        // one group's grouped launch with plan p: device time per execution
        auto trial = [&](const gf2x_batch::Chunk &ch, const gf2x_plan *p, double *ms) -> int {
            for (int r = 0; r <= reps; r++) {
                if (r == 1) cudaEventRecord(e0, s);
                if (plan_run_batch(p, ch.count, B->d_a + ch.first, B->d_b + ch.first,
                                   B->d_out + ch.first, none_in, none_in, none_out,
                                   ch.max_out_words, B->ws, p->ws_bytes, s, T, st, nullptr))
                    return GF2X_ECUDA;
            }
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
        double before = 0, after = 0;
        for (auto &ch : B->chunks) {
            if (!ch.plan || rc) continue;
            const int i0 = B->order[ch.first];
            double best_ms;
            if ((rc = trial(ch, ch.plan.get(), &best_ms))) break;
            before += best_ms;
            std::shared_ptr<gf2x_plan> best = ch.plan;
            // the fusion depths that change the strided-pass count, both tile
            // bufferings, then the BasisCvt tile shape with the best of those;
            // a candidate whose workspace exceeds the batch's is skipped
            std::vector<PlanTune> cands;
            for (int d = 7; d >= 4; d--)
                for (int nb = 2; nb >= 1; nb--) {
                    PlanTune t = ch.plan->tune;
                    t.fft_depth = d;
                    t.fft_nbuf = nb;
                    cands.push_back(t);
                }
            for (int pass = 0; pass < 2 && !rc; pass++) {
                if (pass == 1) {
                    cands.clear();
                    const int tiles[4] = {10, 11, 12, 13}, thr[3] = {128, 256, 512};
                    for (int a = 0; a < 4; a++)
                        for (int b2 = 0; b2 < 3; b2++) {
                            PlanTune t = best->tune;
                            t.bcvt.tile_min_log = tiles[a];
                            t.bcvt.small_threads = thr[b2];
                            cands.push_back(t);
                        }
                }
                for (const PlanTune &t : cands) {
                    std::shared_ptr<gf2x_plan> p;
                    if (api::make_plan(B->na[i0], B->nb[i0], t, &p)) continue;
                    if (p->ws_bytes * (size_t)ch.count > B->ws_bytes) continue;
                    double ms;
                    if ((rc = trial(ch, p.get(), &ms))) break;
                    if (ms < best_ms) {
                        best_ms = ms;
                        best = p;
                    }
                }
            }
            ch.plan = best;
            after += best_ms;
        }
        cudaStreamSynchronize(s);
        const int ds = api::read_status(st);
        api::give_status(st);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaStreamDestroy(s);
        if (rc) return rc;
        if (ds) return ds;
        // the next execution captures the graph again with the chosen plans
        if (B->exec) {
            cudaGraphExecDestroy(B->exec);
            B->exec = nullptr;
        }
        *ms_before = before;
        *ms_after = after;
        return GF2X_OK;
    } catch (const std::bad_alloc &) {
        return GF2X_ENOMEM;
    } catch (...) {
        return GF2X_ECUDA;
    }
}

int gf2x_batch_status(gf2x_batch *B) {
    if (!B) return GF2X_EINVAL;
    std::lock_guard<std::mutex> lk(B->mu);
    if (!B->launched) return GF2X_OK;
    if (cudaEventSynchronize(B->done) != cudaSuccess) {
        cudaGetLastError();
        return GF2X_ECUDA;
    }
    int v = 0;
    if (cudaMemcpy(&v, B->st, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return GF2X_ECUDA;
    }
    return v;
}

}  // extern "C"
