// gf2x_mul_noalloc: the whole product without allocating device memory.
//
// Who needs it: a caller that cannot call cudaMalloc (or any allocator) at
// the time it multiplies -- for instance a service that has handed all device
// memory to its own pool up front, a plugin whose host application owns every
// device allocation, or code on a latency path where an allocation would
// implicitly synchronise the device.  Such a caller passes only its inputs and
// output; the product's scratch (the two N-point transform arrays and the two
// padded operand copies) lives in a file-scope device array instead.
//
// The scratch array, the size-independent tables and the per-pass multiplier
// tables are static __device__ arrays: every GPU that loads the library keeps
// them (about 17.5 MiB) until the process exits.  Their device addresses are
// looked up with cudaGetSymbolAddress once per device (the host-side names of
// the arrays are stand-ins, not device addresses), at the first call on that
// device, with that device current; that first call also copies the tables in
// with synchronous copies, so it must not be made while a stream is being
// captured.
//
// Limits and sharing: products with more than GF2X_NOALLOC_MAX_FFT_POINTS
// transform points are rejected (GF2X_EINVAL).  All calls share the one
// scratch array and status word.  Work that overlapped on the GPU would race
// on them, so every call holds a process-wide lock from before its first
// launch until its stream has drained: calls from other host threads or on
// other streams wait for it (they never overlap on the GPU), and a thread
// holding the lock blocks the others until its product is done.  No part of
// the scratch needs to start at zero: every kernel writes what it later
// reads; the status word is cleared on the stream at the start of each call.
#include <mutex>

#include "../../include/gf2x_gb300.h"
#include "kernels.h"
#include "plan.h"

using namespace gf2x;

namespace {

constexpr size_t kScratchBytes = (size_t)GF2X_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxLog = 18;  // log2 of GF2X_NOALLOC_MAX_FFT_POINTS
static_assert((1ull << kMaxLog) == GF2X_NOALLOC_MAX_FFT_POINTS, "limit");
// The workspace of the largest allowed product: two 16-byte arrays of N =
// 2^18 points, the padded operands (Pa + Pb <= N + 1 words: the most uneven
// shape, N words times one word, pads the long operand to N) and the
// changeRepr'd blocks of the longer one (max(Pa, Pb) <= N elements), plus the
// 256-byte alignment of five sub-buffers.
static_assert(2 * (16ull << kMaxLog) + 8 * ((1ull << kMaxLog) + 1) + (16ull << kMaxLog) + 1280 <=
                  kScratchBytes,
              "scratch holds the largest allowed product");

// Pass table sets that products with N <= 2^18 use: contiguous bottom passes
// (k_lo = 0, g = 0 .. 12, uf = bottom_uf(g)) and one strided pass above them
// (k_lo = 12, g = 1 .. 6, uf = 0).
constexpr int kLocalSets = kFftTileLog + 1;
constexpr int kGlobalSets = kMaxLog - kFftTileLog;
constexpr size_t kPassWords = 288 * 1024;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];
static __device__ __align__(256) DevTables g_tables;
static __device__ __align__(256) uint32_t g_pass_words[kPassWords];
static __device__ int g_status;

struct SetOffsets {
    size_t val, shfl;
};

struct DevState {
    bool ready = false;
    unsigned char *scratch = nullptr;
    DevTables *tables = nullptr;
    uint32_t *pass_words = nullptr;
    int *status = nullptr;
    SetOffsets local[kLocalSets];
    SetOffsets global[kGlobalSets + 1];
};

constexpr int kMaxDevices = 64;
std::mutex g_mu;
DevState g_dev[kMaxDevices];
DevTables g_host_tables;               // host image, static storage
uint32_t g_host_pass_words[kPassWords];  // host image, static storage

DevState *state_of_current(int *dev_out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return nullptr;
    }
    if (dev_out) *dev_out = dev;
    return &g_dev[dev];
}

// Table source for the plan: pointers into the static pass-table array.
int static_pass_tables(int k_lo, int g, int uf, const uint32_t **d_val, const uint32_t **d_shfl) {
    DevState *st = state_of_current(nullptr);
    if (!st || !st->ready) return -3;
    const SetOffsets *o = nullptr;
    if (k_lo == 0 && g >= 0 && g < kLocalSets && uf == bottom_uf(g)) o = &st->local[g];
    if (k_lo == kFftTileLog && g >= 1 && g <= kGlobalSets && uf == 0) o = &st->global[g];
    if (!o) return -1;
    *d_val = st->pass_words + o->val;
    *d_shfl = st->pass_words + o->shfl;
    return 0;
}

int setup_current_device() {
    int dev;
    DevState *st = state_of_current(&dev);
    if (!st) return GF2X_ECUDA;
    if (st->ready) return GF2X_OK;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) goto fail;
    st->scratch = static_cast<unsigned char *>(p);
    if (cudaGetSymbolAddress(&p, g_tables) != cudaSuccess) goto fail;
    st->tables = static_cast<DevTables *>(p);
    if (cudaGetSymbolAddress(&p, g_pass_words) != cudaSuccess) goto fail;
    st->pass_words = static_cast<uint32_t *>(p);
    if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess) goto fail;
    st->status = static_cast<int *>(p);
    {
        // host images of the tables, then one copy of each to the device
        fill_dev_tables(&g_host_tables);
        size_t off = 0;
        auto add = [&](int k_lo, int g, int uf, SetOffsets *o) -> bool {
            size_t nv, ns;
            pass_tables_size(g, uf, &nv, &ns);
            if (off + nv + ns > kPassWords) return false;
            // both arrays start on 16-byte boundaries (the passes read two
            // words of each shuffle table as one 8-byte load)
            const size_t shfl = (off + nv + 3) & ~(size_t)3;
            if (shfl + ns > kPassWords) return false;
            o->val = off;
            o->shfl = shfl;
            pass_tables_fill(k_lo, g, uf, g_host_pass_words + o->val, g_host_pass_words + o->shfl);
            off = (shfl + ns + 3) & ~(size_t)3;
            return true;
        };
        for (int g = 0; g < kLocalSets; g++)
            if (!add(0, g, bottom_uf(g), &st->local[g])) return GF2X_ENOMEM;
        for (int g = 1; g <= kGlobalSets; g++)
            if (!add(kFftTileLog, g, 0, &st->global[g])) return GF2X_ENOMEM;
        if (cudaMemcpy(st->tables, &g_host_tables, sizeof(DevTables), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemcpy(st->pass_words, g_host_pass_words, off * sizeof(uint32_t),
                       cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemset(st->status, 0, sizeof(int)) != cudaSuccess)
            goto fail;
    }
    prepare_bcvt_attributes();
    prepare_fft_attributes();
    if (cudaGetLastError() != cudaSuccess) return GF2X_ECUDA;
    st->ready = true;
    return GF2X_OK;
fail:
    cudaGetLastError();
    return GF2X_ECUDA;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    // device memory must be the current device's own (the kernels run there)
    int dev = -1;
    if (at.type != cudaMemoryTypeDevice || cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.device == dev;
}

bool overlaps(const void *a, size_t na, const void *b, size_t nb) {
    auto x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return na && nb && x < y + nb && y < x + na;
}

}  // namespace

extern "C" int gf2x_mul_noalloc(const uint64_t *a, uint64_t na_bits, const uint64_t *b,
                                uint64_t nb_bits, uint64_t *out, gf2x_stream_t stream) {
    try {
        if (!na_bits || !nb_bits) return GF2X_OK;
        if (gf2x_fft_points(na_bits, nb_bits) > GF2X_NOALLOC_MAX_FFT_POINTS) return GF2X_EINVAL;
        const size_t ba = 8 * words_of(na_bits), bb = 8 * words_of(nb_bits);
        const size_t bo = 8 * gf2x_out_words(na_bits, nb_bits);
        if (!a || !b || !out || !is_device_ptr(a) || !is_device_ptr(b) || !is_device_ptr(out))
            return GF2X_EINVAL;
        if (overlaps(out, bo, a, ba) || overlaps(out, bo, b, bb)) return GF2X_EINVAL;
        std::lock_guard<std::mutex> lk(g_mu);
        int rc = setup_current_device();
        if (rc) return rc;
        DevState *st = state_of_current(nullptr);
        gf2x_plan plan;
        rc = plan_init(&plan, na_bits, nb_bits, static_pass_tables);
        if (rc) return rc == -1 ? GF2X_EINVAL : GF2X_ECUDA;
        if (plan.ws_bytes > kScratchBytes) return GF2X_EINVAL;
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        if (cudaMemsetAsync(st->status, 0, sizeof(int), s) != cudaSuccess) {
            cudaGetLastError();
            return GF2X_ECUDA;
        }
        if (plan_run_core(&plan, a, b, out, st->scratch, s, st->tables, st->status, nullptr))
            return GF2X_ECUDA;
        int dev_status = 0;
        if (cudaStreamSynchronize(s) != cudaSuccess ||
            cudaMemcpy(&dev_status, st->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            return GF2X_ECUDA;
        }
        return dev_status ? GF2X_ETIMEOUT : GF2X_OK;
    } catch (...) {
        return GF2X_ECUDA;
    }
}
