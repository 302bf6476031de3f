// Library internals shared by api.cu, batch.cu and server.cu.
#pragma once
#include <cuda_runtime.h>

#include <memory>

#include "plan.h"

namespace gf2x {
namespace api {

// Size-independent device tables of the current device (uploaded on first use).
int tables(const DevTables **T);
// Status word of the asynchronous calls on stream s of the current device
// (gf2x_stream_status reads it); nullptr if the device has no tables.
int *stream_status(cudaStream_t s);
// A status word for one caller of its own (a server slot); GF2X_EBUSY when
// none is free.  give_status returns it once its work has finished.
int take_status(int **w);
void give_status(int *w);
// Reads and clears one status word once the work that writes it has finished.
int read_status(int *w);
// A new (uncached) plan for these sizes with the given parameters.
int make_plan(uint64_t na_bits, uint64_t nb_bits, const PlanTune &t,
              std::shared_ptr<gf2x_plan> *out);
// Cached plan for these operand sizes on the current device.
int plan_for(uint64_t na_bits, uint64_t nb_bits, std::shared_ptr<gf2x_plan> *p);
// Argument checks of one product (device pointers, sizes, overlap).
int check_product_args(const uint64_t *a, uint64_t na_bits, const uint64_t *b, uint64_t nb_bits,
                       const uint64_t *out);
// Per-stage timer feeding gf2x_profile_read (records only while profiling is on).
StageHook *new_timer(cudaStream_t s);
// Stream-ordered workspace from the library's pool of the current device
// (memory stays mapped between calls).
int ws_alloc(void **p, size_t bytes, cudaStream_t s);
void ws_free(void *p, cudaStream_t s);
// One product with plan p and workspace ws on stream s.
int run_one(const gf2x_plan *p, const uint64_t *a, const uint64_t *b, uint64_t *out, void *ws,
            cudaStream_t s);

}  // namespace api
}  // namespace gf2x
