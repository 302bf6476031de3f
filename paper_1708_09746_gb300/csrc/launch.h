// Kernel launches of the product path with programmatic dependent launch:
// the next kernel of a stream is scheduled while the previous one drains and
// runs its table prologue there, then waits in pdl_acquire (gf2x_dev.cuh) for
// the previous kernels' results.  GF2X_PDL=0 in the environment launches
// without the attribute (plain stream order).
#pragma once
#include <cuda_runtime.h>

#include <utility>

namespace gf2x {

bool pdl_enabled();

// Only for kernels that call pdl_acquire before touching data written or
// read by earlier kernels of the stream.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                            cudaStream_t s, Args &&...args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

}  // namespace gf2x
