// Kernel launches with programmatic dependent launch (sm_90 and later).
//
// Inside a captured chunk of sweeps every kernel depends on the one before
// it.  With the programmatic-serialisation attribute a kernel may be
// scheduled while its predecessor's last CTAs drain: it runs whatever reads
// only data no kernel of the chunk writes (the 1-ring records), then
// griddepcontrol.wait blocks until the predecessor has completed and its
// writes are visible.  Every kernel launched this way calls pdl_wait() before
// its first access to anything another kernel writes, and pdl_release() to
// let its own successor be scheduled.  Without the attribute both are no-ops.
#pragma once

#include "pbng_internal.h"

#include <utility>

namespace pbng {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... K, typename... A>
cudaError_t launch_kernel(void (*kernel)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

}  // namespace pbng
