// pdl.cuh -- programmatic dependent launch for the chain of sweep kernels on
// one stream (init, level 0 -> 1, forward levels, backward levels,
// summaries). A kernel launched with the programmatic-serialization
// attribute may be scheduled while the kernel before it is still running:
// its blocks take the SM slots that the earlier kernel's finished blocks
// free, and wait() holds them until that kernel has completed and its
// memory operations are visible. The launch latency and the block ramp-up of
// every level then overlap the tail of the level before it.
//
// Every kernel started through launch() calls wait() before it touches
// global memory, then launch_dependents() so that the next kernel may be
// scheduled; no kernel waits on a later one, so the chain cannot deadlock.
// In a kernel started without the attribute both are no-ops.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace bcgb {
namespace pdl {

__device__ __forceinline__ void wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Both steps, at the top of a chained kernel.
__device__ __forceinline__ void enter() {
    wait();
    launch_dependents();
}

template <class... P, class... A>
cudaError_t launch(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A &&...args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

}  // namespace pdl
}  // namespace bcgb
