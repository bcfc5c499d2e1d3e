// launch.cuh -- kernel launches with programmatic dependent launch (PDL).
//
// A batch-1 evaluation is a chain of about a hundred short kernels replayed from a CUDA
// graph, so the gap between one kernel's last CTA and the next kernel's first one is a
// visible share of the step.  Inside a stream capture whose pending dependencies are all
// kernel nodes, launches carry the programmatic-serialisation attribute: the next kernel's
// CTAs may be scheduled while the previous kernel drains.  Every kernel of the library
// therefore starts with pdl_enter(), which waits (griddepcontrol.wait) until the grids it
// depends on have completed and their memory is visible, before any global load or store,
// and then allows its own dependants to be scheduled.  Because every thread of every grid
// waits first, a grid completes only after its predecessor did, so the ordering is
// transitive along the chain.  Launched without the attribute both instructions return at
// once.  HEAR_PDL=0 in the environment turns the attribute off.
#pragma once
#include <cuda_runtime.h>
#include "internal.h"

namespace hear {

__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// host: true while `st` is being captured, PDL is enabled and every node the next captured
// node will depend on is a kernel node
bool pdl_allowed(cudaStream_t st);

template <typename... KArgs, typename... Args>
inline void launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_allowed(st) ? 1 : 0;
    HEAR_CHECK_CUDA(cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...));
}

}  // namespace hear
