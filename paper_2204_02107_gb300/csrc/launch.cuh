// Kernel launches with programmatic dependent launch (griddepcontrol, sm_90 and later).
//
// A kernel launched by launch_pdl may be scheduled while its predecessor in the stream is still draining.  Every
// such kernel calls pdl_enter() as its first statement: griddepcontrol.wait returns once the predecessor grid has
// completed and its memory is visible (the ordering of a plain stream launch), and griddepcontrol.launch_dependents
// then lets the successor's CTAs be scheduled.  Since a grid triggers only after its own wait, at most the running
// grid and the next one, waiting, are resident at a time; a grid that does not trigger (a plain launch, or a
// predecessor that is not a kernel) releases its successor at completion.  Under stream capture the launches become
// programmatic edges of the graph.
//
// Off by default (VF_PDL=1 turns it on): on the 256 x 128 x 128 room step it measured slower than plain launches
// (8.54 vs 8.70 Gcell/s), so kernels launched by launch_pdl run as plain stream launches, for which
// griddepcontrol.wait and launch_dependents are no-ops.
#pragma once

#include <cuda_runtime.h>

namespace vf {

__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

bool pdl_on();   // true when VF_PDL is set to a non-zero value

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl_on() ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace vf
