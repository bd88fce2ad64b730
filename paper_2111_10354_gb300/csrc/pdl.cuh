// Programmatic dependent launch (sm_90 and later). A kernel launched with the programmatic
// stream-serialisation attribute may be scheduled while the launch before it in the stream drains.
// Such a kernel calls griddep_wait before it touches memory: it returns once every launch the kernel
// depends on has completed and its writes are visible (at once for a launch without the attribute).
// griddep_launch_dependents lets the next such launch be scheduled onto the SM slots this grid's
// blocks free as they finish; it changes scheduling only, never what a dependent launch sees.
#pragma once
#include <utility>

#include "internal.cuh"

namespace hisq {

__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launches kern<<<grid, block>>>(args...) on the context's stream; with ctx->pdl, as a programmatic
// dependent launch (kern must start with griddep_wait). Inside the library's own solver captures the
// launch stays a plain graph node: there the solves gained nothing from programmatic edges (FP32 mixed
// CG within 0.1% at 48^3x12, 0.6% at 32^3x8) and the plain FP64 CG lost 2.4%.
template <typename... Params, typename... Args>
static cudaError_t launch_dependent(hisq_ctx* ctx, void (*kern)(Params...), int grid, int block,
                                    Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = ctx->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = ctx->pdl && !ctx->capturing ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

}  // namespace hisq
