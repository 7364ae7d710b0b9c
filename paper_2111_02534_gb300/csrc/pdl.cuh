// Programmatic dependent launch for the solver's kernel chains.  A kernel launched with
// launch_pdl may start while its predecessor in the stream is still running: its CTAs are
// scheduled, and pdl_wait() holds each thread until the predecessor grid has completed and
// its memory writes are visible.  pdl_trigger() in the predecessor lets that happen as soon
// as all of its CTAs have started.  Kernels that use these call pdl_entry() (trigger, then
// wait) before their first global memory access, or run only set-up that touches no global
// data produced by the predecessor before pdl_wait().  Both instructions are no-ops for a
// kernel launched without the attribute, so a kernel with pdl_entry() can also be launched
// normally.  What a launch saves is the gap between two dependent kernels (launch latency
// and the next grid's CTA start-up).
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace tps {

#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_entry() {
  pdl_trigger();
  pdl_wait();
}
#endif

// Host switch per thread: with several streams sharing the GPU (the batched sweep), dependent
// CTAs waiting early would hold SM slots that another stream's kernels could use, so the
// batch executor's workers launch normally.
inline thread_local bool pdl_enabled = true;

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = pdl_enabled ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace tps
