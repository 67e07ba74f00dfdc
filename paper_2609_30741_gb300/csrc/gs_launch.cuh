// Kernel launches with programmatic dependent launch.
//
// A frame is a chain of about fifty dependent kernels captured in one CUDA
// graph. Launched with the programmatic-stream-serialization attribute, a
// kernel is set up while its predecessor drains instead of after it has
// completed; every kernel of this library starts with griddep_wait(), which
// blocks until the predecessor grid has finished and its writes are visible,
// so the order of memory effects is that of a plain launch. griddep_wait() is a
// no-op in a kernel launched without the attribute.
#pragma once

#include <cuda_runtime.h>

namespace gs {

__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Process-wide switch (on by default); gs_set_programmatic_launch.
extern int g_pdl;

template <class... P, class... A>
cudaError_t launch_k(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A &&...args) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = g_pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<P>(args)...);
}

}  // namespace gs
