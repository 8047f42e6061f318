// Programmatic dependent launch: every kernel of the library is launched
// with programmatic stream serialization, so it may start while the kernel
// before it on the stream is still running.  Each kernel first does what
// depends on nothing earlier kernels write (its own work descriptors,
// barrier and tensor-memory set-up), then waits for the preceding grid to
// complete and flush (griddepcontrol.wait) before it reads or writes any
// buffer an earlier kernel touches, and only then lets its own dependent
// launch (griddepcontrol.launch_dependents).  Completion is transitive along
// the chain, so a kernel past its wait sees everything launched before it.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace sym {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace sym
