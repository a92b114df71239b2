// Programmatic dependent launch: consecutive kernels of one stream overlap the next kernel's
// launch and ramp-up with the tail of the previous one.
//
// Every kernel of the library begins with pdl_entry(): it first waits until the grids it depends
// on have completed and their memory is visible (griddepcontrol.wait; without a programmatic
// dependency it returns at once), then allows its own dependents to start launching
// (griddepcontrol.launch_dependents).  Because the wait comes before any memory access, stream
// order semantics are unchanged; the dependents' CTAs only take SM slots this grid no longer
// needs and sit in their own wait until this grid completes.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace lfx {

__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// kernel<<<grid, block, smem, st>>>(args...) with programmatic stream serialization allowed
template <class... K, class... A>
inline void pdl_launch(void (*kernel)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

}  // namespace lfx
