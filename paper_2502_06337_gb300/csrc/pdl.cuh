// Programmatic dependent launch (sm_90 and later). A kernel launched with the programmatic
// stream-serialization attribute may be scheduled while its predecessor in the stream is
// still running, once every block of the predecessor has called pdl_launch_dependents (or
// exited). Before it reads anything that an earlier kernel of the stream writes, it must call
// pdl_wait, which returns once the predecessor grid has completed and its memory is visible.
// Every kernel launched this way calls pdl_wait on every path, so that its own completion
// still implies the completion of all earlier kernels. Launched without the attribute, both
// instructions return at once.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace sprot {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launches kernel k as a programmatic dependent of the stream's previous kernel.
template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*k)(KArgs...), int grid, int block, size_t smem, cudaStream_t st,
                             Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at{};
  at.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at.val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

}  // namespace sprot
