// Programmatic dependent launch (sm_90+): a kernel launched with the
// programmatic-stream-serialization attribute may start while its predecessor in
// the stream is still running. It must call pdl_wait() before it reads anything
// the predecessor writes (or writes anything the predecessor reads); pdl_wait()
// returns once every prerequisite grid has completed and its memory is visible.
// pdl_trigger() lets the dependent grid be scheduled once every CTA of this grid
// has triggered or exited. Both are no-ops for a kernel launched normally.
#pragma once
#include <cuda_runtime.h>

namespace pas {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Prefetch the 128-byte line holding p into L2 (no register result, no wait).
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Prefetch the 128-byte line holding p into L1 (and L2).
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Prefetch bytes [p, p + n) line by line into L1, the CTA's threads sharing the lines.
__device__ __forceinline__ void prefetch_l1_span(const void* p, size_t n) {
  const char* c = static_cast<const char*>(p);
  for (size_t o = (size_t)threadIdx.x * 128; o < n; o += (size_t)blockDim.x * 128) prefetch_l1(c + o);
}

// Launch with or without the programmatic-serialization attribute.
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool pdl,
                     Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

}  // namespace pas
