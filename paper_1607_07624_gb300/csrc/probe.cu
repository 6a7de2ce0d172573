// FP32 throughput probe: the denominator of the FP32 roofline of the FFT passes.
// Every thread runs FMA_CHAINS independent fused multiply-add chains for `iters`
// rounds (operands not known at compile time, one store per thread at the end), so
// the kernel issues nothing but FFMA in its loop; its rate, timed by the caller with
// CUDA events, is what this GPU's FP32 pipes sustain at the clock of the moment.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace pas {

constexpr int FMA_CHAINS = 8;

__global__ void __launch_bounds__(256) fma_probe_kernel(float* sink, int iters, float x, float y) {
  const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
  float a[FMA_CHAINS];
#pragma unroll
  for (int q = 0; q < FMA_CHAINS; ++q) a[q] = (float)(tid + q) * 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < FMA_CHAINS; ++q) a[q] = fmaf(a[q], x, y);
  }
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < FMA_CHAINS; ++q) s += a[q];
  sink[tid] = s;
}

}  // namespace pas

extern "C" pas_status pas_fp32_fma_probe(void* cuda_stream, float* d_sink, int32_t n_blocks, int32_t iters,
                                         int64_t* h_flops) {
  if (!d_sink || !h_flops || n_blocks < 1 || iters < 1)
    return pas::set_global_error(PAS_EINVAL, "pas_fp32_fma_probe: bad arguments");
  // x slightly below 1 and y small keep the chains finite for any iteration count
  pas::fma_probe_kernel<<<n_blocks, 256, 0, (cudaStream_t)cuda_stream>>>(d_sink, iters, 0.999999f, 1e-6f);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return pas::set_global_error(PAS_ECUDA, "pas_fp32_fma_probe: %s", cudaGetErrorString(e));
  *h_flops = 2LL * pas::FMA_CHAINS * (int64_t)iters * n_blocks * 256;
  return PAS_OK;
}
