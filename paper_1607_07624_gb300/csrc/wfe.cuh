// The loop step's residual wavefront error, closed by one CTA of the sensor stage
// from the residual kernel's per-tile (sum r, sum r^2) partials: RMS over the pupil
// pixels with the mean (piston) removed, written to the loop's WFE history at the
// step's index. Shared by the pyramid's slopes kernel and the Shack-Hartmann kernel.
#pragma once
#include <cuda_runtime.h>

#include "pyr.cuh"

namespace pas {

// Block sum of one double per thread (shuffle tree within warps, then warp 0 over the
// warps' sums); the result in every thread. red: >= 32 doubles of shared memory.
__device__ inline double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (warp == 0) {
    r = lane < nw ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    if (lane == 0) red[0] = r;
  }
  __syncthreads();
  r = red[0];
  return r;
}

// Called by every thread of one CTA (it synchronises the CTA).
__device__ inline void wfe_finalize(const LoopExtra& w, double* red) {
  // thread t adds partials t, t + blockDim.x, ... in that order; eight loads are in
  // flight before the adds (one latency per eight partials, not per partial)
  constexpr int U = 8;
  double s1 = 0.0, s2 = 0.0;
  for (int t0 = threadIdx.x; t0 < w.n_wfe_part; t0 += U * blockDim.x) {
    double2 p[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = t0 + u * blockDim.x;
      p[u] = t < w.n_wfe_part ? w.wfe_part[t] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      s1 += p[u].x;
      s2 += p[u].y;
    }
  }
  s1 = block_sum(s1, red);
  s2 = block_sum(s2, red);
  if (threadIdx.x == 0) {
    const double m = s1 * w.inv_npix;
    const double var = fmax(s2 * w.inv_npix - m * m, 0.0);
    w.wfe_hist[(*w.step) % w.wfe_hist_len] = sqrt(var);
  }
}

}  // namespace pas
