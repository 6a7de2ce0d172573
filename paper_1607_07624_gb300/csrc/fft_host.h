// Host-side tables of the warp FFT engine (fft.cuh): the per-pass twiddles and the
// frequency held at each buffer position after the forward passes.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "fft.cuh"

namespace pas {

// Twiddles of forward passes 0 .. M-2: entry tw_offset(pass) + (k - 1) S + n1 holds
// w_L^{n1 k} = exp(-2 pi i n1 k / L) of that pass (float32 of the double value),
// written into tw[0 .. tw_size(N)).
inline void fft_twiddles_into(int N, float2* tw) {
  const int M = plan_count(N);
  for (int pass = 0; pass + 1 < M; ++pass) {
    const int R = plan_radix(N, pass), L = block_len(N, pass), S = L / R, off = tw_offset(N, pass);
    for (int k = 1; k < R; ++k)
      for (int n1 = 0; n1 < S; ++n1) {
        const double a = -2.0 * M_PI * (double)(n1 * k) / (double)L;
        tw[off + (k - 1) * S + n1] = make_float2((float)std::cos(a), (float)std::sin(a));
      }
  }
}

inline std::vector<float2> fft_twiddles(int N) {
  std::vector<float2> tw((size_t)tw_size(N));
  fft_twiddles_into(N, tw.data());
  return tw;
}

// Frequency held at buffer position p after all forward passes (the mixed-radix
// digits of p read in reverse order).
inline int fft_freq_at(int N, int p) {
  const int M = plan_count(N);
  int rem = p, L = N, mult = 1, u = 0;
  for (int i = 0; i < M; ++i) {
    const int R = plan_radix(N, i), S = L / R;
    const int k = rem / S;
    rem -= k * S;
    u += k * mult;
    mult *= R;
    L = S;
  }
  return u;
}

}  // namespace pas
