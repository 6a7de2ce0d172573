// Four-step FFT -> mask -> inverse FFT inside one warp, for the pyramid's transform
// lengths N = 32 Q with Q = 8 (N = 256, four transforms per warp), Q = 15 (N = 480, two)
// or Q = 30 (N = 960, one). With n = n1 + 32 n2 and k = Q k1 + k2:
//
//   X[Q k1 + k2] = sum_n1 W_32^(n1 k1) W_N^(n1 k2) [sum_n2 x[n1 + 32 n2] W_Q^(n2 k2)]
//
// so lane n1 takes the Q-point DFT of its own elements in registers, multiplies by
// W_N^(n1 k2), and one shared-memory transpose hands column k2 to lane k2 (Q TPW
// columns per warp: 4 x 8, 2 x 15 or 1 x 30), which does the 32-point DFT over n1, the pyramid mask of
// frequency Q k1 + k2, and the 32-point inverse DFT in registers; the transpose back
// and the conjugate steps in reverse give x'[n1 + 32 n2] in lane n1. Against the
// pass-by-pass engine (fft.cuh) each element crosses shared memory twice per direction
// pair instead of once per radix pass, and the 32-point stage runs with no twiddle
// loads.
//
// Shared memory of a warp: four_buf(N) float2, the transpose buffer T[columns][33]
// (column c at c*33: both transposes are free of bank conflicts), at least TPW N long
// (the callers' staging). Tables shared by the CTA: tw4[(k2-1)*32 + n1] = W_N^(n1 k2)
// for k2 = 1..Q-1, mk4[k2*33 + k1] = mask(Q k1 + k2) (the mask at natural frequency u,
// divided by N).
#pragma once
#include <cuda_runtime.h>

#include "fft.cuh"

namespace pas {

constexpr int F4_PITCH = 33;     // float2 per column of the transpose buffer

__host__ __device__ constexpr bool four_step_ok(int N) { return N == 256 || N == 480 || N == 960; }
__host__ __device__ constexpr int four_q(int N) { return N / 32; }
__host__ __device__ constexpr int four_tpw(int N) { return N == 256 ? 4 : N == 480 ? 2 : 1; }  // transforms per warp
__host__ __device__ constexpr int four_cols(int N) { return four_q(N) * four_tpw(N); }         // columns per warp
__host__ __device__ constexpr int four_buf(int N) {
  return four_cols(N) * F4_PITCH > four_tpw(N) * N ? four_cols(N) * F4_PITCH : four_tpw(N) * N;
}
__host__ __device__ constexpr int four_tw_size(int N) { return (four_q(N) - 1) * 32; }
__host__ __device__ constexpr int four_mask_size(int N) { return four_q(N) * F4_PITCH; }

// cos and sin of 2 pi k / 32, k = 0..15
__device__ __forceinline__ float2 w32(int k) {
  const float c[16] = {1.0f, 0.98078528040323044913f, 0.92387953251128675613f, 0.83146961230254523708f,
                       0.70710678118654752440f, 0.55557023301960222474f, 0.38268343236508977173f,
                       0.19509032201612826785f, 0.0f, -0.19509032201612826785f, -0.38268343236508977173f,
                       -0.55557023301960222474f, -0.70710678118654752440f, -0.83146961230254523708f,
                       -0.92387953251128675613f, -0.98078528040323044913f};
  const float s[16] = {0.0f, 0.19509032201612826785f, 0.38268343236508977173f, 0.55557023301960222474f,
                       0.70710678118654752440f, 0.83146961230254523708f, 0.92387953251128675613f,
                       0.98078528040323044913f, 1.0f, 0.98078528040323044913f, 0.92387953251128675613f,
                       0.83146961230254523708f, 0.70710678118654752440f, 0.55557023301960222474f,
                       0.38268343236508977173f, 0.19509032201612826785f};
  return make_float2(c[k], s[k]);
}

// 32-point DFT in registers, natural order in and out: even and odd halves by
// 16-point transforms, then X[k] = E[k] + w O[k], X[k+16] = E[k] - w O[k] with
// w = exp(-+ 2 pi i k / 32).
template <bool INV>
__device__ __forceinline__ void dft32(float2* x) {
  float2 e[16], o[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    e[j] = x[2 * j];
    o[j] = x[2 * j + 1];
  }
  Bfly<16, INV>::run(e);
  Bfly<16, INV>::run(o);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const float2 w = w32(k);
    const float2 t = INV ? cmul(o[k], w) : cmulc(o[k], w);
    x[k] = cadd(e[k], t);
    x[k + 16] = csub(e[k], t);
  }
}

// 30-point DFT in registers by the prime-factor mapping 30 = 2 x 15: inputs
// n = (15 n1 + 2 n2) mod 30, outputs k = (15 k1 + 16 k2) mod 30, no twiddles.
template <bool INV>
__device__ __forceinline__ void dft30(float2* x) {
  float2 y0[15], y1[15];
#pragma unroll
  for (int n2 = 0; n2 < 15; ++n2) {
    y0[n2] = x[(2 * n2) % 30];
    y1[n2] = x[(15 + 2 * n2) % 30];
  }
  Bfly<15, INV>::run(y0);
  Bfly<15, INV>::run(y1);
#pragma unroll
  for (int k2 = 0; k2 < 15; ++k2) {
    x[(16 * k2) % 30] = cadd(y0[k2], y1[k2]);
    x[(15 + 16 * k2) % 30] = csub(y0[k2], y1[k2]);
  }
}

template <int Q, bool INV>
__device__ __forceinline__ void dft_q(float2* x) {
  if constexpr (Q == 8) Bfly<8, INV>::run(x);
  else if constexpr (Q == 15) Bfly<15, INV>::run(x);
  else dft30<INV>(x);
}

// FFT -> mask -> inverse FFT of four_tpw(N) length-N vectors by one warp.
// load(t, j): element lane + 32 j of transform t; store(t, j, v): output element
// lane + 32 j of transform t (t and j are compile-time constants in the unrolled calls).
// T: this warp's four_buf(N) float2 of shared memory; tw4, mk4: the CTA's tables.
template <int N, class Load, class Store>
__device__ __forceinline__ void four_step_mask(float2* T, const float2* tw4, const float2* mk4, int lane, Load& load,
                                               Store& store) {
  constexpr int Q = four_q(N), TPW = four_tpw(N), COLS = four_cols(N);
  static_assert(COLS <= 32, "one column per lane");
  {
    float2 v[COLS];
#pragma unroll
    for (int t = 0; t < TPW; ++t)
#pragma unroll
      for (int n2 = 0; n2 < Q; ++n2) v[t * Q + n2] = load(t, n2);
#pragma unroll
    for (int t = 0; t < TPW; ++t) {
      dft_q<Q, false>(v + t * Q);
#pragma unroll
      for (int k2 = 1; k2 < Q; ++k2) v[t * Q + k2] = cmul(v[t * Q + k2], tw4[(k2 - 1) * 32 + lane]);
    }
#pragma unroll
    for (int c = 0; c < COLS; ++c) T[c * F4_PITCH + lane] = v[c];
  }
  __syncwarp();
  if (lane < COLS) {
    const int k2 = lane % Q;
    float2* col = T + lane * F4_PITCH;
    float2 w[32];
#pragma unroll
    for (int n1 = 0; n1 < 32; ++n1) w[n1] = col[n1];
    dft32<false>(w);
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) w[k1] = cmul(w[k1], mk4[k2 * F4_PITCH + k1]);
    dft32<true>(w);
#pragma unroll
    for (int n1 = 0; n1 < 32; ++n1) col[n1] = w[n1];
  }
  __syncwarp();
  {
    float2 v[COLS];
#pragma unroll
    for (int c = 0; c < COLS; ++c) v[c] = T[c * F4_PITCH + lane];
    __syncwarp();  // T is read: `store` may write into it
#pragma unroll
    for (int t = 0; t < TPW; ++t) {
#pragma unroll
      for (int k2 = 1; k2 < Q; ++k2) v[t * Q + k2] = cmulc(v[t * Q + k2], tw4[(k2 - 1) * 32 + lane]);
      dft_q<Q, true>(v + t * Q);
#pragma unroll
      for (int n2 = 0; n2 < Q; ++n2) store(t, n2, v[t * Q + n2]);
    }
  }
  __syncwarp();  // T is reused by the next call
}

// ----------------------------------------------- forward transforms in pairs
// Two forward DFTs of length N = 15 R (R = 16: N = 240, R = 32: N = 480) by one warp,
// with no mask and no inverse (the PSF camera's padded transforms). With
// n = n1 + R n2 (n1 < R, n2 < 15) and k = 15 k1 + k2 (k1 < R, k2 < 15):
//
//   X[15 k1 + k2] = sum_n1 W_R^(n1 k1) W_N^(n1 k2) [sum_n2 x[n1 + R n2] W_15^(n2 k2)]
//
// Lane n1 of a group of R lanes takes the 15-point DFT of its elements (R = 16: lanes
// 0-15 transform 0 and lanes 16-31 transform 1; R = 32: every lane holds both), scales
// by W_N^(n1 k2), and one shared-memory transpose hands the 30 columns (transform,
// k2) to lanes 0-29, which take the R-point DFT over n1.
// T: this warp's pair_buf(N) float2 (column c at c (R + 1): no bank conflicts either
// way); tw[(k2 - 1) R + n1] = W_N^(n1 k2), k2 = 1..14 (pair_tw_size(N) entries).
// load(t, n): element n of transform t; store(t, m, v): frequency m of transform t,
// called by lanes 0-29 for m = 15 k1 + k2, k1 = 0..R-1.
__host__ __device__ constexpr bool pair_ok(int N) { return N == 240 || N == 480; }
__host__ __device__ constexpr int pair_r(int N) { return N / 15; }
__host__ __device__ constexpr int pair_buf(int N) { return 30 * (pair_r(N) + 1); }
__host__ __device__ constexpr int pair_tw_size(int N) { return 14 * pair_r(N); }

template <int N, class Load, class Store>
__device__ __forceinline__ void pair_forward(float2* T, const float2* tw, int lane, Load& load, Store& store) {
  constexpr int Q = 15, R = pair_r(N), P = R + 1, TL = R == 32 ? 2 : 1;
  static_assert(R == 16 || R == 32, "N = 240 or 480");
  const int n1 = lane & (R - 1), g = lane / R;
#pragma unroll
  for (int tl = 0; tl < TL; ++tl) {
    const int t = TL == 2 ? tl : g;
    float2 v[Q];
#pragma unroll
    for (int n2 = 0; n2 < Q; ++n2) v[n2] = load(t, n1 + R * n2);
    Bfly<15, false>::run(v);
#pragma unroll
    for (int k2 = 1; k2 < Q; ++k2) v[k2] = cmul(v[k2], __ldg(tw + (k2 - 1) * R + n1));
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) T[(t * Q + k2) * P + n1] = v[k2];
  }
  __syncwarp();
  if (lane < 2 * Q) {
    const int t = lane >= Q ? 1 : 0, k2 = lane - Q * t;
    const float2* col = T + lane * P;
    float2 w[R];
#pragma unroll
    for (int i = 0; i < R; ++i) w[i] = col[i];
    if constexpr (R == 16) Bfly<16, false>::run(w);
    else dft32<false>(w);
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) store(t, Q * k1 + k2, w[k1]);
  }
  __syncwarp();  // T is reused by the next call
}

}  // namespace pas
