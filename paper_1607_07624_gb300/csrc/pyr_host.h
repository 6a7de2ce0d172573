// Host-side tables of the modulated pyramid, written into caller-provided arrays:
// the object path (pas_pyr_create) fills vectors, the allocation-free path fills
// file-scope arrays, and both get the same numbers from the same code.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "fft4.cuh"
#include "fft_host.h"

namespace pas {

// Tilt points of a modulated point or extended source: modulation point k of source
// point q sits at (R cos theta_k + ex_q, R sin theta_k + ey_q) lambda/D, index
// t = q K + k (theta_k = 2 pi k / K from axis 0). The rows pass runs once per
// distinct (sin theta, ey): theta and pi - theta share one (even K), and so do source
// points of equal ey. Outputs (Kt = K P entries unless stated):
//   kmap[t]   rows-pass index of tilt point t;
//   alpha[t]  column tilt phase slope (cycles per pixel, centring ramp included);
//   amp[t]    column-tilt amplitude sqrt(w_q P) (NULL: not written);
//   beta[s]   row tilt phase slope of rows pass s (s < return value <= Kt);
//   key_rep / key_ey: scratch of Kt entries each.
// P = 1 with ex = ey = NULL is the point source. Returns the number of rows passes.
inline int pyr_tilt_tables(int Np, int N, int K, double mod_radius, int P, const double* ex, const double* ey,
                           const double* w_norm, int* kmap, float* alpha, float* amp, float* beta, int* key_rep,
                           int* key_ey) {
  const bool ext = ex != nullptr && ey != nullptr;
  int n_s = 0;
  for (int q = 0; q < P; ++q) {
    int eq = q;
    for (int r = 0; r < q; ++r)
      if (ext && ey[r] == ey[q]) {
        eq = r;
        break;
      }
    for (int k = 0; k < K; ++k) {
      int rep = k;
      if (K % 2 == 0) rep = std::min(k, ((K / 2 - k) % K + K) % K);
      int s = -1;
      for (int t = 0; t < n_s; ++t)
        if (key_rep[t] == rep && key_ey[t] == eq) s = t;
      if (s < 0) {
        s = n_s++;
        key_rep[s] = rep;
        key_ey[s] = eq;
      }
      kmap[q * K + k] = s;
    }
  }
  const double ramp = 1.0 / (2.0 * N);
  for (int q = 0; q < P; ++q) {
    const double oxq = ext ? ex[q] : 0.0;
    for (int k = 0; k < K; ++k) {
      const double th = 2.0 * M_PI * (double)k / (double)K;
      alpha[q * K + k] = (float)((mod_radius * std::cos(th) + oxq) / Np - ramp);
      if (amp) amp[q * K + k] = (float)std::sqrt((w_norm ? w_norm[q] : 1.0 / P) * P);
    }
  }
  for (int s = 0; s < n_s; ++s) {
    const double th = 2.0 * M_PI * (double)key_rep[s] / (double)K;
    const double oyq = ext ? ey[key_ey[s]] : 0.0;
    beta[s] = (float)((mod_radius * std::sin(th) + oyq) / Np - ramp);
  }
  return n_s;
}

// Pyramid mask in the FFT engine's padded digit-reversed layout (buf_n entries):
// delta = N/4 gives the phase (pi/2)|u~| at centred frequency u~; divided by N (the
// unitary normalisation of the forward and inverse transforms together).
inline void pyr_mask_table(int N, int buf_n, float2* mk) {
  for (int j = 0; j < buf_n; ++j) mk[j] = make_float2(0.f, 0.f);
  for (int j = 0; j < N; ++j) {
    const double ut = std::fabs((double)fft_freq_at(N, j) - 0.5 * (N - 1));
    const double ph = 0.5 * M_PI * ut;
    mk[phys(j)] = make_float2((float)(std::cos(ph) / N), (float)(std::sin(ph) / N));
  }
}

// Tables of the four-step engine (fft4.cuh) for N = 32 Q: tw4[(k2 - 1) 32 + n1] =
// exp(-2 pi i n1 k2 / N), k2 = 1..Q-1; mk4[k2 33 + k1] = the pyramid mask at natural
// frequency u = Q k1 + k2, exp(i (pi/2) |u - (N-1)/2|) / N (pads zero).
inline void four_step_tables(int N, float2* tw4, float2* mk4) {
  const int Q = four_q(N);
  for (int k2 = 1; k2 < Q; ++k2)
    for (int n1 = 0; n1 < 32; ++n1) {
      const double a = -2.0 * M_PI * (double)(n1 * k2) / (double)N;
      tw4[(k2 - 1) * 32 + n1] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
  for (int t = 0; t < four_mask_size(N); ++t) mk4[t] = make_float2(0.f, 0.f);
  for (int k2 = 0; k2 < Q; ++k2)
    for (int k1 = 0; k1 < 32; ++k1) {
      const double ph = 0.5 * M_PI * std::fabs((double)(Q * k1 + k2) - 0.5 * (N - 1));
      mk4[k2 * F4_PITCH + k1] = make_float2((float)(std::cos(ph) / N), (float)(std::sin(ph) / N));
    }
}

// Detector pixels of the valid sub-apertures in all four quadrants (nd = 2 n_sub).
inline void quadrant_valid_map(int n_sub, const int32_t* valid, int n_valid, unsigned char* vpix) {
  const int nd = 2 * n_sub, ns = n_sub;
  for (int t = 0; t < nd * nd; ++t) vpix[t] = 0;
  for (int j = 0; j < n_valid; ++j) {
    const int r = valid[j] / ns, c = valid[j] % ns;
    vpix[r * nd + c] = vpix[r * nd + ns + c] = vpix[(ns + r) * nd + c] = vpix[(ns + r) * nd + ns + c] = 1;
  }
}

// Modulation grouping of the columns pass: nd x G CTAs, each warp doing
// kper = ceil(K / G) transforms in ceil(kper / tpw) engine calls (tpw transforms per
// call); G minimises (waves of CTAs) x calls for `slots` resident CTAs on the GPU.
inline void pick_modulation_groups(int K, int nd, int slots, int* kper_out, int* G_out, int tpw = 1) {
  double best = 1e30;
  for (int G = 1; G <= K; ++G) {
    const int kper = (K + G - 1) / G, Gc = (K + kper - 1) / kper;
    const int waves = (nd * Gc + slots - 1) / slots;
    const double cost = (double)waves * ((kper + tpw - 1) / tpw) + 1e-3 * Gc;  // engine calls per warp
    if (cost < best) {
      best = cost;
      *kper_out = kper;
      *G_out = Gc;
    }
  }
}

}  // namespace pas
