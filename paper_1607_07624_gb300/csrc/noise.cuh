// Detector noise for the CCD object (Table 1 detector: photon_noise, readout_noise,
// readout_level). Counter-based Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11):
// key = seed, counter = (pixel, frame low, frame high, block). Uniforms
// u = (x + 0.5) 2^-32 in double. Read noise: Box-Muller on block 0 words 0, 1.
// Photon noise: Poisson by sequential-search inversion on block 0 word 2 for
// lambda < 16, else Hoermann's (1993) PTRS transformed rejection on the pairs
// (word 2, word 3) of blocks 0, 1, 2, ...; every decision in double.
#pragma once
#include <cstdint>

namespace pas {

struct u32x4 { uint32_t v[4]; };

__host__ __device__ inline u32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    uint64_t p0 = (uint64_t)M0 * c0;
    uint64_t p1 = (uint64_t)M1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  u32x4 o;
  o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
  return o;
}

__device__ inline double u01(uint32_t x) { return ((double)x + 0.5) * 2.3283064365386963e-10; }

__device__ inline u32x4 noise_block(uint64_t seed, uint32_t pixel, uint64_t frame, uint32_t blk) {
  return philox4x32_10(pixel, (uint32_t)frame, (uint32_t)(frame >> 32), blk, (uint32_t)seed,
                       (uint32_t)(seed >> 32));
}

__device__ inline double poisson_draw(double lam, uint64_t seed, uint32_t pixel, uint64_t frame) {
  if (!(lam > 0.0)) return 0.0;
  u32x4 w = noise_block(seed, pixel, frame, 0);
  if (lam < 16.0) {
    double u = u01(w.v[2]);
    int k = 0;
    double p = exp(-lam);
    double F = p;
    while (u > F && k < 1000) {
      ++k;
      p *= lam / k;
      F += p;
    }
    return (double)k;
  }
  double slam = sqrt(lam), loglam = log(lam);
  double b = 0.931 + 2.53 * slam;
  double a = -0.059 + 0.02483 * b;
  double invalpha = 1.1239 + 1.1328 / (b - 3.4);
  double vr = 0.9277 - 3.6224 / (b - 2.0);
  for (uint32_t blk = 0; blk < 64; ++blk) {
    if (blk > 0) w = noise_block(seed, pixel, frame, blk);
    double U = u01(w.v[2]) - 0.5;
    double V = u01(w.v[3]);
    double us = 0.5 - fabs(U);
    double k = floor((2.0 * a / us + b) * U + lam + 0.43);
    if (us >= 0.07 && V <= vr) return k;
    if (k < 0.0 || (us < 0.013 && V > us)) continue;
    if (log(V) + log(invalpha) - log(a / (us * us) + b) <= -lam + k * loglam - lgamma(k + 1.0))
      return k;
  }
  return floor(lam + 0.5);
}

__device__ inline double gaussian_draw(uint64_t seed, uint32_t pixel, uint64_t frame) {
  u32x4 w = noise_block(seed, pixel, frame, 0);
  return sqrt(-2.0 * log(u01(w.v[0]))) * cospi(2.0 * u01(w.v[1]));
}

}  // namespace pas
