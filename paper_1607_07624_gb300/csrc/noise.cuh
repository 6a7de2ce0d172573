// Detector noise for the CCD object (Table 1 detector: photon_noise, readout_noise,
// readout_level). Counter-based Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11):
// key = seed, counter = (pixel, frame low, frame high, block).
// All decisions in float32 with IEEE products, quotients and sums (no contraction):
//   uniform u = ((x >> 8) + 1/2) 2^-24 (exact);
//   read noise: Box-Muller on block 0 words 0, 1;
//   photons, lambda < 10: sequential-search inversion on block 0 word 2, starting
//     from expf(-lambda), each term p_k = p_{k-1} (lambda rn(1/k)) with the
//     correctly rounded reciprocal;
//   photons, lambda >= 10: Hoermann's (1993) PTRS transformed rejection (valid from
//     lambda = 10, O(1) expected draws) on the pairs (word 2, word 3) of blocks
//     0, 1, 2, ..., with lgammaf.
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

__device__ inline float u01f(uint32_t x) { return ((float)(x >> 8) + 0.5f) * 5.9604644775390625e-8f; }

__device__ inline u32x4 noise_block(uint64_t seed, uint32_t pixel, uint64_t frame, uint32_t blk) {
  return philox4x32_10(pixel, (uint32_t)frame, (uint32_t)(frame >> 32), blk, (uint32_t)seed,
                       (uint32_t)(seed >> 32));
}

// Inversion by sequential search (lambda < 10) on block 0 word 2. The float32 CDF
// stops growing once the terms fall below its resolution near 1; a uniform above that
// last value takes the count at which it stopped (the tail beyond is below float32
// resolution), instead of running the search to its bound.
__device__ inline float poisson_small(float lam, const u32x4& w0) {
  const float u = u01f(w0.v[2]);
  float p = expf(-lam);
  float F = p;
  int k = 0;
  while (u > F && k < 256) {
    ++k;
    p = __fmul_rn(p, __fmul_rn(lam, __frcp_rn((float)k)));
    const float Fn = __fadd_rn(F, p);
    if (Fn == F) break;
    F = Fn;
  }
  return (float)k;
}

// Constants of the PTRS rejection for one lambda >= 10.
struct Ptrs {
  float lam, loglam, b, a, invalpha, vr;
  __device__ explicit Ptrs(float l) : lam(l) {
    const float slam = sqrtf(lam);
    loglam = logf(lam);
    b = __fadd_rn(0.931f, __fmul_rn(2.53f, slam));
    a = __fadd_rn(-0.059f, __fmul_rn(0.02483f, b));
    invalpha = __fadd_rn(1.1239f, __fdiv_rn(1.1328f, __fsub_rn(b, 3.4f)));
    vr = __fsub_rn(0.9277f, __fdiv_rn(3.6224f, __fsub_rn(b, 2.0f)));
  }
  // One candidate from the words (2, 3) of a counter block: true with *k if accepted.
  __device__ bool attempt(const u32x4& w, float* k_out) const {
    const float U = __fsub_rn(u01f(w.v[2]), 0.5f);
    const float V = u01f(w.v[3]);
    const float us = __fsub_rn(0.5f, fabsf(U));
    const float k = floorf(__fadd_rn(__fadd_rn(__fmul_rn(__fadd_rn(__fdiv_rn(__fmul_rn(2.0f, a), us), b), U), lam), 0.43f));
    *k_out = k;
    if (us >= 0.07f && V <= vr) return true;
    if (k < 0.f || (us < 0.013f && V > us)) return false;
    const float lhs = __fsub_rn(__fadd_rn(logf(V), logf(invalpha)),
                                logf(__fadd_rn(__fdiv_rn(a, __fmul_rn(us, us)), b)));
    const float rhs = __fsub_rn(__fadd_rn(-lam, __fmul_rn(k, loglam)), lgammaf(__fadd_rn(k, 1.0f)));
    return lhs <= rhs;
  }
};

constexpr uint32_t PTRS_MAX_BLOCKS = 64;  // candidates before the rounded-mean fallback

__device__ inline float poisson_draw(float lam, uint64_t seed, uint32_t pixel, uint64_t frame) {
  if (!(lam > 0.f)) return 0.f;
  u32x4 w = noise_block(seed, pixel, frame, 0);
  if (lam < 10.f) return poisson_small(lam, w);
  const Ptrs P(lam);
  for (uint32_t blk = 0; blk < PTRS_MAX_BLOCKS; ++blk) {
    if (blk > 0) w = noise_block(seed, pixel, frame, blk);
    float k;
    if (P.attempt(w, &k)) return k;
  }
  return floorf(lam + 0.5f);
}

// The same draw by a group of g adjacent lanes (g = 1, 2, 4 or 8, groups aligned in
// the warp; lane `sub` of its group): in round r the lanes try the candidates of
// blocks r g + sub side by side and the group keeps the first accepted one in block
// order, which is the candidate the sequential search accepts, so the result equals
// poisson_draw's. Every lane of the warp must call it (warp-wide votes); `active`
// false for lanes without a pixel. Returned to every lane of the group.
__device__ inline float poisson_draw_group(float lam, uint64_t seed, uint32_t pixel, uint64_t frame, int sub,
                                           int g, bool active) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, gbase = lane - sub;
  const unsigned gmask = (g == 32 ? FULL : ((1u << g) - 1u)) << gbase;
  bool done = !active || !(lam > 0.f);
  float result = 0.f;
  if (!done && lam < 10.f) {
    if (sub == 0) result = poisson_small(lam, noise_block(seed, pixel, frame, 0));
    done = true;
  }
  // the small-lambda result lives in the group's first lane
  const float small = __shfl_sync(FULL, result, gbase);
  if (active && lam > 0.f && lam < 10.f) result = small;
  const Ptrs P(done ? 10.f : lam);
  for (uint32_t r = 0; r < PTRS_MAX_BLOCKS; r += (uint32_t)g) {
    if (!__any_sync(FULL, !done)) break;
    const uint32_t blk = r + (uint32_t)sub;
    bool acc = false;
    float k = 0.f;
    if (!done && blk < PTRS_MAX_BLOCKS) acc = P.attempt(noise_block(seed, pixel, frame, blk), &k);
    const unsigned m = __ballot_sync(FULL, acc) & gmask;
    const int first = m ? __ffs(m) - 1 : lane;
    const float kf = __shfl_sync(FULL, k, first);
    if (!done && m) {
      result = kf;
      done = true;
    }
  }
  if (!done) result = floorf(lam + 0.5f);
  return result;
}

__device__ inline float gaussian_draw(uint64_t seed, uint32_t pixel, uint64_t frame) {
  u32x4 w = noise_block(seed, pixel, frame, 0);
  return __fmul_rn(sqrtf(__fmul_rn(-2.0f, logf(u01f(w.v[0])))), cospif(__fmul_rn(2.0f, u01f(w.v[1]))));
}

// Noisy value of one detector pixel: Poisson(v * scale) + ron * N(0, 1) in
// photo-electrons; scale <= 0 leaves v unchanged.
__device__ inline float noisy_pixel(float v, float scale, float ron, uint64_t seed, uint32_t pixel,
                                    uint64_t frame) {
  if (!(scale > 0.f)) return v;
  float e = poisson_draw(__fmul_rn(v, scale), seed, pixel, frame);
  if (ron > 0.f) e = __fadd_rn(e, __fmul_rn(ron, gaussian_draw(seed, pixel, frame)));
  return e;
}

// noisy_pixel by a group of g adjacent lanes (poisson_draw_group's contract; scale
// and ron uniform across the warp). Same value as noisy_pixel, in every lane.
__device__ inline float noisy_pixel_group(float v, float scale, float ron, uint64_t seed, uint32_t pixel,
                                          uint64_t frame, int sub, int g, bool active) {
  if (!(scale > 0.f)) return v;
  float e = poisson_draw_group(__fmul_rn(v, scale), seed, pixel, frame, sub, g, active);
  if (ron > 0.f && active) e = __fadd_rn(e, __fmul_rn(ron, gaussian_draw(seed, pixel, frame)));
  return e;
}

}  // namespace pas
