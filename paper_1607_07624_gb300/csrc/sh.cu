// Shack-Hartmann wavefront sensor (the framework's second sensor type; Sec. GPU
// acceleration, "Pyramid and Shack Hartmann propagation (from wavefront to detector
// plane)"). The paper gives no parameters; the model is the textbook one:
//
//   lenslet (r, c) of an n_sub x n_sub array covers the b x b pupil pixels
//   [r b, (r+1) b) x [c b, (c+1) b); its field E = A exp(2 pi i opd / lambda) is
//   zero-padded to M x M (M = ovs b) and its spot is
//     I(k, l) = |sum_ij E(i, j) exp(-2 pi i ((k - M/2) i + (l - M/2) j) / M)|^2 / M^2,
//   zero frequency at pixel (M/2, M/2), total = the lenslet's lit pupil pixels;
//   spots tile the detector frame (lenslet (r, c) at rows r M.., columns c M..);
//   slopes = centre of gravity about (M/2, M/2) in pixels, [x; y] over the valid
//   lenslets, minus the reference slopes.
//
// With b and M of a few to a few tens of pixels the padded 2-D DFT of a lenslet is
// two small dense products with the M x b matrix W(k, i) = exp(-2 pi i (k - M/2) i / M):
// T = E W^T (b x M), F = W T (M x M). One CTA per lenslet, one thread per spot pixel,
// E, W and T in shared memory; the centroid moments are reduced in a fixed order
// (float within a warp, double across warps).
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"
#include "noise.cuh"
#include "pdl.cuh"
#include "phasor.cuh"
#include "sh.cuh"
#include "wfe.cuh"

namespace pas {

struct ShArgs {
  const float* opd;      // [Np][Np] nm
  const float2* W;       // [M][b]
  const int* slope_of;   // [n_sub^2]: index in the valid list, or -1
  const float* ref;      // [2 nv] reference slopes or null
  float* frame;          // [(n_sub M)^2] or null
  float* slopes;         // [2 nv] or null
  int Np, n_sub, b, M, nv, T_obs;
  float inv_hi, inv_lo, inv_M2;
  float scale, ron;            // detector noise: photons per intensity unit (<= 0: none), read noise
  unsigned long long seed;
  const long long* frame_ctr;  // the frame's noise counter (the loop's step in a loop)
  LoopExtra wfe;               // in a loop: the step's residual WFE, closed by CTA 0
};

__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}

// NOISE: the detector-noise variant (its sampler needs more registers).
template <bool NOISE>
__global__ void __launch_bounds__(1024) sh_kernel(ShArgs a) {
  extern __shared__ float2 sh_smem[];
  __shared__ float3 red[32];
  __shared__ double dred[32];
  const int b = a.b, M = a.M;
  float2* W_s = sh_smem;          // [M][b]
  float2* E_s = W_s + M * b;      // [b][b]
  float2* T_s = E_s + b * b;      // [b][M]
  const int lens = blockIdx.x, r = lens / a.n_sub, c = lens - r * a.n_sub;
  const int tid = threadIdx.x;
  pdl_trigger();
  for (int t = tid; t < M * b; t += blockDim.x) W_s[t] = a.W[t];
  pdl_wait();  // the OPD (and the WFE partials) may come from the preceding kernel
  if (blockIdx.x == 0 && a.wfe.wfe_part) wfe_finalize(a.wfe, dred);
  const int Np = a.Np;
  for (int t = tid; t < b * b; t += blockDim.x) {
    const int i = t / b, j = t - i * b;
    const int gi = r * b + i, gj = c * b + j;
    const int ai = 2 * gi - Np + 1, aj = 2 * gj - Np + 1;
    const int d2 = ai * ai + aj * aj;
    float2 e = make_float2(0.f, 0.f);
    if (d2 <= Np * Np && d2 >= a.T_obs) e = opd_phasor(__ldg(a.opd + (size_t)gi * Np + gj), a.inv_hi, a.inv_lo);
    E_s[t] = e;
  }
  __syncthreads();
  for (int t = tid; t < b * M; t += blockDim.x) {  // T[i][l] = sum_j E[i][j] W[l][j]
    const int i = t / M, l = t - i * M;
    float2 acc = make_float2(0.f, 0.f);
    for (int j = 0; j < b; ++j) acc = cfma(E_s[i * b + j], W_s[l * b + j], acc);
    T_s[t] = acc;
  }
  __syncthreads();
  // one thread per spot pixel; blockDim is M * M rounded up to whole warps (the
  // extra threads hold no pixel and add zeros to the sums)
  const int k = tid / M, l = tid - k * M;
  const bool pix = tid < M * M;
  // a detector integrating n_int steps (loops): the spots add up in wfe.acc and are
  // read out as the window's mean at the steps t with (t + 1) mod n_int = 0 (frame_ctr
  // holds t); in between there is no frame and the slopes keep their value
  const bool hold = a.wfe.n_int > 1 && (*a.frame_ctr + 1) % a.wfe.n_int != 0;  // uniform
  float I = 0.f;
  if (pix) {
    float2 f = make_float2(0.f, 0.f);
    for (int i = 0; i < b; ++i) f = cfma(W_s[k * b + i], T_s[i * M + l], f);
    I = __fmul_rn(__fmaf_rn(f.x, f.x, __fmul_rn(f.y, f.y)), a.inv_M2);
    const size_t px = ((size_t)r * M + k) * ((size_t)a.n_sub * M) + (size_t)c * M + l;
    if (a.wfe.n_int > 1) {
      const float acc = __fadd_rn(__ldcg(a.wfe.acc + px), I);
      a.wfe.acc[px] = hold ? acc : 0.f;
      I = __fdiv_rn(acc, (float)a.wfe.n_int);
    }
    if (!hold) {
      if constexpr (NOISE) I = noisy_pixel(I, a.scale, a.ron, a.seed, (uint32_t)px, (uint64_t)*a.frame_ctr);
      if (a.frame) a.frame[px] = I;
    }
  }
  const int s = a.slope_of[lens];
  if (s >= 0 && a.slopes && !hold) {  // uniform across the CTA
    // the three moments: float within a warp (fixed shuffle tree), the warps' partials
    // added in double in warp order by thread 0
    const float half = 0.5f * (float)M;
    float m0 = I, m1 = I * ((float)k - half), m2 = I * ((float)l - half);
    for (int o = 16; o > 0; o >>= 1) {
      m0 += __shfl_down_sync(0xffffffffu, m0, o);
      m1 += __shfl_down_sync(0xffffffffu, m1, o);
      m2 += __shfl_down_sync(0xffffffffu, m2, o);
    }
    if ((tid & 31) == 0) red[tid >> 5] = make_float3(m0, m1, m2);
    __syncthreads();
    if (tid == 0) {
      double s0 = 0.0, s1 = 0.0, s2 = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        s0 += red[w].x;
        s1 += red[w].y;
        s2 += red[w].z;
      }
      float cx = s0 > 0.0 ? (float)(s1 / s0) : 0.f, cy = s0 > 0.0 ? (float)(s2 / s0) : 0.f;
      if (a.ref) {
        cx -= a.ref[s];
        cy -= a.ref[a.nv + s];
      }
      a.slopes[s] = cx;
      a.slopes[a.nv + s] = cy;
    }
  }
}

}  // namespace pas

struct pas_sh_s {
  pas_ctx_t ctx = nullptr;
  int Np = 0, n_sub = 0, b = 0, M = 0, nv = 0, T_obs = 0;
  float inv_hi = 0.f, inv_lo = 0.f, inv_M2 = 0.f;
  bool has_ref = false;
  int n_pupil = 0;
  float photon_scale = 0.f, ron = 0.f;
  unsigned long long seed = 0;
  long long* d_frame_ctr = nullptr;  // noise counter of standalone measurements
  float2* d_W = nullptr;
  int* d_slope_of = nullptr;
  int32_t* d_valid = nullptr;
  float* d_ref = nullptr;
};

namespace pas {

__global__ void sh_count_frame(long long* ctr) { *ctr += 1; }

pas_status sh_launch(pas_sh_t S, const float* d_opd, float* d_frame, float* d_slopes, cudaStream_t st,
                     const LoopExtra* extra, bool pdl) {
  ShArgs a;
  a.opd = d_opd;
  a.W = S->d_W;
  a.slope_of = S->d_slope_of;
  a.ref = S->has_ref ? S->d_ref : nullptr;
  a.frame = d_frame;
  a.slopes = d_slopes;
  a.Np = S->Np;
  a.n_sub = S->n_sub;
  a.b = S->b;
  a.M = S->M;
  a.nv = S->nv;
  a.T_obs = S->T_obs;
  a.inv_hi = S->inv_hi;
  a.inv_lo = S->inv_lo;
  a.inv_M2 = S->inv_M2;
  a.scale = S->photon_scale;
  a.ron = S->ron;
  a.seed = S->seed;
  a.frame_ctr = extra && extra->frame_ctr ? extra->frame_ctr : S->d_frame_ctr;
  a.wfe = extra ? *extra : LoopExtra();
  const size_t smem = sizeof(float2) * ((size_t)2 * S->M * S->b + (size_t)S->b * S->b);
  const int threads = (S->M * S->M + 31) / 32 * 32;
  cudaError_t e = a.scale > 0.f ? launch_k(sh_kernel<true>, dim3(S->n_sub * S->n_sub), dim3(threads), smem, st, pdl, a)
                                 : launch_k(sh_kernel<false>, dim3(S->n_sub * S->n_sub), dim3(threads), smem, st, pdl, a);
  if (e != cudaSuccess) return set_error(S->ctx, PAS_ECUDA, "Shack-Hartmann launch: %s", cudaGetErrorString(e));
  return PAS_OK;
}

pas_status sh_measure_noiseless(pas_sh_t S, const float* d_opd, float* d_frame, float* d_slopes, cudaStream_t st) {
  const float scale = S->photon_scale;
  S->photon_scale = 0.f;
  const pas_status r = sh_launch(S, d_opd, d_frame, d_slopes, st, nullptr, false);
  S->photon_scale = scale;
  return r;
}

int sh_n_slopes(pas_sh_t S) { return 2 * S->nv; }
int sh_frame_side(pas_sh_t S) { return S->n_sub * S->M; }
int sh_np(pas_sh_t S) { return S->Np; }

}  // namespace pas

extern "C" {

void pas_sh_destroy(pas_sh_t S) {
  if (!S) return;
  pas::dev_free(S->d_W);
  pas::dev_free(S->d_slope_of);
  pas::dev_free(S->d_valid);
  pas::dev_free(S->d_ref);
  pas::dev_free(S->d_frame_ctr);
  delete S;
}

pas_status pas_sh_create(pas_ctx_t ctx, int32_t Np, int32_t n_sub, int32_t ovs, double wavelength_nm, double obs,
                         const int32_t* h_valid, int32_t n_valid, pas_sh_t* out) {
  if (!ctx || !out) return pas::set_global_error(PAS_EINVAL, "pas_sh_create: NULL argument");
  *out = nullptr;
  PAS_CHECK_ARG(ctx, Np > 0 && n_sub > 0 && Np % n_sub == 0 && ovs >= 1 && wavelength_nm > 0 && obs >= 0 && obs < 1,
                "pas_sh_create: need n_sub dividing Np, ovs >= 1, wavelength > 0, 0 <= obs < 1");
  const int b = Np / n_sub, M = ovs * b;
  PAS_CHECK_ARG(ctx, M % 2 == 0 && M >= 2 && M <= 32, "pas_sh_create: spot side ovs*Np/n_sub must be even, <= 32");
  std::vector<int32_t> valid;
  if (h_valid) {
    PAS_CHECK_ARG(ctx, n_valid > 0, "pas_sh_create: n_valid must be > 0");
    valid.assign(h_valid, h_valid + n_valid);
    for (int j = 0; j < n_valid; ++j)
      PAS_CHECK_ARG(ctx, valid[j] >= 0 && valid[j] < n_sub * n_sub && (j == 0 || valid[j] > valid[j - 1]),
                    "pas_sh_create: valid indices must be ascending in [0, n_sub^2)");
  } else {
    int32_t nv = 0;
    pas_status st = pas_valid_subaps(Np, obs, n_sub, nullptr, 0, &nv);
    if (st != PAS_OK) return pas::set_error(ctx, st, "pas_sh_create: valid lenslets");
    valid.resize(nv);
    pas_valid_subaps(Np, obs, n_sub, valid.data(), nv, &nv);
  }
  PAS_CHECK_ARG(ctx, !valid.empty(), "pas_sh_create: no valid lenslet");
  std::vector<int> slope_of((size_t)n_sub * n_sub, -1);
  for (size_t j = 0; j < valid.size(); ++j) slope_of[valid[j]] = (int)j;
  std::vector<float2> W((size_t)M * b);
  for (int k = 0; k < M; ++k)
    for (int i = 0; i < b; ++i) {
      const long long e = ((long long)(k - M / 2) * i) % M;
      const double a = -2.0 * M_PI * (double)e / (double)M;
      W[(size_t)k * b + i] = make_float2((float)std::cos(a), (float)std::sin(a));
    }

  pas_sh_t S = new pas_sh_s();
  S->ctx = ctx;
  S->Np = Np;
  S->n_sub = n_sub;
  S->b = b;
  S->M = M;
  S->nv = (int)valid.size();
  S->T_obs = (int)pas::obstruction_threshold(Np, obs);
  const double inv = 1.0 / wavelength_nm;
  S->inv_hi = (float)inv;
  S->inv_lo = (float)(inv - (double)S->inv_hi);
  S->inv_M2 = (float)(1.0 / ((double)M * M));
  pas_pupil_mask(Np, obs, nullptr, &S->n_pupil);
  pas_status st = PAS_OK;
  auto A = [&](void** p, size_t bytes) {
    if (st == PAS_OK) st = pas::dev_alloc(ctx, p, bytes);
  };
  A((void**)&S->d_W, sizeof(float2) * W.size());
  A((void**)&S->d_slope_of, sizeof(int) * slope_of.size());
  A((void**)&S->d_valid, sizeof(int32_t) * valid.size());
  A((void**)&S->d_ref, sizeof(float) * 2 * valid.size());
  A((void**)&S->d_frame_ctr, sizeof(long long));
  if (st != PAS_OK) {
    pas_sh_destroy(S);
    return st;
  }
  cudaError_t e = cudaMemcpy(S->d_W, W.data(), sizeof(float2) * W.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(S->d_slope_of, slope_of.data(), sizeof(int) * slope_of.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(S->d_valid, valid.data(), sizeof(int32_t) * valid.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(S->d_frame_ctr, 0, sizeof(long long));
  if (e != cudaSuccess) {
    pas_sh_destroy(S);
    return pas::set_error(ctx, PAS_ECUDA, "pas_sh_create: %s", cudaGetErrorString(e));
  }
  *out = S;
  return PAS_OK;
}

int32_t pas_sh_n_valid(pas_sh_t S) { return S ? S->nv : -1; }
int32_t pas_sh_frame_side(pas_sh_t S) { return S ? S->n_sub * S->M : -1; }

pas_status pas_sh_get_valid(pas_sh_t S, int32_t* h_valid, int32_t cap) {
  if (!S || !h_valid) return pas::set_global_error(PAS_EINVAL, "pas_sh_get_valid: NULL argument");
  PAS_CHECK_ARG(S->ctx, cap >= S->nv, "pas_sh_get_valid: cap too small");
  PAS_CUDA_TRY(S->ctx, cudaMemcpy(h_valid, S->d_valid, sizeof(int32_t) * S->nv, cudaMemcpyDeviceToHost));
  return PAS_OK;
}

pas_status pas_sh_set_reference(pas_sh_t S, const float* d_ref) {
  if (!S) return pas::set_global_error(PAS_EINVAL, "pas_sh_set_reference: NULL sensor");
  if (!d_ref) {
    S->has_ref = false;
    return PAS_OK;
  }
  PAS_CUDA_TRY(S->ctx, cudaMemcpyAsync(S->d_ref, d_ref, sizeof(float) * 2 * S->nv, cudaMemcpyDeviceToDevice,
                                       S->ctx->stream));
  S->has_ref = true;
  return PAS_OK;
}

pas_status pas_sh_measure(pas_sh_t S, const float* d_opd, float* d_frame, float* d_slopes) {
  if (!S || !d_opd) return pas::set_global_error(PAS_EINVAL, "pas_sh_measure: NULL argument");
  pas_status st = pas::sh_launch(S, d_opd, d_frame, d_slopes, S->ctx->stream, nullptr, false);
  if (st != PAS_OK || !(S->photon_scale > 0.f)) return st;
  pas::sh_count_frame<<<1, 1, 0, S->ctx->stream>>>(S->d_frame_ctr);  // the next frame's counter
  return pas::check_launch(S->ctx, "Shack-Hartmann frame counter");
}

pas_status pas_sh_set_noise(pas_sh_t S, double photons_per_frame, double read_noise_e, uint64_t seed,
                            int64_t frame_index) {
  if (!S) return pas::set_global_error(PAS_EINVAL, "pas_sh_set_noise: NULL sensor");
  PAS_CHECK_ARG(S->ctx, read_noise_e >= 0.0 && frame_index >= 0, "pas_sh_set_noise: bad read noise or frame index");
  S->photon_scale = photons_per_frame > 0.0 ? (float)(photons_per_frame / (double)S->n_pupil) : 0.f;
  S->ron = (float)read_noise_e;
  S->seed = seed;
  long long f = frame_index;
  PAS_CUDA_TRY(S->ctx, cudaMemcpyAsync(S->d_frame_ctr, &f, sizeof(f), cudaMemcpyHostToDevice, S->ctx->stream));
  PAS_CUDA_TRY(S->ctx, cudaStreamSynchronize(S->ctx->stream));
  return PAS_OK;
}

}  // extern "C"
