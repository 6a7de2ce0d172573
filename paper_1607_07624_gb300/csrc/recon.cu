// Modal reconstructor dmodes = R * slopes (Table 1 modalrec.recmat_tag) and the
// integrator control c_t = c_{t-1} + g * dmodes (Table 1 control, type 'INT'),
// fused into one kernel for the loop.
//
// The matrix-vector product reads every element of R once per step: it is bound
// by memory bandwidth, so it runs on CUDA cores with 16-byte loads: four warps per
// mode row and the slope vector staged in shared memory for short vectors, two warps
// per row and slopes read through L1 for long ones (recon_stream_kernel). PAS_BF16 stores R as
// bfloat16 scaled per row (row max |R| = 1) with float32 accumulation.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "pdl.cuh"
#include "recon.cuh"

namespace pas {

__device__ inline float dot4(float4 a, float4 b, float acc) {
  acc = fmaf(a.x, b.x, acc);
  acc = fmaf(a.y, b.y, acc);
  acc = fmaf(a.z, b.z, acc);
  return fmaf(a.w, b.w, acc);
}

// CTA: 256 threads = RECON_ROWS rows x RECON_SPLIT warps per row; the warps of a
// row take interleaved 16-byte chunks and meet in shared memory. With the
// integrator active, the last CTA to finish advances the step counter.
constexpr int RECON_SPLIT = 4;
constexpr int RECON_ROWS = 8 / RECON_SPLIT;

template <bool BF16>
__global__ void __launch_bounds__(256) recon_kernel(ReconArgs a) {
  using Chunk = typename std::conditional<BF16, uint4, float4>::type;  // one 16-byte load
  constexpr int PRE = 4;                                               // chunks loaded before the wait
  constexpr int STEP = RECON_SPLIT * 32;
  extern __shared__ float4 s4[];  // [n_s_pad / 4]
  __shared__ float part[8];
  __shared__ bool is_last;
  pdl_trigger();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row_local = warp / RECON_SPLIT, part_idx = warp % RECON_SPLIT;
  const int m = blockIdx.x * RECON_ROWS + row_local;
  const int c0 = part_idx * 32 + lane;
  const int nc = a.n_s_pad / (BF16 ? 8 : 4);
  const Chunk* row = nullptr;
  if (m < a.n_m) {
    if constexpr (BF16) row = reinterpret_cast<const uint4*>(a.Rb + (size_t)m * a.n_s_pad);
    else row = reinterpret_cast<const float4*>(a.R + (size_t)m * a.n_s_pad);
  }
  // Before the wait for the slopes: everything else this CTA reads is final. The
  // reconstructor is constant (its first PRE chunks per thread go to registers,
  // the rest of the CTA's rows towards L2); the step counter and the previous
  // command were written by the previous step's reconstructor, which has completed.
  Chunk pre[PRE];
#pragma unroll
  for (int u = 0; u < PRE; ++u) {
    const int c = c0 + u * STEP;
    pre[u] = (row && c < nc) ? __ldg(row + c) : Chunk{};
  }
  {
    const int m0 = blockIdx.x * RECON_ROWS;
    const size_t row_bytes = (size_t)a.n_s_pad * (BF16 ? 2 : 4);
    const char* base = BF16 ? reinterpret_cast<const char*>(a.Rb) : reinterpret_cast<const char*>(a.R);
    const int nrow = min(RECON_ROWS, a.n_m - m0);
    const size_t skip = (size_t)PRE * STEP * 16;  // bytes of a row already in registers
    if (row_bytes > skip) {
      const int lines = (int)((row_bytes - skip + 127) / 128);
      for (int t = threadIdx.x; t < lines * nrow; t += blockDim.x) {
        const int r = t / lines, l = t - r * lines;
        prefetch_l2(base + row_bytes * (m0 + r) + skip + (size_t)l * 128);
      }
    }
  }
  const bool writer = part_idx == 0 && lane == 0 && m < a.n_m;
  long long t_step = 0;
  float prev = 0.f;
  bool hold = false;  // between the read-outs of a detector integrating several steps
  if (writer && a.ring) {
    t_step = *a.step;
    prev = a.ring[(size_t)((t_step - 1 + a.delay) % a.delay) * a.n_m + m];
    hold = a.n_int > 1 && (t_step + 1) % a.n_int != 0;
  }
  pdl_wait();
  float* s_s = reinterpret_cast<float*>(s4);
  for (int t = threadIdx.x; t < a.n_s_pad; t += blockDim.x) s_s[t] = t < a.n_s ? a.s[t] : 0.f;
  __syncthreads();
  float acc = 0.f;
  if (row) {
    auto fma_chunk = [&](const Chunk& u, int c) {
      if constexpr (BF16) {
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
        const float2 f0 = __bfloat1622float2(h[0]), f1 = __bfloat1622float2(h[1]);
        const float2 f2 = __bfloat1622float2(h[2]), f3 = __bfloat1622float2(h[3]);
        acc = dot4(make_float4(f0.x, f0.y, f1.x, f1.y), s4[2 * c], acc);
        acc = dot4(make_float4(f2.x, f2.y, f3.x, f3.y), s4[2 * c + 1], acc);
      } else {
        acc = dot4(u, s4[c], acc);
      }
    };
#pragma unroll
    for (int u = 0; u < PRE; ++u) {
      const int c = c0 + u * STEP;
      if (c < nc) fma_chunk(pre[u], c);
    }
#pragma unroll 4
    for (int c = c0 + PRE * STEP; c < nc; c += STEP) fma_chunk(__ldg(row + c), c);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) part[warp] = acc;
  __syncthreads();
  if (writer) {
    float tot = 0.f;
#pragma unroll
    for (int q = 0; q < RECON_SPLIT; ++q) tot += part[warp + q];
    const float dm = hold ? 0.f : (BF16 ? tot * a.scale[m] : tot);
    if (a.dmodes) a.dmodes[m] = dm;
    if (a.ring) {
      const float c = hold ? prev : fmaf(a.gain ? a.gain[m] : 1.0f, dm, prev);
      a.ring[(size_t)(t_step % a.delay) * a.n_m + m] = c;
      if (a.cmd_last) a.cmd_last[m] = c;
    }
  }
  if (a.step_inc) {
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      is_last = atomicAdd(a.done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (is_last && threadIdx.x == 0) {
      *a.step_inc += 1;
      *a.done = 0u;
    }
  }
}

// The same product for long slope vectors (n_s >= RECON_STREAM_MIN_NS): staging the
// whole vector in shared memory per CTA would move as many bytes from L2 as R itself
// and cap the CTAs per SM, so here the slopes are read through L1 (every CTA of an SM
// shares one copy) and each warp keeps RECON_STREAM_U 16-byte chunks of R in flight.
// CTA: 256 threads = 4 rows x RECON_STREAM_SPLIT (2) warps; the first chunks of R
// are loaded before the programmatic wait (R is constant). Slopes must be 16-byte
// aligned (checked by the launcher).
constexpr int RECON_STREAM_SPLIT = 2;
constexpr int RECON_STREAM_ROWS = 8 / RECON_STREAM_SPLIT;
constexpr int RECON_STREAM_U = 8;
constexpr int RECON_STREAM_MIN_NS = 4096;

template <bool BF16>
__device__ __forceinline__ void slope_chunk(const float* s, int n_s, int c, float4* lo, float4* hi) {
  constexpr int W = BF16 ? 8 : 4;  // slopes per 16-byte chunk of R
  const int j0 = c * W;
  if (j0 + W <= n_s) {
    *lo = __ldg(reinterpret_cast<const float4*>(s + j0));
    if constexpr (BF16) *hi = __ldg(reinterpret_cast<const float4*>(s + j0 + 4));
  } else {
    float v[8];
#pragma unroll
    for (int q = 0; q < W; ++q) v[q] = j0 + q < n_s ? __ldg(s + j0 + q) : 0.f;
    *lo = make_float4(v[0], v[1], v[2], v[3]);
    if constexpr (BF16) *hi = make_float4(v[4], v[5], v[6], v[7]);
  }
}

template <bool BF16>
__global__ void __launch_bounds__(256) recon_stream_kernel(ReconArgs a) {
  using Chunk = typename std::conditional<BF16, uint4, float4>::type;
  constexpr int STEP = RECON_STREAM_SPLIT * 32;
  constexpr int U = RECON_STREAM_U;
  __shared__ float part[8];
  __shared__ bool is_last;
  pdl_trigger();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row_local = warp / RECON_STREAM_SPLIT, part_idx = warp % RECON_STREAM_SPLIT;
  const int m = blockIdx.x * RECON_STREAM_ROWS + row_local;
  const int c0 = part_idx * 32 + lane;
  const int nc = a.n_s_pad / (BF16 ? 8 : 4);
  const Chunk* row = nullptr;
  if (m < a.n_m) {
    if constexpr (BF16) row = reinterpret_cast<const uint4*>(a.Rb + (size_t)m * a.n_s_pad);
    else row = reinterpret_cast<const float4*>(a.R + (size_t)m * a.n_s_pad);
  }
  Chunk buf[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int c = c0 + u * STEP;
    buf[u] = (row && c < nc) ? __ldcs(row + c) : Chunk{};
  }
  const bool writer = part_idx == 0 && lane == 0 && m < a.n_m;
  long long t_step = 0;
  float prev = 0.f;
  bool hold = false;
  if (writer && a.ring) {
    t_step = *a.step;
    prev = a.ring[(size_t)((t_step - 1 + a.delay) % a.delay) * a.n_m + m];
    hold = a.n_int > 1 && (t_step + 1) % a.n_int != 0;
  }
  pdl_wait();
  float acc = 0.f;
  if (row) {
    auto fma_chunk = [&](const Chunk& u, int c) {
      float4 lo, hi;
      slope_chunk<BF16>(a.s, a.n_s, c, &lo, &hi);
      if constexpr (BF16) {
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
        const float2 f0 = __bfloat1622float2(h[0]), f1 = __bfloat1622float2(h[1]);
        const float2 f2 = __bfloat1622float2(h[2]), f3 = __bfloat1622float2(h[3]);
        acc = dot4(make_float4(f0.x, f0.y, f1.x, f1.y), lo, acc);
        acc = dot4(make_float4(f2.x, f2.y, f3.x, f3.y), hi, acc);
      } else {
        acc = dot4(u, lo, acc);
      }
    };
    for (int cb = c0; cb < nc; cb += U * STEP) {
      // the batch in buf is being consumed; the next one is requested first
      Chunk nxt[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int c = cb + (U + u) * STEP;
        nxt[u] = c < nc ? __ldcs(row + c) : Chunk{};
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int c = cb + u * STEP;
        if (c < nc) fma_chunk(buf[u], c);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) buf[u] = nxt[u];
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) part[warp] = acc;
  __syncthreads();
  if (writer) {
    float tot = 0.f;
#pragma unroll
    for (int q = 0; q < RECON_STREAM_SPLIT; ++q) tot += part[warp + q];
    const float dm = hold ? 0.f : (BF16 ? tot * a.scale[m] : tot);
    if (a.dmodes) a.dmodes[m] = dm;
    if (a.ring) {
      const float c = hold ? prev : fmaf(a.gain ? a.gain[m] : 1.0f, dm, prev);
      a.ring[(size_t)(t_step % a.delay) * a.n_m + m] = c;
      if (a.cmd_last) a.cmd_last[m] = c;
    }
  }
  if (a.step_inc) {
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      is_last = atomicAdd(a.done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (is_last && threadIdx.x == 0) {
      *a.step_inc += 1;
      *a.done = 0u;
    }
  }
}

static uint16_t f32_to_bf16_rne(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  return (uint16_t)(u >> 16);
}

pas_status recon_launch(pas_recon_t r, ReconArgs a, cudaStream_t st, bool pdl) {
  a.R = r->d_R;
  a.Rb = r->d_Rb;
  a.scale = r->d_scale;
  a.n_m = r->n_modes;
  a.n_s = r->n_slopes;
  a.n_s_pad = r->n_s_pad;
  a.done = r->d_done;
  cudaError_t e;
  if (r->n_slopes >= RECON_STREAM_MIN_NS && (reinterpret_cast<uintptr_t>(a.s) & 15u) == 0) {
    const int grid = (r->n_modes + RECON_STREAM_ROWS - 1) / RECON_STREAM_ROWS;
    e = r->prec == PAS_BF16 ? launch_k(recon_stream_kernel<true>, dim3(grid), dim3(256), 0, st, pdl, a)
                            : launch_k(recon_stream_kernel<false>, dim3(grid), dim3(256), 0, st, pdl, a);
  } else {
    const size_t smem = sizeof(float) * (size_t)r->n_s_pad;
    const int grid = (r->n_modes + RECON_ROWS - 1) / RECON_ROWS;
    e = r->prec == PAS_BF16 ? launch_k(recon_kernel<true>, dim3(grid), dim3(256), smem, st, pdl, a)
                            : launch_k(recon_kernel<false>, dim3(grid), dim3(256), smem, st, pdl, a);
  }
  if (e != cudaSuccess) return set_error(r->ctx, PAS_ECUDA, "reconstructor launch: %s", cudaGetErrorString(e));
  return PAS_OK;
}

}  // namespace pas

extern "C" {

void pas_recon_destroy(pas_recon_t r) {
  if (!r) return;
  pas::dev_free(r->d_R);
  pas::dev_free(r->d_Rb);
  pas::dev_free(r->d_scale);
  pas::dev_free(r->d_done);
  delete r;
}

pas_status pas_recon_create(pas_ctx_t ctx, const float* h_R, int32_t n_modes, int32_t n_slopes,
                            pas_precision prec, pas_recon_t* out) {
  if (!ctx || !h_R || !out) return pas::set_global_error(PAS_EINVAL, "pas_recon_create: NULL argument");
  *out = nullptr;
  PAS_CHECK_ARG(ctx, n_modes >= 1 && n_slopes >= 1, "pas_recon_create: bad sizes");
  PAS_CHECK_ARG(ctx, prec == PAS_FP32 || prec == PAS_BF16, "pas_recon_create: bad precision");
  pas_recon_t r = new pas_recon_s();
  r->ctx = ctx;
  r->n_modes = n_modes;
  r->n_slopes = n_slopes;
  r->n_s_pad = ((n_slopes + 7) / 8) * 8;
  r->prec = prec;
  const size_t smem = sizeof(float) * (size_t)r->n_s_pad;
  pas_status st = PAS_OK;
  cudaError_t e = cudaSuccess;
  if (prec == PAS_FP32) {
    std::vector<float> R((size_t)n_modes * r->n_s_pad, 0.f);
    for (int m = 0; m < n_modes; ++m)
      std::memcpy(&R[(size_t)m * r->n_s_pad], h_R + (size_t)m * n_slopes, sizeof(float) * n_slopes);
    st = pas::dev_alloc(ctx, (void**)&r->d_R, sizeof(float) * R.size());
    if (st == PAS_OK) e = cudaMemcpy(r->d_R, R.data(), sizeof(float) * R.size(), cudaMemcpyHostToDevice);
    if (st == PAS_OK && e == cudaSuccess)
      e = pas::raise_dyn_smem((const void*)pas::recon_kernel<false>, smem);
  } else {
    std::vector<uint16_t> Rb((size_t)n_modes * r->n_s_pad, 0);
    std::vector<float> scale(n_modes, 1.f);
    for (int m = 0; m < n_modes; ++m) {
      float mx = 0.f;
      for (int j = 0; j < n_slopes; ++j) mx = std::max(mx, std::fabs(h_R[(size_t)m * n_slopes + j]));
      scale[m] = mx > 0.f ? mx : 1.f;
      for (int j = 0; j < n_slopes; ++j)
        Rb[(size_t)m * r->n_s_pad + j] = pas::f32_to_bf16_rne(h_R[(size_t)m * n_slopes + j] / scale[m]);
    }
    st = pas::dev_alloc(ctx, (void**)&r->d_Rb, sizeof(uint16_t) * Rb.size());
    if (st == PAS_OK) st = pas::dev_alloc(ctx, (void**)&r->d_scale, sizeof(float) * n_modes);
    if (st == PAS_OK) e = cudaMemcpy(r->d_Rb, Rb.data(), sizeof(uint16_t) * Rb.size(), cudaMemcpyHostToDevice);
    if (st == PAS_OK && e == cudaSuccess)
      e = cudaMemcpy(r->d_scale, scale.data(), sizeof(float) * n_modes, cudaMemcpyHostToDevice);
    if (st == PAS_OK && e == cudaSuccess)
      e = pas::raise_dyn_smem((const void*)pas::recon_kernel<true>, smem);
  }
  if (st == PAS_OK) st = pas::dev_alloc(ctx, (void**)&r->d_done, sizeof(unsigned int));
  if (st == PAS_OK && e == cudaSuccess) e = cudaMemset(r->d_done, 0, sizeof(unsigned int));
  if (st != PAS_OK) {
    pas_recon_destroy(r);
    return st;
  }
  if (e != cudaSuccess) {
    pas_recon_destroy(r);
    return pas::set_error(ctx, PAS_ECUDA, "pas_recon_create: %s", cudaGetErrorString(e));
  }
  *out = r;
  return PAS_OK;
}

pas_status pas_recon_apply(pas_recon_t r, const float* d_slopes, float* d_dmodes) {
  if (!r || !d_slopes || !d_dmodes) return pas::set_global_error(PAS_EINVAL, "pas_recon_apply: NULL argument");
  pas::ReconArgs a;
  a.s = d_slopes;
  a.dmodes = d_dmodes;
  return pas::recon_launch(r, a, r->ctx->stream);
}

}  // extern "C"
