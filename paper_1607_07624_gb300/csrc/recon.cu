// Modal reconstructor dmodes = R * slopes (Table 1 modalrec.recmat_tag) and the
// integrator control c_t = c_{t-1} + g * dmodes (Table 1 control, type 'INT'),
// fused into one kernel for the loop.
//
// The matrix-vector product reads every element of R once per step: it is bound
// by memory bandwidth, so it runs on CUDA cores with 16-byte loads: four warps per
// mode row and the slope vector staged in shared memory for short vectors, one warp
// per row fed by bulk copies and slopes read through L1 for long ones
// (recon_bulk_kernel). PAS_BF16 stores R as
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

// The same product for long slope vectors (n_s >= RECON_BULK_MIN_NS): each warp owns
// one mode row and streams it through a ring of RB_NS shared-memory slots filled by
// 1-D bulk copies (cp.async.bulk, the TMA engine, completion on one mbarrier per slot),
// so the bytes in flight do not depend on registers; the slopes are read through L1
// (every CTA of an SM shares one copy). The first slots are requested before the
// programmatic wait (R is constant). Every wait is bounded: a slot that does not fill
// sets *err, and the warp waits (with the long bound) for the copies it still has in
// flight before it leaves.
constexpr int RB_WARPS = 4;            // rows (warps) per CTA
constexpr int RB_NS = 3;               // slots per warp (24 KB per CTA: 9 CTAs per SM, one wave of rows)
constexpr int RB_CH = 2048;            // bytes per slot (a multiple of 512: 16 bytes per lane per step)
constexpr int RECON_BULK_MIN_NS = 4096;
constexpr size_t RB_SMEM = (size_t)RB_WARPS * RB_NS * RB_CH;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Slopes of the 16-byte chunk c of an R row (8 bf16 or 4 float32 columns) from
// global memory through L1; columns at or beyond n_s (row padding) read as 0.
template <bool BF16>
__device__ __forceinline__ void slope_chunk(const float* s, int n_s, int c, float4* lo, float4* hi) {
  constexpr int W = BF16 ? 8 : 4;
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

constexpr uint32_t RB_WAIT_LIMIT = 1u << 22;  // tries of one wait (seconds, far beyond a copy)

template <bool BF16>
__global__ void __launch_bounds__(RB_WARPS * 32) recon_bulk_kernel(ReconArgs a) {
  extern __shared__ __align__(128) unsigned char rb_ring[];  // [warp][slot][RB_CH]
  __shared__ __align__(8) uint64_t bar[RB_WARPS][RB_NS];
  __shared__ bool is_last;
  pdl_trigger();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = blockIdx.x * RB_WARPS + warp;
  constexpr int ES = BF16 ? 2 : 4;  // bytes per element of R
  const int row_bytes = a.n_s_pad * ES;
  const int nch = (row_bytes + RB_CH - 1) / RB_CH;
  const char* src = nullptr;
  if (m < a.n_m) src = (BF16 ? reinterpret_cast<const char*>(a.Rb) : reinterpret_cast<const char*>(a.R)) +
                       (size_t)m * row_bytes;
  unsigned char* ring = rb_ring + (size_t)warp * RB_NS * RB_CH;
  if (lane == 0) {
    for (int s = 0; s < RB_NS; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[warp][s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  auto issue = [&](int c) {
    const int bytes = min(RB_CH, row_bytes - c * RB_CH);
    bulk_copy_g2s(ring + (size_t)(c % RB_NS) * RB_CH, src + (size_t)c * RB_CH, (uint32_t)bytes,
                  &bar[warp][c % RB_NS]);
  };
  if (lane == 0 && src)
    for (int c = 0; c < min(RB_NS, nch); ++c) issue(c);
  const bool writer = lane == 0 && m < a.n_m;
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
  int c = 0;
  bool ok = true;
  if (src) {
    for (; c < nch; ++c) {
      const int s = c % RB_NS;
      // every lane observes the slot's phase; the decision to go on is the warp's
      const bool got = bar_wait(&bar[warp][s], (uint32_t)(c / RB_NS) & 1u, RB_WAIT_LIMIT);
      if (!__all_sync(0xffffffffu, got)) {
        ok = false;
        break;
      }
      const int bytes = min(RB_CH, row_bytes - c * RB_CH);
      const unsigned char* slot = ring + (size_t)s * RB_CH;
#pragma unroll
      for (int q = 0; q < RB_CH / 512; ++q) {
        const int off = q * 512 + lane * 16;
        if (off < bytes) {
          const uint4 u = *reinterpret_cast<const uint4*>(slot + off);
          const int chunk = (c * RB_CH + off) / 16;  // index of this 16-byte chunk in the row
          float4 lo, hi;
          slope_chunk<BF16>(a.s, a.n_s, chunk, &lo, &hi);
          if constexpr (BF16) {
            const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
            const float2 f0 = __bfloat1622float2(h[0]), f1 = __bfloat1622float2(h[1]);
            const float2 f2 = __bfloat1622float2(h[2]), f3 = __bfloat1622float2(h[3]);
            acc = dot4(make_float4(f0.x, f0.y, f1.x, f1.y), lo, acc);
            acc = dot4(make_float4(f2.x, f2.y, f3.x, f3.y), hi, acc);
          } else {
            acc = dot4(*reinterpret_cast<const float4*>(&u), lo, acc);
          }
        }
      }
      __syncwarp();  // every lane has read slot s
      if (lane == 0 && c + RB_NS < nch) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // reads before the copy's writes
        issue(c + RB_NS);
      }
    }
  }
  if (!ok && lane == 0) {
    // a slot did not fill: record it, then let the copies still in flight land
    atomicOr(a.err, 1u);
    for (int d = c; d < min(nch, c + RB_NS); ++d)
      if (!bar_wait(&bar[warp][d % RB_NS], (uint32_t)(d / RB_NS) & 1u, RB_WAIT_LIMIT)) atomicOr(a.err, 2u);
  }
  __syncwarp();
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (writer) {
    const float dm = hold ? 0.f : (BF16 ? acc * a.scale[m] : acc);
    if (a.dmodes) a.dmodes[m] = dm;
    if (a.ring) {
      const float cnew = hold ? prev : fmaf(a.gain ? a.gain[m] : 1.0f, dm, prev);
      a.ring[(size_t)(t_step % a.delay) * a.n_m + m] = cnew;
      if (a.cmd_last) a.cmd_last[m] = cnew;
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

// The product for long slope vectors up to RT_MAX_NS: a TMA pipeline over whole rows.
// Thread 0 streams the CTA's mode rows, one bulk copy per row (split into pieces of at
// most 16 KB, all counted on the row slot's "full" mbarrier), into a ring of RT_NS row
// slots; each of the 8 warps owns the same column groups of every row (group g = u 8 +
// warp: 32 chunks of 16 bytes, so a warp reads 512 contiguous bytes per step), keeps
// the slopes of those columns in registers, and arrives on the slot's "empty" barrier
// when it has read its part; thread 0 refills a slot once all 8 warps have arrived.
// Per-row, per-warp partial sums meet in shared memory and are added in warp order.
// Waits are bounded: one that gives up sets *err and a shared abort flag, every warp
// leaves the row loop, and thread 0 waits (long bound) for its copies still in flight.
constexpr int RT_WARPS = 8;
constexpr int RT_MAX_NS = 16384;           // slopes held in registers: 64 per lane
constexpr int RT_MAX_ROWS = 64;            // rows per CTA (partial-sum table)
constexpr size_t RT_SLOT_BUDGET = 96 * 1024;  // shared memory for the row slots of one CTA

template <bool BF16>
__global__ void __launch_bounds__(RT_WARPS * 32) recon_tma_kernel(ReconArgs a, int rows_per_cta, int ns_slots,
                                                                  int slot_bytes) {
  constexpr int W = BF16 ? 8 : 4;       // columns per 16-byte chunk
  constexpr int MAXG = BF16 ? 8 : 16;   // column groups per warp (64 slopes per lane)
  extern __shared__ __align__(128) unsigned char rt_smem[];  // [ns_slots][slot_bytes]
  __shared__ __align__(8) uint64_t full[4], empty[4];
  __shared__ float part[RT_MAX_ROWS][RT_WARPS];
  __shared__ volatile int abort_flag;
  __shared__ bool is_last;
  pdl_trigger();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int ES = BF16 ? 2 : 4;
  const int row_bytes = a.n_s_pad * ES;
  const int nc = a.n_s_pad / W;
  const int r0 = blockIdx.x * rows_per_cta;
  const int nrow = max(0, min(a.n_m, r0 + rows_per_cta) - r0);
  const char* Rbase = BF16 ? reinterpret_cast<const char*>(a.Rb) : reinterpret_cast<const char*>(a.R);
  if (threadIdx.x == 0) {
    for (int s = 0; s < ns_slots; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[s])), "r"(RT_WARPS) : "memory");
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int i) {  // row r0 + i into slot i % ns_slots
    unsigned char* dst = rt_smem + (size_t)(i % ns_slots) * slot_bytes;
    const char* src = Rbase + (size_t)(r0 + i) * row_bytes;
    uint64_t* bar = &full[i % ns_slots];
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(row_bytes)
                 : "memory");
    for (int o = 0; o < row_bytes; o += 16384) {
      const int bytes = min(16384, row_bytes - o);
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       smem_u32(dst + o)),
                   "l"(src + o), "r"(bytes), "r"(smem_u32(bar))
                   : "memory");
    }
  };
  int issued = 0;  // thread 0: rows requested so far
  if (threadIdx.x == 0)
    for (; issued < min(ns_slots, nrow); ++issued) issue(issued);  // R is constant: before the wait
  // the writer of row r0 + t is thread t; its integrator state is final before the wait
  const bool writer = threadIdx.x < nrow;
  long long t_step = 0;
  float prev = 0.f;
  bool hold = false;
  if (writer && a.ring) {
    t_step = *a.step;
    prev = a.ring[(size_t)((t_step - 1 + a.delay) % a.delay) * a.n_m + r0 + threadIdx.x];
    hold = a.n_int > 1 && (t_step + 1) % a.n_int != 0;
  }
  pdl_wait();
  // slopes of this lane's chunks (columns at or beyond n_s read as 0)
  float sl[MAXG][W];
#pragma unroll
  for (int u = 0; u < MAXG; ++u) {
    const int c = (u * RT_WARPS + warp) * 32 + lane;
    float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;
    if (c < nc) slope_chunk<BF16>(a.s, a.n_s, c, &lo, &hi);
    sl[u][0] = lo.x; sl[u][1] = lo.y; sl[u][2] = lo.z; sl[u][3] = lo.w;
    if constexpr (BF16) {
      sl[u][4] = hi.x; sl[u][5] = hi.y; sl[u][6] = hi.z; sl[u][7] = hi.w;
    }
  }
  for (int i = 0; i < nrow; ++i) {
    const int s = i % ns_slots;
    const uint32_t par = (uint32_t)(i / ns_slots) & 1u;
    const bool got = bar_wait(&full[s], par, RB_WAIT_LIMIT);
    if (!__all_sync(0xffffffffu, got)) {
      if (lane == 0) {
        atomicOr(a.err, 1u);
        abort_flag = 1;
      }
    }
    __syncwarp();
    if (abort_flag) break;
    const unsigned char* slot = rt_smem + (size_t)s * slot_bytes;
    float acc = 0.f;
#pragma unroll
    for (int u = 0; u < MAXG; ++u) {
      const int c = (u * RT_WARPS + warp) * 32 + lane;
      if (c < nc) {
        const uint4 q = *reinterpret_cast<const uint4*>(slot + (size_t)c * 16);
        if constexpr (BF16) {
          const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
          const float2 f0 = __bfloat1622float2(h[0]), f1 = __bfloat1622float2(h[1]);
          const float2 f2 = __bfloat1622float2(h[2]), f3 = __bfloat1622float2(h[3]);
          acc = fmaf(f0.x, sl[u][0], acc); acc = fmaf(f0.y, sl[u][1], acc);
          acc = fmaf(f1.x, sl[u][2], acc); acc = fmaf(f1.y, sl[u][3], acc);
          acc = fmaf(f2.x, sl[u][4], acc); acc = fmaf(f2.y, sl[u][5], acc);
          acc = fmaf(f3.x, sl[u][6], acc); acc = fmaf(f3.y, sl[u][7], acc);
        } else {
          const float4 f = *reinterpret_cast<const float4*>(&q);
          acc = fmaf(f.x, sl[u][0], acc); acc = fmaf(f.y, sl[u][1], acc);
          acc = fmaf(f.z, sl[u][2], acc); acc = fmaf(f.w, sl[u][3], acc);
        }
      }
    }
    __syncwarp();  // this warp has read its part of the slot
    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[s])) : "memory");
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) part[i][warp] = acc;
    if (threadIdx.x == 0 && issued < nrow) {
      // refill slot s with row `issued` once every warp has read row i
      if (!bar_wait(&empty[s], par, RB_WAIT_LIMIT)) {
        atomicOr(a.err, 4u);
        abort_flag = 1;
      } else {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(issued);
        ++issued;
      }
    }
  }
  if (threadIdx.x == 0 && abort_flag) {
    // the last requested row of each slot may still be in flight: let those copies land
    // (an earlier row of a slot completed before the slot was refilled)
    for (int i = max(0, issued - ns_slots); i < issued; ++i)
      if (!bar_wait(&full[i % ns_slots], (uint32_t)(i / ns_slots) & 1u, RB_WAIT_LIMIT)) atomicOr(a.err, 2u);
  }
  __syncthreads();
  if (writer && !abort_flag) {
    const int m = r0 + threadIdx.x;
    float tot = 0.f;
#pragma unroll
    for (int w = 0; w < RT_WARPS; ++w) tot += part[threadIdx.x][w];
    const float dm = hold ? 0.f : (BF16 ? tot * a.scale[m] : tot);
    if (a.dmodes) a.dmodes[m] = dm;
    if (a.ring) {
      const float cnew = hold ? prev : fmaf(a.gain ? a.gain[m] : 1.0f, dm, prev);
      a.ring[(size_t)(t_step % a.delay) * a.n_m + m] = cnew;
      if (a.cmd_last) a.cmd_last[m] = cnew;
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
  a.err = r->d_err;
  cudaError_t e;
  const size_t row_bytes = (size_t)r->n_s_pad * (r->prec == PAS_BF16 ? 2 : 4);
  const bool aligned = (reinterpret_cast<uintptr_t>(a.s) & 15u) == 0;
  if (r->rt_rows > 0 && aligned) {
    const size_t smem = (size_t)r->rt_slots * row_bytes;
    const int grid = (r->n_modes + r->rt_rows - 1) / r->rt_rows;
    e = r->prec == PAS_BF16
            ? launch_k(recon_tma_kernel<true>, dim3(grid), dim3(RT_WARPS * 32), smem, st, pdl, a, r->rt_rows,
                       r->rt_slots, (int)row_bytes)
            : launch_k(recon_tma_kernel<false>, dim3(grid), dim3(RT_WARPS * 32), smem, st, pdl, a, r->rt_rows,
                       r->rt_slots, (int)row_bytes);
  } else if (r->n_slopes >= RECON_BULK_MIN_NS && aligned) {
    const int grid = (r->n_modes + RB_WARPS - 1) / RB_WARPS;
    e = r->prec == PAS_BF16 ? launch_k(recon_bulk_kernel<true>, dim3(grid), dim3(RB_WARPS * 32), RB_SMEM, st, pdl, a)
                            : launch_k(recon_bulk_kernel<false>, dim3(grid), dim3(RB_WARPS * 32), RB_SMEM, st, pdl, a);
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
  pas::dev_free(r->d_err);
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
  if (st == PAS_OK) st = pas::dev_alloc(ctx, (void**)&r->d_err, sizeof(unsigned int));
  if (st == PAS_OK && e == cudaSuccess) e = cudaMemset(r->d_done, 0, sizeof(unsigned int));
  if (st == PAS_OK && e == cudaSuccess) e = cudaMemset(r->d_err, 0, sizeof(unsigned int));
  if (st == PAS_OK && e == cudaSuccess)
    e = prec == PAS_BF16 ? pas::raise_dyn_smem((const void*)pas::recon_bulk_kernel<true>, pas::RB_SMEM)
                         : pas::raise_dyn_smem((const void*)pas::recon_bulk_kernel<false>, pas::RB_SMEM);
  if (st == PAS_OK && e == cudaSuccess && n_slopes >= pas::RECON_BULK_MIN_NS && r->n_s_pad <= pas::RT_MAX_NS) {
    // the TMA row pipeline: 2 to 4 row slots within the budget; rows per CTA so that
    // every CTA is resident at once (the CTAs per SM the registers and slots allow)
    const size_t rb = (size_t)r->n_s_pad * (prec == PAS_BF16 ? 2 : 4);
    r->rt_slots = (int)std::max<size_t>(2, std::min<size_t>(4, pas::RT_SLOT_BUDGET / rb));
    const void* kern = prec == PAS_BF16 ? (const void*)pas::recon_tma_kernel<true>
                                        : (const void*)pas::recon_tma_kernel<false>;
    e = pas::raise_dyn_smem(kern, r->rt_slots * rb);
    int occ = 0;
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, pas::RT_WARPS * 32, r->rt_slots * rb);
    if (e == cudaSuccess && occ > 0) {
      const int slots_total = occ * std::max(1, ctx->sm_count);
      r->rt_rows = std::min(pas::RT_MAX_ROWS, std::max(1, (n_modes + slots_total - 1) / slots_total));
    }
  }
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

pas_status pas_recon_check(pas_recon_t r, uint32_t* h_fault) {
  if (!r) return pas::set_global_error(PAS_EINVAL, "pas_recon_check: NULL argument");
  unsigned int f = 0;
  PAS_CUDA_TRY(r->ctx, cudaMemcpy(&f, r->d_err, sizeof(f), cudaMemcpyDeviceToHost));
  if (h_fault) *h_fault = f;
  if (f) {
    PAS_CUDA_TRY(r->ctx, cudaMemset(r->d_err, 0, sizeof(unsigned int)));
    return pas::set_error(r->ctx, PAS_ETIMEOUT, "reconstructor: a bulk-copy wait gave up (code %u)", f);
  }
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
