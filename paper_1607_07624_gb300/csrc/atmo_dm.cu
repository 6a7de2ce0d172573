// Atmosphere propagation (wind-shifted layers summed on the pupil) and the modal DM
// (influence-function multiplication) with the residual seen by the sensor
// (Table 1 atmo / wind_speed / wind_direction / DM; Table 2 get_atmo_propagation,
// add_layer_to_layer_list(dm.out_layer); Sec. GPU acceleration, "wavefront
// propagation through phase screens" and "influence function multiplication").
#include <algorithm>
#include <cmath>
#include <vector>

#include "atmo_dm.cuh"
#include "internal.h"
#include "pdl.cuh"
#include "tc.cuh"

namespace pas {

// Per-layer integer shift and float32 bilinear weights at `step`: sample position of
// pupil pixel i is i + o - step*v = i + n + f, n = floor(o - step*v) (o: the layer's
// footprint offset for an off-axis source, 0 on axis).
__device__ inline void layer_shift(double v, double o, long long step, int S, int* n_mod, float* f) {
  const double d = o - (double)step * v;
  const double n = floor(d);
  *f = (float)(d - n);
  long long ni = (long long)n % S;
  if (ni < 0) ni += S;
  *n_mod = (int)ni;
}

// Cone effect of a source at finite height: the sample position of pupil pixel i in
// a layer whose footprint is scaled by s about the pupil centre c = (Np - 1) / 2 is
// c + (i - c) s + o - step*v, one FP64 value per (layer, pixel) with explicit
// rounding; n_mod = floor mod S, f = the float32 fraction.
__device__ inline void cone_shift(int i, int Np, double s, double v, double o, long long step, int S, int* n_mod,
                                  float* f) {
  const double c = 0.5 * (double)(Np - 1);
  const double d = __dadd_rn(__dadd_rn(c, __dmul_rn(__dsub_rn((double)i, c), s)),
                             __dsub_rn(o, __dmul_rn((double)step, v)));
  const double n = floor(d);
  *f = (float)(d - n);
  long long ni = (long long)n % S;
  if (ni < 0) ni += S;
  *n_mod = (int)ni;
}

// Bilinear interpolation of one layer from its four taps, with explicit float32
// rounding (the same value in every kernel that samples the atmosphere).
__device__ __forceinline__ float bilinear(float fx, float fy, float v00, float v10, float v01, float v11) {
  const float gx = __fsub_rn(1.f, fx), gy = __fsub_rn(1.f, fy);
  float s = __fmul_rn(__fmul_rn(gx, gy), v00);
  s = __fmaf_rn(__fmul_rn(fx, gy), v10, s);
  s = __fmaf_rn(__fmul_rn(gx, fy), v01, s);
  return __fmaf_rn(__fmul_rn(fx, fy), v11, s);
}

// Offsets of the four taps (00, 10, 01, 11) of pupil pixel (i, j) in one layer.
__device__ __forceinline__ void tap_offsets(int i, int j, int shift_i, int shift_j, int S, size_t off[4]) {
  int i0 = i + shift_i;
  if (i0 >= S) i0 -= S;
  int j0 = j + shift_j;
  if (j0 >= S) j0 -= S;
  const int i1 = (i0 + 1 == S) ? 0 : i0 + 1;
  const int j1 = (j0 + 1 == S) ? 0 : j0 + 1;
  off[0] = (size_t)i0 * S + j0;
  off[1] = (size_t)i1 * S + j0;
  off[2] = (size_t)i0 * S + j1;
  off[3] = (size_t)i1 * S + j1;
}

__device__ inline float atmo_sample(const AtmoArgs& a, const int* six, const int* siy,
                                    const float* sfx, const float* sfy, int i, int j) {
  float acc = 0.f;
  const int S = a.S;
  for (int l = 0; l < a.L; ++l) {
    size_t o[4];
    tap_offsets(i, j, six[l], siy[l], S, o);
    const float* sc = a.screens + (size_t)l * S * S;
    acc = __fadd_rn(acc, bilinear(sfx[l], sfy[l], __ldg(sc + o[0]), __ldg(sc + o[1]), __ldg(sc + o[2]),
                                  __ldg(sc + o[3])));
  }
  return acc;
}

// Same sum with the layer count known at compile time: all 4 L taps are issued
// before the first one is used.
template <int L>
__device__ inline float atmo_sample_fixed(const AtmoArgs& a, const int* six, const int* siy,
                                          const float* sfx, const float* sfy, int i, int j) {
  const int S = a.S;
  float v[L][4];
#pragma unroll
  for (int l = 0; l < L; ++l) {
    size_t o[4];
    tap_offsets(i, j, six[l], siy[l], S, o);
    const float* sc = a.screens + (size_t)l * S * S;
#pragma unroll
    for (int t = 0; t < 4; ++t) v[l][t] = __ldg(sc + o[t]);
  }
  float acc = 0.f;
#pragma unroll
  for (int l = 0; l < L; ++l) acc = __fadd_rn(acc, bilinear(sfx[l], sfy[l], v[l][0], v[l][1], v[l][2], v[l][3]));
  return acc;
}

__device__ inline float atmo_sample_any(const AtmoArgs& a, const int* six, const int* siy,
                                        const float* sfx, const float* sfy, int i, int j) {
  switch (a.L) {
    case 1: return atmo_sample_fixed<1>(a, six, siy, sfx, sfy, i, j);
    case 2: return atmo_sample_fixed<2>(a, six, siy, sfx, sfy, i, j);
    case 3: return atmo_sample_fixed<3>(a, six, siy, sfx, sfy, i, j);
    case 4: return atmo_sample_fixed<4>(a, six, siy, sfx, sfy, i, j);
    case 5: return atmo_sample_fixed<5>(a, six, siy, sfx, sfy, i, j);
    case 6: return atmo_sample_fixed<6>(a, six, siy, sfx, sfy, i, j);
    default: return atmo_sample(a, six, siy, sfx, sfy, i, j);
  }
}

// The same sum for a source at finite height (per-pixel cone positions).
__device__ inline float atmo_sample_cone(const AtmoArgs& a, long long step, int i, int j) {
  float acc = 0.f;
  const int S = a.S;
  for (int l = 0; l < a.L; ++l) {
    int ni, nj;
    float fx, fy;
    cone_shift(i, a.Np, a.sc[l], a.vx[l], a.ox[l], step, S, &ni, &fx);
    cone_shift(j, a.Np, a.sc[l], a.vy[l], a.oy[l], step, S, &nj, &fy);
    size_t o[4];
    tap_offsets(0, 0, ni, nj, S, o);
    const float* sc = a.screens + (size_t)l * S * S;
    acc = __fadd_rn(acc, bilinear(fx, fy, __ldg(sc + o[0]), __ldg(sc + o[1]), __ldg(sc + o[2]), __ldg(sc + o[3])));
  }
  return acc;
}

__global__ void atmo_kernel(AtmoArgs a, const long long* d_step, long long h_step, float* out) {
  __shared__ int six[PAS_MAX_LAYERS], siy[PAS_MAX_LAYERS];
  __shared__ float sfx[PAS_MAX_LAYERS], sfy[PAS_MAX_LAYERS];
  const long long step = d_step ? *d_step : h_step;
  if (threadIdx.x < a.L) {
    layer_shift(a.vx[threadIdx.x], a.ox[threadIdx.x], step, a.S, &six[threadIdx.x], &sfx[threadIdx.x]);
    layer_shift(a.vy[threadIdx.x], a.oy[threadIdx.x], step, a.S, &siy[threadIdx.x], &sfy[threadIdx.x]);
  }
  __syncthreads();
  const int n = a.Np * a.Np;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int i = p / a.Np, j = p - i * a.Np;
    out[p] = a.cone ? atmo_sample_cone(a, step, i, j) : atmo_sample_any(a, six, siy, sfx, sfy, i, j);
  }
}

// Residual over the pupil pixel list: out[pix] = atm - dm_sign * (M c), atm the
// layers sampled at the step (a.atmo.L > 0), else read from opd_atm (or zero). CTA: one 64-pixel tile, whose basis block [n_m][64] is
// one contiguous stretch of memory. Each thread owns VEC consecutive pixels (one
// 16-byte load: 4 float or 8 bfloat16 values) and every ROWS-th mode: it streams
// those rows straight from global memory (a warp reads whole 256-byte or 128-byte
// mode rows per load) with RES_U loads in flight, accumulating in float32; the
// ROWS partial sums per pixel meet once in shared memory at the end. The basis is
// constant, so the first loads are issued before the programmatic wait and
// overlap the predecessor kernel.
constexpr int RES_THREADS = 256;
constexpr int RES_U = 5;            // loads in flight per thread

// Floats of the residual kernel's shared head: the command, which the ROWS partial
// sums per pixel and the L bilinear values per pixel replace after the stream.
template <typename T>
__host__ __device__ inline int res_head(int n_m, int L) {
  constexpr int rows = RES_THREADS / (RES_TILE / (16 / (int)sizeof(T)));
  const int post = (rows + L) * RES_TILE;
  return n_m > post ? n_m : (post > 1 ? post : 1);
}

__device__ __forceinline__ uint4 ld_stream16(const void* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

template <typename T>
__device__ __forceinline__ void unpack16(const uint4& u, float* f) {
  if constexpr (sizeof(T) == 4) {
    f[0] = __uint_as_float(u.x);
    f[1] = __uint_as_float(u.y);
    f[2] = __uint_as_float(u.z);
    f[3] = __uint_as_float(u.w);
  } else {  // bfloat16: the value is the upper half of a float32
    const unsigned w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      f[2 * i] = __uint_as_float(w[i] << 16);
      f[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
  }
}

// 4-byte asynchronous global -> shared copy (no register holds the value in flight).
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
// One box of 2 rows x RES_BOX floats of layer z from screen row y, column x (a
// multiple of 4) into shared memory (128-byte aligned), counted on `bar` in bytes.
__device__ __forceinline__ void tma_load_box(float* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(
          tc::smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(tc::smem_addr(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// With a.atmo.L > 0 the atmosphere is sampled here (the loop's step: layers
// shifted by the wind of the device step, bilinear taps at the tile's pupil
// pixels): the 4 L taps of the tile's pixels are copied to shared memory
// asynchronously before the basis stream and combined after it, so their latency
// hides under the stream; otherwise the atmosphere is read from opd_atm (or zero).
// CONE: a source at finite height; each (layer, pixel) has its own taps and
// weights (cone_shift), the weights kept in shared memory after the taps.
// TMA (sources at infinity, a.tma): the taps come as tensor copies instead: per layer
// and pupil-row segment of the tile, one box of the two screen rows it samples,
// RES_BOX floats from the segment's first column rounded down to 16 bytes, issued by
// one thread on one mbarrier before the basis stream and read back after it. Taps
// past the screen's last row or column (the periodic screen wraps there; the box
// holds the fill value) are read from global memory instead.
template <typename T, bool CONE, bool TMA>
__global__ void __launch_bounds__(RES_THREADS, 5) residual_kernel(const __grid_constant__ ResArgs a) {
  constexpr int VEC = 16 / (int)sizeof(T);         // pixels per 16-byte load
  constexpr int COLS = RES_TILE / VEC;              // loads per mode row
  constexpr int ROWS = RES_THREADS / COLS;          // modes per CTA-wide load
  // [P] the command (after the stream: the ROWS partial sums [ROWS][RES_TILE], then
  // with TMA the bilinear values [L][RES_TILE]), then the taps [L][4][RES_TILE] or the
  // boxes
  extern __shared__ float c_s[];
  __shared__ int s_flat[RES_TILE];
  __shared__ double wred[2][RES_THREADS / 32];
  __shared__ int six[PAS_MAX_LAYERS], siy[PAS_MAX_LAYERS];
  __shared__ float sfx[PAS_MAX_LAYERS], sfy[PAS_MAX_LAYERS];
  __shared__ int4 s_seg[TMA ? RES_SEG_MAX : 1];
  __shared__ __align__(8) uint64_t tbar;
  const int tid = threadIdx.x;
  const T* MT = nullptr;
  if constexpr (sizeof(T) == 4) MT = a.MT;
  else MT = a.MTb;
  const int n_m = MT ? a.n_m : 0;
  const int col = tid % COLS, row = tid / COLS;
  const T* blk = MT + (size_t)blockIdx.x * n_m * RES_TILE + col * VEC;
  uint4 v[RES_U];
#pragma unroll
  for (int u = 0; u < RES_U; ++u) {
    const int m = row + ROWS * u;
    v[u] = m < n_m ? ld_stream16(blk + (size_t)m * RES_TILE) : make_uint4(0u, 0u, 0u, 0u);
  }
  const int base = blockIdx.x * RES_TILE;
  const int L = a.atmo.L;
  if (tid < RES_TILE) s_flat[tid] = base + tid < a.n_pix ? a.pix[base + tid] : 0;  // constant
  if constexpr (TMA) {
    if (tid < a.seg_max) s_seg[tid] = a.seg[(size_t)blockIdx.x * a.seg_max + tid];  // constant
    if (tid == 0) {
      tc::mbar_init(&tbar, 1);
      tc::fence_barrier_init();
    }
    if (tid == 32) tc::prefetch_tensormap(&a.tmap);
  }
  pdl_trigger();
  pdl_wait();
  const long long step = a.d_step ? *a.d_step : a.h_step;
  const float* cmd = a.cmd;
  if (a.cmd_ring) cmd = a.cmd_ring + (size_t)(step % a.delay) * a.n_m;
  if (!CONE && tid < L) {
    layer_shift(a.atmo.vx[tid], a.atmo.ox[tid], step, a.atmo.S, &six[tid], &sfx[tid]);
    layer_shift(a.atmo.vy[tid], a.atmo.oy[tid], step, a.atmo.S, &siy[tid], &sfy[tid]);
  }
  for (int m = tid; m < n_m; m += RES_THREADS) c_s[m] = cmd[m];
  __syncthreads();
  float* taps = c_s + res_head<T>(a.n_m, L);
  float* wts = taps + L * 4 * RES_TILE;             // CONE: [L][2][RES_TILE] weights
  // TMA: boxes [L][seg_max][RES_BOX_PITCH] (2 rows of RES_BOX), from the first
  // 128-byte boundary after the command
  float* boxes = nullptr;
  if constexpr (TMA) {
    const uint32_t sa = tc::smem_addr(taps);
    boxes = taps + (((sa + 127u) & ~127u) - sa) / 4u;
  }
  const int S = a.atmo.S;
  if constexpr (TMA) {
    // thread 0 announces the bytes; thread t < L seg_max copies box (t / seg_max,
    // t % seg_max) (a copy that lands before the announcement leaves the phase open:
    // it completes on thread 0's arrival)
    if (tid == 0 && L > 0) {
      int ns = 0;
      for (int sg = 0; sg < a.seg_max; ++sg) ns += s_seg[sg].z > 0 ? 1 : 0;
      tc::mbar_arrive_expect_tx(&tbar, (uint32_t)(L * ns) * 2u * RES_BOX * 4u);
    }
    if (tid < L * a.seg_max) {
      const int l = tid / a.seg_max, sg = tid - l * a.seg_max;
      const int4 q = s_seg[sg];
      if (q.z > 0) {
        int c = q.y + siy[l];
        if (c >= S) c -= S;
        int row = q.x + six[l];
        if (row >= S) row -= S;
        tma_load_box(boxes + (size_t)tid * RES_BOX_PITCH, &a.tmap, &tbar, c & ~3, row, l);
      }
    }
  }
  if (!TMA && L > 0) {
    const int S = a.atmo.S;
    for (int t = tid; t < L * RES_TILE; t += RES_THREADS) {
      const int l = t / RES_TILE, q = t - l * RES_TILE;
      if (base + q < a.n_pix) {
        const int flat = s_flat[q];
        const int i = flat / a.atmo.Np, j = flat - i * a.atmo.Np;
        size_t o[4];
        if constexpr (CONE) {
          int ni, nj;
          cone_shift(i, a.atmo.Np, a.atmo.sc[l], a.atmo.vx[l], a.atmo.ox[l], step, S, &ni, wts + 2 * l * RES_TILE + q);
          cone_shift(j, a.atmo.Np, a.atmo.sc[l], a.atmo.vy[l], a.atmo.oy[l], step, S, &nj,
                     wts + (2 * l + 1) * RES_TILE + q);
          tap_offsets(0, 0, ni, nj, S, o);
        } else {
          tap_offsets(i, j, six[l], siy[l], S, o);
        }
        const float* sc = a.atmo.screens + (size_t)l * S * S;
#pragma unroll
        for (int k = 0; k < 4; ++k) cp_async4(taps + (l * 4 + k) * RES_TILE + q, sc + o[k]);
      }
    }
    cp_async_commit();
  }
  float acc[VEC];
#pragma unroll
  for (int i = 0; i < VEC; ++i) acc[i] = 0.f;
  for (int mb = row; mb < n_m; mb += ROWS * RES_U) {
#pragma unroll
    for (int u = 0; u < RES_U; ++u) {
      const int m = mb + ROWS * u;
      if (m < n_m) {
        const float cm = c_s[m];
        float f[VEC];
        unpack16<T>(v[u], f);
#pragma unroll
        for (int i = 0; i < VEC; ++i) acc[i] = fmaf(cm, f[i], acc[i]);
      }
      const int mn = m + ROWS * RES_U;
      if (mn < n_m) v[u] = ld_stream16(blk + (size_t)mn * RES_TILE);
    }
  }
  __syncthreads();  // every thread is done with the command
  float* red = c_s;
#pragma unroll
  for (int i = 0; i < VEC; ++i) red[row * RES_TILE + col * VEC + i] = acc[i];
  if constexpr (TMA) {
    // the boxes have landed (the threads that read them wait; a wait that gives up
    // flags the atmosphere and waits again, with the long bound, so that no copy is
    // in flight when the CTA moves on)
    if (L > 0 && !tc::mbar_wait(&tbar, 0, a.wait_limit)) {
      if (a.err) atomicOr(a.err, 1u);
      if (!tc::mbar_wait(&tbar, 0, tc::WAIT_LIMIT) && a.err) atomicOr(a.err, 2u);
    }
    // each (layer, pixel) pair's bilinear value, [L][RES_TILE] after the partial sums:
    // the pixel's segment, its column offset in the segment's box, taps past the
    // screen's last row or column from global memory
    float* bil = c_s + ROWS * RES_TILE;
    for (int t = tid; t < L * RES_TILE; t += RES_THREADS) {
      const int l = t / RES_TILE, px = t - l * RES_TILE;
      if (base + px < a.n_pix) {
        int si = 0;
        for (int sg = 1; sg < a.seg_max; ++sg)
          if (s_seg[sg].z > 0 && px >= s_seg[sg].w) si = sg;
        const int4 q = s_seg[si];
        int c = q.y + siy[l];
        if (c >= S) c -= S;
        int r0 = q.x + six[l];
        if (r0 >= S) r0 -= S;
        const int x0 = c & ~3, u0 = c - x0 + (px - q.w);
        const float* bx = boxes + (size_t)(l * a.seg_max + si) * RES_BOX_PITCH;
        const float* sc = a.atmo.screens + (size_t)l * S * S;
        auto tap = [&](int r, int u) {
          const int rr = r0 + r, cc = x0 + u;
          if (rr < S && cc < S) return bx[r * RES_BOX + u];
          return __ldg(sc + (size_t)(rr < S ? rr : rr - S) * S + (cc < S ? cc : cc - S));
        };
        bil[t] = bilinear(sfx[l], sfy[l], tap(0, u0), tap(1, u0), tap(0, u0 + 1), tap(1, u0 + 1));
      }
    }
  }
  if (!TMA && L > 0) {
    // each (layer, pixel) pair's bilinear value replaces its first tap
    cp_async_wait_all();
    __syncthreads();
    for (int t = tid; t < L * RES_TILE; t += RES_THREADS) {
      const int l = t / RES_TILE, q = t - l * RES_TILE;
      float* tp = taps + l * 4 * RES_TILE + q;
      if (base + q < a.n_pix) {
        float fx, fy;
        if constexpr (CONE) {
          fx = wts[2 * l * RES_TILE + q];
          fy = wts[(2 * l + 1) * RES_TILE + q];
        } else {
          fx = sfx[l];
          fy = sfy[l];
        }
        tp[0] = bilinear(fx, fy, tp[0], tp[RES_TILE], tp[2 * RES_TILE], tp[3 * RES_TILE]);
      }
    }
  }
  __syncthreads();
  const int px = tid;
  const int p = base + px;
  float s1 = 0.f, s2 = 0.f;
  if (px < RES_TILE && p < a.n_pix) {
    const int flat = s_flat[px];
    float atm = 0.f;
    if (TMA && L > 0) {
      const float* bil = c_s + ROWS * RES_TILE;
      for (int l = 0; l < L; ++l) atm = __fadd_rn(atm, bil[l * RES_TILE + px]);
    } else if (L > 0) {
      for (int l = 0; l < L; ++l) atm = __fadd_rn(atm, taps[l * 4 * RES_TILE + px]);
    } else if (a.opd_atm) {
      atm = a.opd_atm[flat];
    }
    float dm = 0.f;
#pragma unroll
    for (int r = 0; r < ROWS; ++r) dm += red[r * RES_TILE + px];
    const float r = atm - a.dm_sign * dm;
    a.out[flat] = r;
    s1 = r;
    s2 = r * r;
  }
  if (a.wfe_part) {
    // the tile's (sum r, sum r^2): float within each of the output warps (FP64 is a
    // slow pipe here), the warps' sums added in double by thread 0
    constexpr int OUT_WARPS = RES_TILE / 32;
    const int warp = tid >> 5, lane = tid & 31;
    if (warp < OUT_WARPS) {
      float f1 = (float)s1, f2 = (float)s2;
      for (int o = 16; o > 0; o >>= 1) {
        f1 += __shfl_down_sync(0xffffffffu, f1, o);
        f2 += __shfl_down_sync(0xffffffffu, f2, o);
      }
      if (lane == 0) {
        wred[0][warp] = f1;
        wred[1][warp] = f2;
      }
    }
    __syncthreads();
    if (tid == 0) {
      double t1 = 0.0, t2 = 0.0;
      for (int w = 0; w < OUT_WARPS; ++w) {
        t1 += wred[0][w];
        t2 += wred[1][w];
      }
      a.wfe_part[blockIdx.x] = make_double2(t1, t2);
    }
  }
}

// Zero the pixels of an Np x Np map outside the pupil.
__global__ void zero_outside_kernel(float* out, int Np, long long T) {
  const int n = Np * Np;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const int i = p / Np, j = p - i * Np;
    const long long ai = 2LL * i - Np + 1, bj = 2LL * j - Np + 1;
    const long long d2 = ai * ai + bj * bj;
    if (!(d2 <= (long long)Np * Np && d2 >= T)) out[p] = 0.f;
  }
}

__global__ void integrate_kernel(float* cmd, const float* dmodes, const float* gain, int n) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < n) cmd[m] += (gain ? gain[m] : 1.0f) * dmodes[m];
}

int residual_tiles(int n_pix) { return (n_pix + RES_TILE - 1) / RES_TILE; }

// The residual kernel streams its basis through registers, not the L1 cache: its
// launch bounds (at most 51 registers) and a shared-memory carveout preference keep
// five CTAs resident per SM (one wave for the 700 tiles of a 240 px pupil); the rest of
// the unified memory stays L1, where the loads in flight land.
template <typename T, bool CONE, bool TMA>
static cudaError_t residual_prepare(size_t smem) {
  static bool carveout_set = false;
  cudaError_t e = raise_dyn_smem((const void*)residual_kernel<T, CONE, TMA>, smem);
  if (e == cudaSuccess && !carveout_set) {
    e = cudaFuncSetAttribute((const void*)residual_kernel<T, CONE, TMA>,
                             cudaFuncAttributePreferredSharedMemoryCarveout, 50);
    carveout_set = e == cudaSuccess;
  }
  return e;
}

template <typename T, bool CONE, bool TMA>
static cudaError_t residual_start(const ResArgs& a, int tiles, size_t smem, cudaStream_t st, bool pdl) {
  cudaError_t e = residual_prepare<T, CONE, TMA>(smem);
  if (e == cudaSuccess) e = launch_k(residual_kernel<T, CONE, TMA>, dim3(tiles), dim3(RES_THREADS), smem, st, pdl, a);
  return e;
}

pas_status residual_launch(pas_ctx_t ctx, const ResArgs& a, cudaStream_t st, bool pdl) {
  const int tiles = residual_tiles(a.n_pix);
  if (tiles == 0) return PAS_OK;
  if (a.atmo.L < 0 || a.atmo.L > PAS_MAX_LAYERS)
    return set_error(ctx, PAS_EINVAL, "residual kernel: 0 <= layers <= %d", PAS_MAX_LAYERS);
  const bool cone = a.atmo.L > 0 && a.atmo.cone;
  const bool tma = a.atmo.L > 0 && !cone && a.tma && a.seg && a.seg_max >= 1 && a.seg_max <= RES_SEG_MAX;
  const int head = a.MTb ? res_head<__nv_bfloat16>(a.n_m, a.atmo.L) : res_head<float>(a.n_m, a.atmo.L);
  const size_t smem =
      tma ? sizeof(float) * ((size_t)head + 32 + (size_t)a.atmo.L * a.seg_max * RES_BOX_PITCH)
          : sizeof(float) * ((size_t)head + (size_t)a.atmo.L * (cone ? 6 : 4) * RES_TILE);
  cudaError_t e;
  if (a.MTb)
    e = cone  ? residual_start<__nv_bfloat16, true, false>(a, tiles, smem, st, pdl)
        : tma ? residual_start<__nv_bfloat16, false, true>(a, tiles, smem, st, pdl)
              : residual_start<__nv_bfloat16, false, false>(a, tiles, smem, st, pdl);
  else
    e = cone  ? residual_start<float, true, false>(a, tiles, smem, st, pdl)
        : tma ? residual_start<float, false, true>(a, tiles, smem, st, pdl)
              : residual_start<float, false, false>(a, tiles, smem, st, pdl);
  if (e != cudaSuccess) return set_error(ctx, PAS_ECUDA, "residual kernel launch: %s", cudaGetErrorString(e));
  return PAS_OK;
}

// Modal projection c_j = (1/n_pix) sum_p M[p][j] opd[pix[p]]: the least-squares
// modal coefficients for a basis with M^T M = n_pix I (the orthonormalised
// bases of the DM). One CTA per mode streams that mode's column of the tiled
// matrix; the OPD gather stays in L2 across CTAs.
template <typename T>
__global__ void __launch_bounds__(256) dm_project_kernel(const T* MT, const int32_t* pix, int n_pix, int n_m,
                                                         const float* opd, float* c) {
  __shared__ float red[8];
  const int j = blockIdx.x;
  float acc = 0.f;
  for (int p = threadIdx.x; p < n_pix; p += blockDim.x) {
    float m;
    if constexpr (sizeof(T) == 4) m = MT[((size_t)(p >> 6) * n_m + j) * 64 + (p & 63)];
    else m = __bfloat162float(MT[((size_t)(p >> 6) * n_m + j) * 64 + (p & 63)]);
    acc = fmaf(m, opd[pix[p]], acc);
  }
  for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < 8; ++i) t += red[i];
    c[j] = t / (float)n_pix;
  }
}

pas_status dm_project_launch(pas_dm_t dm, const float* opd, float* coeffs, cudaStream_t st) {
  if (dm->d_MTb)
    dm_project_kernel<<<dm->n_modes, 256, 0, st>>>(dm->d_MTb, dm->d_pix, dm->n_pix, dm->n_modes, opd, coeffs);
  else
    dm_project_kernel<<<dm->n_modes, 256, 0, st>>>(dm->d_MT, dm->d_pix, dm->n_pix, dm->n_modes, opd, coeffs);
  return check_launch(dm->ctx, "modal projection launch");
}


// ------------------------------------------------------------ batched residual
// The residuals of B loops that share one DM (realisations of one system): one pass
// over the basis serves them all. CTA (chunk, tile): the tile's basis block is
// streamed once for BC loops, each thread keeping BC x VEC accumulators; the
// chunks of a tile are neighbouring CTAs and share the block through L2. Per loop
// and pixel the arithmetic is that of residual_kernel (the same thread's modes in
// the same order, the same fused multiply-adds, the same sum over the ROWS partials,
// the same atmosphere taps and tile WFE sums), so every loop's residual and WFE
// partials equal those of its own residual kernel, bit for bit.
constexpr int RB_U = 6;  // basis loads in flight per thread

template <typename T>
__host__ __device__ constexpr int res_batch_bc() { return sizeof(T) == 4 ? 8 : 4; }  // BC x VEC = 32 accumulators

// cmdg[m][b] = the command that loop b's residual subtracts at its current step
// (slot step % delay of its ring); 0 in the padding columns.
__global__ void gather_cmds_kernel(const ResBatchLoop* loops, int B, int Bp, int n_m, float* cmdg) {
  pdl_trigger();
  const int tot = n_m * Bp;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x) {
    const int m = t / Bp, b = t - m * Bp;
    float c = 0.f;
    if (b < B) {
      const ResBatchLoop& L = loops[b];
      const long long step = *L.d_step;
      c = L.cmd_ring[(size_t)(step % L.delay) * n_m + m];
    }
    cmdg[t] = c;
  }
}

template <typename T>
__global__ void __launch_bounds__(RES_THREADS, 3) residual_batch_kernel(ResBatchArgs a) {
  constexpr int VEC = 16 / (int)sizeof(T);
  constexpr int COLS = RES_TILE / VEC;
  constexpr int ROWS = RES_THREADS / COLS;
  constexpr int BC = res_batch_bc<T>();
  extern __shared__ float taps[];                  // [BC][Lmax][4][RES_TILE]
  __shared__ float red[BC][ROWS][RES_TILE];
  __shared__ int s_flat[RES_TILE];
  __shared__ double wred[BC][2][RES_TILE / 32];
  __shared__ int six[BC][PAS_MAX_LAYERS], siy[BC][PAS_MAX_LAYERS];
  __shared__ float sfx[BC][PAS_MAX_LAYERS], sfy[BC][PAS_MAX_LAYERS];
  __shared__ int s_L[BC];
  const int tid = threadIdx.x;
  const T* MT = nullptr;
  if constexpr (sizeof(T) == 4) MT = a.MT;
  else MT = a.MTb;
  const int n_m = a.n_m;
  const int col = tid % COLS, row = tid / COLS;
  const int tile = blockIdx.y, b0 = blockIdx.x * BC;
  const int nb = min(BC, a.B - b0);
  const T* blk = MT + (size_t)tile * n_m * RES_TILE + col * VEC;
  uint4 v[RB_U];
#pragma unroll
  for (int u = 0; u < RB_U; ++u) {
    const int m = row + ROWS * u;
    v[u] = m < n_m ? ld_stream16(blk + (size_t)m * RES_TILE) : make_uint4(0u, 0u, 0u, 0u);
  }
  const int base = tile * RES_TILE;
  if (tid < RES_TILE) s_flat[tid] = base + tid < a.n_pix ? a.pix[base + tid] : 0;
  pdl_trigger();
  pdl_wait();  // the gathered commands
  const int Lmax = a.Lmax;
  for (int t = tid; t < BC * PAS_MAX_LAYERS; t += RES_THREADS) {
    const int b = t / PAS_MAX_LAYERS, l = t - b * PAS_MAX_LAYERS;
    if (b < nb) {
      const AtmoArgs& at = a.loops[b0 + b].atmo;
      if (l == 0) s_L[b] = at.L;
      if (l < at.L) {
        const long long step = *a.loops[b0 + b].d_step;
        layer_shift(at.vx[l], at.ox[l], step, at.S, &six[b][l], &sfx[b][l]);
        layer_shift(at.vy[l], at.oy[l], step, at.S, &siy[b][l], &sfy[b][l]);
      }
    }
  }
  __syncthreads();
  for (int t = tid; t < nb * Lmax * RES_TILE; t += RES_THREADS) {
    const int bl = t / RES_TILE, q = t - bl * RES_TILE;
    const int b = bl / Lmax, l = bl - b * Lmax;
    if (l < s_L[b] && base + q < a.n_pix) {
      const AtmoArgs& at = a.loops[b0 + b].atmo;
      const int flat = s_flat[q];
      const int i = flat / at.Np, j = flat - i * at.Np;
      size_t o[4];
      tap_offsets(i, j, six[b][l], siy[b][l], at.S, o);
      const float* sc = at.screens + (size_t)l * at.S * at.S;
#pragma unroll
      for (int k = 0; k < 4; ++k) cp_async4(taps + ((b * Lmax + l) * 4 + k) * RES_TILE + q, sc + o[k]);
    }
  }
  cp_async_commit();
  float acc[BC][VEC];
#pragma unroll
  for (int b = 0; b < BC; ++b)
#pragma unroll
    for (int i = 0; i < VEC; ++i) acc[b][i] = 0.f;
  const float* cg = a.cmdg + b0;
  for (int mb = row; mb < n_m; mb += ROWS * RB_U) {
#pragma unroll
    for (int u = 0; u < RB_U; ++u) {
      const int m = mb + ROWS * u;
      if (m < n_m) {
        float cm[BC];
#pragma unroll
        for (int k = 0; k < BC / 4; ++k) {
          const float4 c4 = __ldg(reinterpret_cast<const float4*>(cg + (size_t)m * a.Bp) + k);
          cm[4 * k] = c4.x;
          cm[4 * k + 1] = c4.y;
          cm[4 * k + 2] = c4.z;
          cm[4 * k + 3] = c4.w;
        }
        float f[VEC];
        unpack16<T>(v[u], f);
#pragma unroll
        for (int b = 0; b < BC; ++b)
#pragma unroll
          for (int i = 0; i < VEC; ++i) acc[b][i] = fmaf(cm[b], f[i], acc[b][i]);
      }
      const int mn = m + ROWS * RB_U;
      if (mn < n_m) v[u] = ld_stream16(blk + (size_t)mn * RES_TILE);
    }
  }
#pragma unroll
  for (int b = 0; b < BC; ++b)
#pragma unroll
    for (int i = 0; i < VEC; ++i) red[b][row][col * VEC + i] = acc[b][i];
  cp_async_wait_all();
  __syncthreads();
  for (int t = tid; t < nb * Lmax * RES_TILE; t += RES_THREADS) {
    const int bl = t / RES_TILE, q = t - bl * RES_TILE;
    const int b = bl / Lmax, l = bl - b * Lmax;
    if (l < s_L[b] && base + q < a.n_pix) {
      float* tp = taps + (b * Lmax + l) * 4 * RES_TILE + q;
      tp[0] = bilinear(sfx[b][l], sfy[b][l], tp[0], tp[RES_TILE], tp[2 * RES_TILE], tp[3 * RES_TILE]);
    }
  }
  __syncthreads();
  // output: thread t of a round takes loop t / RES_TILE, pixel t % RES_TILE (the
  // warps of one loop's tile in the order of residual_kernel's output warps)
  constexpr int PER_ROUND = RES_THREADS / RES_TILE;
  for (int r0 = 0; r0 < BC; r0 += PER_ROUND) {
    const int b = r0 + tid / RES_TILE, px = tid % RES_TILE;
    const int p = base + px;
    float s1 = 0.f, s2 = 0.f;
    if (b < nb && p < a.n_pix) {
      const ResBatchLoop& L = a.loops[b0 + b];
      const int flat = s_flat[px];
      float atm = 0.f;
      for (int l = 0; l < s_L[b]; ++l) atm = __fadd_rn(atm, taps[(b * Lmax + l) * 4 * RES_TILE + px]);
      float dm = 0.f;
#pragma unroll
      for (int r = 0; r < ROWS; ++r) dm += red[b][r][px];
      const float rr = atm - dm;
      L.out[flat] = rr;
      s1 = rr;
      s2 = rr * rr;
    }
    const int w = px >> 5, lane = tid & 31;
    float f1 = s1, f2 = s2;
    for (int o = 16; o > 0; o >>= 1) {
      f1 += __shfl_down_sync(0xffffffffu, f1, o);
      f2 += __shfl_down_sync(0xffffffffu, f2, o);
    }
    if (lane == 0 && b < BC) {
      wred[b][0][w] = f1;
      wred[b][1][w] = f2;
    }
  }
  __syncthreads();
  if (tid < nb) {
    const ResBatchLoop& L = a.loops[b0 + tid];
    if (L.wfe_part) {
      double t1 = 0.0, t2 = 0.0;
      for (int w = 0; w < RES_TILE / 32; ++w) {
        t1 += wred[tid][0][w];
        t2 += wred[tid][1][w];
      }
      L.wfe_part[tile] = make_double2(t1, t2);
    }
  }
}

struct ResBatch {
  pas_ctx_t ctx = nullptr;
  ResBatchArgs args{};
  ResBatchLoop* d_loops = nullptr;
  float* d_cmdg = nullptr;
  int chunks = 0, tiles = 0;
  size_t smem = 0;
  bool bf16 = false;
};

void res_batch_destroy(ResBatch* r) {
  if (!r) return;
  dev_free(r->d_loops);
  dev_free(r->d_cmdg);
  delete r;
}

bool res_batch_ok(const AtmoArgs& atmo) { return !atmo.cone && atmo.L >= 0 && atmo.L <= PAS_MAX_LAYERS; }

pas_status res_batch_create(pas_ctx_t ctx, pas_dm_t dm, int B, const ResBatchLoop* loops, ResBatch** out) {
  *out = nullptr;
  PAS_CHECK_ARG(ctx, dm && B >= 1, "batched residual: a DM and at least one loop");
  int Lmax = 0;
  for (int b = 0; b < B; ++b) {
    PAS_CHECK_ARG(ctx, res_batch_ok(loops[b].atmo), "batched residual: on-axis or off-axis sources at infinity");
    PAS_CHECK_ARG(ctx, loops[b].atmo.L == 0 || loops[b].atmo.Np == dm->Np, "batched residual: pupil sizes differ");
    PAS_CHECK_ARG(ctx, loops[b].cmd_ring && loops[b].d_step && loops[b].out && loops[b].delay >= 1,
                  "batched residual: loop buffers");
    Lmax = std::max(Lmax, loops[b].atmo.L);
  }
  ResBatch* r = new ResBatch();
  r->ctx = ctx;
  r->bf16 = dm->d_MTb != nullptr;
  const int BC = r->bf16 ? res_batch_bc<__nv_bfloat16>() : res_batch_bc<float>();
  r->chunks = (B + BC - 1) / BC;
  r->tiles = residual_tiles(dm->n_pix);
  const int Bp = r->chunks * BC;
  pas_status st = dev_alloc(ctx, (void**)&r->d_loops, sizeof(ResBatchLoop) * B);
  if (st == PAS_OK) st = dev_alloc(ctx, (void**)&r->d_cmdg, sizeof(float) * (size_t)std::max(dm->n_modes, 1) * Bp);
  if (st != PAS_OK) {
    res_batch_destroy(r);
    return st;
  }
  cudaError_t e = cudaMemcpy(r->d_loops, loops, sizeof(ResBatchLoop) * B, cudaMemcpyHostToDevice);
  ResBatchArgs& a = r->args;
  a.MT = dm->d_MT;
  a.MTb = dm->d_MTb;
  a.pix = dm->d_pix;
  a.n_pix = dm->n_pix;
  a.n_m = dm->n_modes;
  a.loops = r->d_loops;
  a.B = B;
  a.Bp = Bp;
  a.cmdg = r->d_cmdg;
  a.Lmax = Lmax;
  r->smem = sizeof(float) * (size_t)BC * Lmax * 4 * RES_TILE;
  if (e == cudaSuccess)
    e = r->bf16 ? raise_dyn_smem((const void*)residual_batch_kernel<__nv_bfloat16>, r->smem)
                : raise_dyn_smem((const void*)residual_batch_kernel<float>, r->smem);
  if (e != cudaSuccess) {
    res_batch_destroy(r);
    return set_error(ctx, PAS_ECUDA, "batched residual: %s", cudaGetErrorString(e));
  }
  *out = r;
  return PAS_OK;
}

pas_status res_batch_launch(ResBatch* r, cudaStream_t st) {
  if (r->tiles == 0) return PAS_OK;
  const ResBatchArgs& a = r->args;
  const int tot = std::max(a.n_m, 1) * a.Bp;
  cudaError_t e = launch_k(gather_cmds_kernel, dim3(std::min(1024, (tot + 255) / 256)), dim3(256), 0, st, false,
                           (const ResBatchLoop*)a.loops, a.B, a.Bp, a.n_m, r->d_cmdg);
  if (e == cudaSuccess) {
    const dim3 grid(r->chunks, r->tiles);
    e = r->bf16 ? launch_k(residual_batch_kernel<__nv_bfloat16>, grid, dim3(RES_THREADS), r->smem, st, true, a)
                : launch_k(residual_batch_kernel<float>, grid, dim3(RES_THREADS), r->smem, st, true, a);
  }
  if (e != cudaSuccess) return set_error(r->ctx, PAS_ECUDA, "batched residual launch: %s", cudaGetErrorString(e));
  return PAS_OK;
}

}  // namespace pas

// ------------------------------------------------------------------ objects

extern "C" {

pas_status pas_atmo_create(pas_ctx_t ctx, const pas_atmo_params* p, const float* d_screens,
                           pas_atmo_t* out) {
  if (!ctx || !p || !d_screens || !out) return pas::set_global_error(PAS_EINVAL, "pas_atmo_create: NULL argument");
  *out = nullptr;
  PAS_CHECK_ARG(ctx, p->n_layers >= 1 && p->n_layers <= PAS_MAX_LAYERS, "pas_atmo_create: 1..16 layers");
  PAS_CHECK_ARG(ctx, p->Np > 0 && p->S >= p->Np + 2, "pas_atmo_create: need S >= Np + 2");
  PAS_CHECK_ARG(ctx, p->vx && p->vy, "pas_atmo_create: NULL velocity arrays");
  pas_atmo_t a = new pas_atmo_s();
  a->ctx = ctx;
  a->args.screens = d_screens;
  a->args.L = p->n_layers;
  a->args.S = p->S;
  a->args.Np = p->Np;
  for (int l = 0; l < PAS_MAX_LAYERS; ++l) {
    a->args.vx[l] = l < p->n_layers ? p->vx[l] : 0.0;
    a->args.vy[l] = l < p->n_layers ? p->vy[l] : 0.0;
  }
  pas_status st = pas::dev_alloc(ctx, (void**)&a->d_err, sizeof(unsigned int));
  if (st != PAS_OK) {
    delete a;
    return st;
  }
  a->owns_err = true;
  cudaError_t e = cudaMemset(a->d_err, 0, sizeof(unsigned int));
  if (e != cudaSuccess) {
    pas_atmo_destroy(a);
    return pas::set_error(ctx, PAS_ECUDA, "pas_atmo_create: %s", cudaGetErrorString(e));
  }
  // the screens as [L][S][S] floats for two-row boxes of the tap staging: a row pitch
  // of whole 16-byte units, a box no wider than a row, a 16-byte aligned start
  if (p->S % 4 == 0 && p->S >= pas::RES_BOX && (reinterpret_cast<uintptr_t>(d_screens) & 15) == 0)
    a->tma = pas::make_tmap_rows_f32(&a->tmap, d_screens, (uint64_t)p->S, (uint64_t)p->n_layers,
                                     (uint32_t)pas::RES_BOX);
  *out = a;
  return PAS_OK;
}

pas_status pas_atmo_advance(pas_atmo_t a, int64_t step, float* d_opd) {
  if (!a || !d_opd) return pas::set_global_error(PAS_EINVAL, "pas_atmo_advance: NULL argument");
  PAS_CHECK_ARG(a->ctx, step >= 0, "pas_atmo_advance: negative step");
  const int n = a->args.Np * a->args.Np;
  const int blocks = std::min((n + 255) / 256, 4 * std::max(a->ctx->sm_count, 1));
  pas::atmo_kernel<<<blocks, 256, 0, a->ctx->stream>>>(a->args, nullptr, step, d_opd);
  return pas::check_launch(a->ctx, "pas_atmo_advance launch");
}

pas_status pas_atmo_create_cone_view(pas_atmo_t base, const double* h_ox, const double* h_oy,
                                     const double* h_scale, pas_atmo_t* out) {
  if (!base || !h_ox || !h_oy || !out) return pas::set_global_error(PAS_EINVAL, "pas_atmo_create_view: NULL argument");
  *out = nullptr;
  for (int l = 0; l < base->args.L; ++l) {
    PAS_CHECK_ARG(base->ctx, std::isfinite(h_ox[l]) && std::isfinite(h_oy[l]), "pas_atmo_create_view: offsets not finite");
    if (h_scale)
      PAS_CHECK_ARG(base->ctx, h_scale[l] > 0.0 && h_scale[l] <= 1.0, "pas_atmo_create_cone_view: scales in (0, 1]");
  }
  pas_atmo_t a = new pas_atmo_s(*base);
  a->owns_err = false;  // the base's error word
  a->args.cone = 0;
  for (int l = 0; l < PAS_MAX_LAYERS; ++l) {
    // the view's pupil position p maps to c + (p - c) s_base + o_base in the base
    const double sb = base->args.sc[l];
    const bool in = l < base->args.L;
    a->args.ox[l] = in ? base->args.ox[l] + sb * h_ox[l] : 0.0;
    a->args.oy[l] = in ? base->args.oy[l] + sb * h_oy[l] : 0.0;
    a->args.sc[l] = in ? sb * (h_scale ? h_scale[l] : 1.0) : 1.0;
    if (a->args.sc[l] != 1.0) a->args.cone = 1;
  }
  *out = a;
  return PAS_OK;
}

pas_status pas_atmo_create_view(pas_atmo_t base, const double* h_ox, const double* h_oy, pas_atmo_t* out) {
  return pas_atmo_create_cone_view(base, h_ox, h_oy, nullptr, out);
}

void pas_atmo_destroy(pas_atmo_t a) {
  if (!a) return;
  if (a->owns_err) pas::dev_free(a->d_err);
  delete a;
}

int32_t pas_atmo_tma(pas_atmo_t a) { return a ? (a->tma && !a->args.cone ? 1 : 0) : -1; }

pas_status pas_atmo_set_tap_staging(pas_atmo_t a, int32_t mode) {
  if (!a) return pas::set_global_error(PAS_EINVAL, "pas_atmo_set_tap_staging: NULL atmosphere");
  PAS_CHECK_ARG(a->ctx, mode == PAS_TAPS_AUTO || mode == PAS_TAPS_TMA || mode == PAS_TAPS_COPY,
                "pas_atmo_set_tap_staging: mode PAS_TAPS_AUTO, PAS_TAPS_TMA or PAS_TAPS_COPY");
  PAS_CHECK_ARG(a->ctx, mode != PAS_TAPS_TMA || pas_atmo_tma(a) == 1,
                "pas_atmo_set_tap_staging: these screens or this source do not allow TMA staging");
  a->taps = mode;
  return PAS_OK;
}

pas_status pas_atmo_set_wait_limit(pas_atmo_t a, uint32_t tries) {
  if (!a) return pas::set_global_error(PAS_EINVAL, "pas_atmo_set_wait_limit: NULL atmosphere");
  a->wait_limit = tries;
  return PAS_OK;
}

pas_status pas_atmo_check(pas_atmo_t a, uint32_t* h_fault) {
  if (!a) return pas::set_global_error(PAS_EINVAL, "pas_atmo_check: NULL atmosphere");
  unsigned int f = 0;
  PAS_CUDA_TRY(a->ctx, cudaMemcpy(&f, a->d_err, sizeof(f), cudaMemcpyDeviceToHost));
  if (f) PAS_CUDA_TRY(a->ctx, cudaMemset(a->d_err, 0, sizeof(unsigned int)));
  if (h_fault) *h_fault = f;
  if (f) return pas::set_error(a->ctx, PAS_ETIMEOUT, "atmosphere tap staging: a wait gave up (%u)", f);
  return PAS_OK;
}

void pas_dm_destroy(pas_dm_t d) {
  if (!d) return;
  pas::dev_free(d->d_MT);
  pas::dev_free(d->d_MTb);
  pas::dev_free(d->d_pix);
  pas::dev_free(d->d_seg);
  delete d;
}

pas_status pas_dm_create(pas_ctx_t ctx, const float* h_M, int32_t n_pix, int32_t n_modes, int32_t Np,
                         double obs, pas_precision prec, pas_dm_t* out) {
  if (!ctx || !h_M || !out) return pas::set_global_error(PAS_EINVAL, "pas_dm_create: NULL argument");
  *out = nullptr;
  PAS_CHECK_ARG(ctx, n_modes >= 1 && Np > 0, "pas_dm_create: bad sizes");
  PAS_CHECK_ARG(ctx, prec == PAS_FP32 || prec == PAS_BF16, "pas_dm_create: precision PAS_FP32 or PAS_BF16");
  int32_t npx = 0;
  if (pas_pupil_pixels(Np, obs, nullptr, 0, &npx) != PAS_OK || npx != n_pix)
    return pas::set_error(ctx, PAS_EINVAL, "pas_dm_create: n_pix=%d does not match the pupil (%d)", n_pix, npx);
  std::vector<int32_t> pix(n_pix);
  pas_pupil_pixels(Np, obs, pix.data(), n_pix, &npx);
  pas_dm_t d = new pas_dm_s();
  d->ctx = ctx;
  d->n_pix = n_pix;
  d->n_modes = n_modes;
  d->Np = Np;
  // tiled layout: tile t (RES_TILE pixels) holds [n_modes][RES_TILE] contiguously
  const int tiles = pas::residual_tiles(n_pix);
  d->n_pad = tiles * pas::RES_TILE;
  d->T_obs = pas::obstruction_threshold(Np, obs);
  std::vector<float> MT((size_t)n_modes * d->n_pad, 0.f);
  for (int p = 0; p < n_pix; ++p) {
    const int t = p / pas::RES_TILE, pl = p % pas::RES_TILE;
    for (int m = 0; m < n_modes; ++m)
      MT[((size_t)t * n_modes + m) * pas::RES_TILE + pl] = h_M[(size_t)p * n_modes + m];
  }
  d->prec = prec;
  pas_status st = PAS_OK;
  cudaError_t e = cudaSuccess;
  if (prec == PAS_BF16) {
    // round to nearest even; the pad pixels stay zero
    std::vector<__nv_bfloat16> MTb(MT.size());
    for (size_t i = 0; i < MT.size(); ++i) MTb[i] = __float2bfloat16_rn(MT[i]);
    st = pas::dev_alloc(ctx, (void**)&d->d_MTb, sizeof(__nv_bfloat16) * MTb.size());
    if (st == PAS_OK) st = pas::dev_alloc(ctx, (void**)&d->d_pix, sizeof(int32_t) * n_pix);
    if (st != PAS_OK) {
      pas_dm_destroy(d);
      return st;
    }
    e = cudaMemcpy(d->d_MTb, MTb.data(), sizeof(__nv_bfloat16) * MTb.size(), cudaMemcpyHostToDevice);
  } else {
    st = pas::dev_alloc(ctx, (void**)&d->d_MT, sizeof(float) * MT.size());
    if (st == PAS_OK) st = pas::dev_alloc(ctx, (void**)&d->d_pix, sizeof(int32_t) * n_pix);
    if (st != PAS_OK) {
      pas_dm_destroy(d);
      return st;
    }
    e = cudaMemcpy(d->d_MT, MT.data(), sizeof(float) * MT.size(), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMemcpy(d->d_pix, pix.data(), sizeof(int32_t) * n_pix, cudaMemcpyHostToDevice);
  // each tile's runs of consecutive pixels of one pupil row (the TMA tap staging's
  // segments); a tile with more than RES_SEG_MAX keeps the 4-byte copies for all
  std::vector<int4> seg;
  int smax = 0;
  for (int t = 0; t < tiles; ++t) {
    int ns = 0;
    for (int q = 0; q < pas::RES_TILE && t * pas::RES_TILE + q < n_pix; ++q) {
      const int f = pix[t * pas::RES_TILE + q], i = f / Np, j = f - i * Np;
      if (q > 0) {
        const int g = pix[t * pas::RES_TILE + q - 1];
        if (g / Np == i && g - (g / Np) * Np == j - 1) continue;
      }
      ++ns;
    }
    smax = std::max(smax, ns);
  }
  if (e == cudaSuccess && smax >= 1 && smax <= pas::RES_SEG_MAX) {
    seg.assign((size_t)tiles * smax, make_int4(0, 0, 0, 0));
    for (int t = 0; t < tiles; ++t) {
      int ns = -1;
      for (int q = 0; q < pas::RES_TILE && t * pas::RES_TILE + q < n_pix; ++q) {
        const int f = pix[t * pas::RES_TILE + q], i = f / Np, j = f - i * Np;
        bool cont = false;
        if (q > 0) {
          const int g = pix[t * pas::RES_TILE + q - 1];
          cont = g / Np == i && g - (g / Np) * Np == j - 1;
        }
        if (!cont) seg[(size_t)t * smax + ++ns] = make_int4(i, j, 0, q);
        seg[(size_t)t * smax + ns].z += 1;
      }
    }
    st = pas::dev_alloc(ctx, (void**)&d->d_seg, sizeof(int4) * seg.size());
    if (st != PAS_OK) {
      pas_dm_destroy(d);
      return st;
    }
    e = cudaMemcpy(d->d_seg, seg.data(), sizeof(int4) * seg.size(), cudaMemcpyHostToDevice);
    d->seg_max = smax;
  }
  if (e != cudaSuccess) {
    pas_dm_destroy(d);
    return pas::set_error(ctx, PAS_ECUDA, "pas_dm_create: %s", cudaGetErrorString(e));
  }
  *out = d;
  return PAS_OK;
}

pas_status pas_dm_update(pas_dm_t d, const float* d_dmodes, const float* d_gain, float* d_cmd,
                         float* d_opd_dm) {
  if (!d || !d_cmd) return pas::set_global_error(PAS_EINVAL, "pas_dm_update: NULL argument");
  cudaStream_t st = d->ctx->stream;
  if (d_dmodes) {
    pas::integrate_kernel<<<(d->n_modes + 255) / 256, 256, 0, st>>>(d_cmd, d_dmodes, d_gain, d->n_modes);
    pas_status s = pas::check_launch(d->ctx, "pas_dm_update integrate launch");
    if (s != PAS_OK) return s;
  }
  if (d_opd_dm) {
    pas::ResArgs a = pas::make_res_args(d);
    a.cmd = d_cmd;
    a.out = d_opd_dm;
    a.dm_sign = -1.0f;  // out = 0 - (-1) M c = M c
    pas::zero_outside_kernel<<<(d->Np * d->Np + 255) / 256, 256, 0, st>>>(d_opd_dm, d->Np, d->T_obs);
    return pas::residual_launch(d->ctx, a, st);
  }
  return PAS_OK;
}

pas_status pas_dm_residual(pas_dm_t d, const float* d_opd_atm, const float* d_cmd, float* d_opd_res) {
  if (!d || !d_opd_atm || !d_cmd || !d_opd_res)
    return pas::set_global_error(PAS_EINVAL, "pas_dm_residual: NULL argument");
  cudaStream_t st = d->ctx->stream;
  pas::ResArgs a = pas::make_res_args(d);
  a.opd_atm = d_opd_atm;
  a.cmd = d_cmd;
  a.out = d_opd_res;
  a.dm_sign = 1.0f;
  pas_status s = pas::residual_launch(d->ctx, a, st);
  if (s != PAS_OK) return s;
  pas::zero_outside_kernel<<<(d->Np * d->Np + 255) / 256, 256, 0, st>>>(d_opd_res, d->Np, d->T_obs);
  return pas::check_launch(d->ctx, "pas_dm_residual zero launch");
}

pas_status pas_dm_project(pas_dm_t d, const float* d_opd, float* d_coeffs) {
  if (!d || !d_opd || !d_coeffs) return pas::set_global_error(PAS_EINVAL, "pas_dm_project: NULL argument");
  return pas::dm_project_launch(d, d_opd, d_coeffs, d->ctx->stream);
}

}  // extern "C"
