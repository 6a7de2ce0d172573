// Learned nonlinear reconstructor: a multilayer perceptron from standardised
// slopes to modal coefficients, z_l = W_l h_{l-1} + b_l, h_l = gelu(z_l) on the
// hidden layers, a linear output layer; trained with the mean squared error of
// the coefficients and Adam. The paper's reconstructor is the linear modal one
// (Table 1 modalrec); this object is an extension that the loop can use instead.
//
// Training runs on the tensor cores: every product of a training step is one
// BF16 GEMM C = A B^T with both operands K-major (gemm.cuh, tcgen05 + TMA), which
// is why the object keeps transposed copies of the activations (H^T), the output
// gradients (dZ^T) and the weights (W^T): forward Z = X W^T, input gradient
// dH = dZ W = dZ (W^T)^T, weight gradient dW = dZ^T H = (dZ^T)(H^T)^T. The
// epilogues fuse bias, GELU, GELU' and the transposed copies. Master weights and
// Adam moments are float32; the GEMM operands are bf16 with float32 accumulation.
//
// Inference inside the loop (one slope vector per step) is a chain of bf16
// matrix-vector products on CUDA cores, each layer a kernel that follows its
// predecessor programmatically; the last layer applies the loop's integrator.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "atmo_dm.cuh"
#include "gemm.cuh"
#include "internal.h"
#include "mlp.cuh"
#include "pdl.cuh"
#include "pyr.cuh"

namespace pas {

// ---------------------------------------------------------------- GEMM host side

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

bool make_tmap_bf16(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint64_t ld,
                    uint32_t box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || !base || rows == 0 || cols == 0 || (ld * 2) % 16 != 0 || ld < cols ||
      (reinterpret_cast<uintptr_t>(base) & 15) != 0)
    return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {ld * 2};
  cuuint32_t box[2] = {64, box_rows};
  cuuint32_t es[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_tmap_rows_f32(CUtensorMap* map, const float* base, uint64_t S, uint64_t L, uint32_t box) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || !base || S < 2 || L == 0 || (S * 4) % 16 != 0 || box > S || (box * 4) % 16 != 0 ||
      (reinterpret_cast<uintptr_t>(base) & 15) != 0)
    return false;
  cuuint64_t dims[3] = {S, S, L};
  cuuint64_t strides[2] = {S * 4, S * S * 4};
  cuuint32_t boxd[3] = {box, 2, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, boxd, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int gemm_pick_bn(int M, int N, int sms) {
  const int tm = (M + 127) / 128;
  int best = 128;
  long best_cost = -1;
  for (int bn : {256, 128, 64}) {
    const long ctas = (long)tm * ((N + bn - 1) / bn);
    const long waves = (ctas + sms - 1) / sms;
    const long cost = waves * (bn + 48);  // per-tile cost ~ MMA columns + a fixed prologue/epilogue share
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = bn;
    }
  }
  return best;
}

bool gemm_prepare(GemmOp* op, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
                  int sms) {
  op->M = M;
  op->N = N;
  op->K = K;
  op->bn = gemm_pick_bn(M, N, sms);
  // at least two tiles per SM: persistent CTAs, the epilogue of one tile under the
  // products of the next
  gemm_set_persist(op, sms);
  return make_tmap_bf16(&op->a, A, (uint64_t)M, (uint64_t)K, (uint64_t)lda, 128) &&
         make_tmap_bf16(&op->b, B, (uint64_t)N, (uint64_t)K, (uint64_t)ldb, (uint32_t)op->bn);
}

// ---------------------------------------------------------------- epilogues

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

__device__ __forceinline__ uint4 pack8_bf16(const float* v) {
  uint4 u;
  __nv_bfloat162 h[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
  memcpy(&u, h, 16);
  return u;
}

// C[row][col] = acc (float32)
struct EpiF32 {
  float* C;
  int ldc, N;
  __device__ void store(int row, int col, const float (&v)[16]) const {
    float* c = C + (size_t)row * ldc + col;
    if (col + 16 <= N && (reinterpret_cast<uintptr_t>(c) & 15) == 0) {
#pragma unroll
      for (int j = 0; j < 16; j += 4) *reinterpret_cast<float4*>(c + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
    } else {
      for (int j = 0; j < 16 && col + j < N; ++j) c[j] = v[j];
    }
  }
};

// hidden layer: z = acc + b; Z = z (float32), H = gelu(z) and H^T (bf16)
struct EpiHidden {
  const float* bias;
  float* Z;
  __nv_bfloat16* H;
  __nv_bfloat16* Ht;
  int ld, ldt, N;
  __device__ void store(int row, int col, const float (&v)[16]) const {
    float z[16], h[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      z[j] = v[j] + (col + j < N ? bias[col + j] : 0.f);
      h[j] = gelu_f(z[j]);
    }
    float* zr = Z + (size_t)row * ld + col;
    __nv_bfloat16* hr = H + (size_t)row * ld + col;
    if (col + 16 <= N) {
#pragma unroll
      for (int j = 0; j < 16; j += 4) *reinterpret_cast<float4*>(zr + j) = make_float4(z[j], z[j + 1], z[j + 2], z[j + 3]);
      *reinterpret_cast<uint4*>(hr) = pack8_bf16(h);
      *reinterpret_cast<uint4*>(hr + 8) = pack8_bf16(h + 8);
#pragma unroll
      for (int j = 0; j < 16; ++j) Ht[(size_t)(col + j) * ldt + row] = __float2bfloat16_rn(h[j]);
    } else {
      for (int j = 0; j < 16 && col + j < N; ++j) {
        zr[j] = z[j];
        hr[j] = __float2bfloat16_rn(h[j]);
        Ht[(size_t)(col + j) * ldt + row] = __float2bfloat16_rn(h[j]);
      }
    }
  }
};

// output layer: out = acc + b (float32)
struct EpiOut {
  const float* bias;
  float* out;
  int ld, N;
  __device__ void store(int row, int col, const float (&v)[16]) const {
    float* o = out + (size_t)row * ld + col;
    for (int j = 0; j < 16 && col + j < N; ++j) o[j] = v[j] + bias[col + j];
  }
};

// input gradient of a hidden layer: dz = acc * gelu'(z); dZ and dZ^T (bf16)
struct EpiBack {
  const float* Z;
  __nv_bfloat16* dZ;
  __nv_bfloat16* dZt;
  int ld, ldt, N;
  __device__ void store(int row, int col, const float (&v)[16]) const {
    const float* zr = Z + (size_t)row * ld + col;
    __nv_bfloat16* gr = dZ + (size_t)row * ld + col;
    float g[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) g[j] = col + j < N ? v[j] * gelu_grad_f(zr[j]) : 0.f;
    if (col + 16 <= N) {
      *reinterpret_cast<uint4*>(gr) = pack8_bf16(g);
      *reinterpret_cast<uint4*>(gr + 8) = pack8_bf16(g + 8);
#pragma unroll
      for (int j = 0; j < 16; ++j) dZt[(size_t)(col + j) * ldt + row] = __float2bfloat16_rn(g[j]);
    } else {
      for (int j = 0; j < 16 && col + j < N; ++j) {
        gr[j] = __float2bfloat16_rn(g[j]);
        dZt[(size_t)(col + j) * ldt + row] = __float2bfloat16_rn(g[j]);
      }
    }
  }
};

// ---------------------------------------------------------------- element kernels

constexpr unsigned MLP_ERR_INDEX = 16u;

// X[b][i] = (S[idx[b]][i] - mean[i]) * istd[i] in bf16, and X^T; 32 x 32 tiles.
__global__ void mlp_input_kernel(const float* S, int n_data, const int* idx, const int* iter, int B, int n_in,
                                 const float* mean, const float* istd, __nv_bfloat16* X, int ldx,
                                 __nv_bfloat16* Xt, int ldt, unsigned* err) {
  __shared__ float tile[32][33];
  pdl_trigger();
  pdl_wait();
  const int i0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
  const int* id = idx ? idx + (size_t)(*iter) * B : nullptr;
  const int tx = threadIdx.x;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int b = b0 + r, i = i0 + tx;
    float x = 0.f;
    if (b < B && i < n_in) {
      int sb = id ? id[b] : b;
      if (sb < 0 || sb >= n_data) {
        atomicOr(err, MLP_ERR_INDEX);
        sb = 0;
      }
      x = (S[(size_t)sb * n_in + i] - mean[i]) * istd[i];
      X[(size_t)b * ldx + i] = __float2bfloat16_rn(x);
    }
    tile[r][tx] = x;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = i0 + r, b = b0 + tx;
    if (i < n_in && b < B) Xt[(size_t)i * ldt + b] = __float2bfloat16_rn(tile[tx][r]);
  }
}

// The same for B vectors given by pointer (the slopes of a batch's loops):
// X[b][i] = (S_b[i] - mean[i]) * istd[i] in bf16, and X^T.
__global__ void mlp_gather_input_kernel(const float* const* S, int B, int n_in, const float* mean,
                                        const float* istd, __nv_bfloat16* X, int ldx, __nv_bfloat16* Xt, int ldt) {
  __shared__ float tile[32][33];
  const int i0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
  const int tx = threadIdx.x;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int b = b0 + r, i = i0 + tx;
    float x = 0.f;
    if (b < B && i < n_in) {
      x = (S[b][i] - mean[i]) * istd[i];
      X[(size_t)b * ldx + i] = __float2bfloat16_rn(x);
    }
    tile[r][tx] = x;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = i0 + r, b = b0 + tx;
    if (i < n_in && b < B) Xt[(size_t)i * ldt + b] = __float2bfloat16_rn(tile[tx][r]);
  }
}

// dZ = 2 (out - y) / (B n_out) (bf16, and dZ^T); loss = mean (out - y)^2 into
// loss[*iter], summed in a fixed order by the last CTA.
__global__ void mlp_loss_kernel(const float* out, int ldo, const float* Y, int n_data, const int* idx,
                                const int* iter, int B, int n_out, __nv_bfloat16* dZ, int ldz, __nv_bfloat16* dZt,
                                int ldt, float* part, unsigned* done, float* loss) {
  __shared__ float tile[32][33];
  __shared__ float red[8];
  __shared__ bool is_last;
  pdl_trigger();
  pdl_wait();
  const int o0 = blockIdx.x * 32, b0 = blockIdx.y * 32, tx = threadIdx.x;
  const int* id = idx ? idx + (size_t)(*iter) * B : nullptr;
  const float gs = 2.0f / ((float)B * (float)n_out);
  float acc = 0.f;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int b = b0 + r, o = o0 + tx;
    float g = 0.f;
    if (b < B && o < n_out) {
      int sb = id ? id[b] : b;
      if (sb < 0 || sb >= n_data) sb = 0;  // reported by the input kernel
      const float d = out[(size_t)b * ldo + o] - Y[(size_t)sb * n_out + o];
      acc = fmaf(d, d, acc);
      g = gs * d;
      dZ[(size_t)b * ldz + o] = __float2bfloat16_rn(g);
    }
    tile[r][tx] = g;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int o = o0 + r, b = b0 + tx;
    if (o < n_out && b < B) dZt[(size_t)o * ldt + b] = __float2bfloat16_rn(tile[tx][r]);
  }
  for (int s = 16; s > 0; s >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, s);
  const int w = (threadIdx.y * 32 + tx) >> 5;
  if ((tx & 31) == 0) red[w] = acc;
  __syncthreads();
  const int nblk = gridDim.x * gridDim.y, bid = blockIdx.y * gridDim.x + blockIdx.x;
  if (threadIdx.y == 0 && tx == 0) {
    float t = 0.f;
    for (int i = 0; i < blockDim.y; ++i) t += red[i];
    part[bid] = t;
    __threadfence();
    is_last = atomicAdd(done, 1u) == (unsigned)nblk - 1;
  }
  __syncthreads();  // also orders the reads of red above before its reuse below
  if (is_last) {  // fixed-order reduction of the block partials by the whole last block
    __threadfence();
    const int tid = threadIdx.y * 32 + tx;
    float t = 0.f;
    for (int i = tid; i < nblk; i += 256) t += part[i];
    for (int s = 16; s > 0; s >>= 1) t += __shfl_down_sync(0xffffffffu, t, s);
    if ((tx & 31) == 0) red[tid >> 5] = t;
    __syncthreads();
    if (tid == 0) {
      float tot = 0.f;
      for (int i = 0; i < 8; ++i) tot += red[i];
      loss[*iter] = tot / ((float)B * (float)n_out);
      *done = 0u;
    }
  }
}

struct BiasGradArgs {
  const __nv_bfloat16* dZt[PAS_MLP_MAX_LAYERS];
  size_t offb[PAS_MLP_MAX_LAYERS];
  int start[PAS_MLP_MAX_LAYERS + 1];  // cumulative bias counts
  int L, ldt, B;
  float* g;
};

// db_l[o] = sum_b dZ_l[b][o]: one warp per bias element, reading a row of dZ^T.
__global__ void mlp_bias_grad_kernel(BiasGradArgs a) {
  pdl_trigger();
  pdl_wait();
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= a.start[a.L]) return;
  int l = 0;
  while (w >= a.start[l + 1]) ++l;
  const int o = w - a.start[l];
  const __nv_bfloat16* row = a.dZt[l] + (size_t)o * a.ldt;
  float s = 0.f;
  for (int b = lane; b < a.B; b += 32) s += __bfloat162float(row[b]);
  for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
  if (lane == 0) a.g[a.offb[l] + o] = s;
}

struct AdamArgs {
  float* p;
  float* m;
  float* v;
  const float* g;
  int L;
  int out[PAS_MLP_MAX_LAYERS], in[PAS_MLP_MAX_LAYERS];
  size_t offW[PAS_MLP_MAX_LAYERS], offb[PAS_MLP_MAX_LAYERS];
  __nv_bfloat16* W[PAS_MLP_MAX_LAYERS];
  __nv_bfloat16* Wt[PAS_MLP_MAX_LAYERS];
  int ldW[PAS_MLP_MAX_LAYERS], ldWt[PAS_MLP_MAX_LAYERS];
  int tile_start[PAS_MLP_MAX_LAYERS + 1];  // 32 x 32 weight tiles, cumulative
  int bias_start[PAS_MLP_MAX_LAYERS + 1];  // bias elements, cumulative
  int update;                               // 0: only refresh the bf16 copies
  const float* lr;                          // indexed by *iter
  const int* iter;
  long long* t;
  float b1, b2, eps;
  unsigned* done;
  int* iter_inc;                            // advanced by the last CTA (or null)
};

__device__ __forceinline__ float adam_one(const AdamArgs& a, size_t k, float lr, float c1, float c2) {
  const float g = a.g[k];
  const float m = a.b1 * a.m[k] + (1.f - a.b1) * g;
  const float v = a.b2 * a.v[k] + (1.f - a.b2) * g * g;
  a.m[k] = m;
  a.v[k] = v;
  const float p = a.p[k] - lr * (m / c1) / (sqrtf(v / c2) + a.eps);
  a.p[k] = p;
  return p;
}

// Adam over every parameter, then the bf16 weight copies W and W^T. Blocks
// [0, tile_start[L]) take 32 x 32 weight tiles, the rest 256 biases each.
__global__ void __launch_bounds__(256) mlp_adam_kernel(AdamArgs a) {
  __shared__ float tile[32][33];
  __shared__ bool is_last;
  pdl_trigger();
  pdl_wait();
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  float lr = 0.f, c1 = 1.f, c2 = 1.f;
  if (a.update) {
    const float t = (float)(*a.t + 1);
    lr = a.lr[*a.iter];
    c1 = 1.f - powf(a.b1, t);
    c2 = 1.f - powf(a.b2, t);
  }
  const int blk = blockIdx.x;
  if (blk < a.tile_start[a.L]) {
    int l = 0;
    while (blk >= a.tile_start[l + 1]) ++l;
    const int in = a.in[l], out = a.out[l];
    const int tiles_in = (in + 31) / 32, t = blk - a.tile_start[l];
    const int o0 = (t / tiles_in) * 32, i0 = (t % tiles_in) * 32;
    for (int r = ty; r < 32; r += 8) {
      const int o = o0 + r, i = i0 + tx;
      float p = 0.f;
      if (o < out && i < in) {
        const size_t k = a.offW[l] + (size_t)o * in + i;
        p = a.update ? adam_one(a, k, lr, c1, c2) : a.p[k];
        a.W[l][(size_t)o * a.ldW[l] + i] = __float2bfloat16_rn(p);
      }
      tile[r][tx] = p;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
      const int i = i0 + r, o = o0 + tx;
      if (i < in && o < out) a.Wt[l][(size_t)i * a.ldWt[l] + o] = __float2bfloat16_rn(tile[tx][r]);
    }
  } else if (a.update) {
    const int j = (blk - a.tile_start[a.L]) * 256 + tid;
    if (j < a.bias_start[a.L]) {
      int l = 0;
      while (j >= a.bias_start[l + 1]) ++l;
      adam_one(a, a.offb[l] + (j - a.bias_start[l]), lr, c1, c2);
    }
  }
  if (!a.update) return;
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    is_last = atomicAdd(a.done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (is_last && tid == 0) {
    *a.t += 1;
    if (a.iter_inc) *a.iter_inc += 1;
    *a.done = 0u;
  }
}

// ---------------------------------------------------------------- single-vector chain

struct GemvArgs {
  const __nv_bfloat16* W;
  int ld, n_in, n_out;
  const float* bias;
  const float* x;
  float* y;
  const float* mean;  // first layer: x = (x - mean) * istd
  const float* istd;
  int gelu;
  // last layer: the loop integrator (as the linear reconstructor's kernel)
  const float* gain;
  float* ring;
  int delay;
  const long long* step;
  float* cmd_last;
  long long* step_inc;
  unsigned* done;
  unsigned* fault;
};

constexpr int GEMV_ROWS = 8;  // one warp per output row

__global__ void __launch_bounds__(256) mlp_gemv_kernel(GemvArgs a) {
  extern __shared__ float4 xs4[];
  __shared__ bool is_last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int o = blockIdx.x * GEMV_ROWS + warp;
  pdl_trigger();
  {
    const int nrow = min(GEMV_ROWS, a.n_out - (int)blockIdx.x * GEMV_ROWS);
    const char* base = reinterpret_cast<const char*>(a.W + (size_t)blockIdx.x * GEMV_ROWS * a.ld);
    const int lines = (int)(((size_t)nrow * a.ld * 2 + 127) / 128);
    for (int t = threadIdx.x; t < lines; t += blockDim.x) prefetch_l2(base + (size_t)t * 128);
  }
  pdl_wait();
  float* xs = reinterpret_cast<float*>(xs4);
  for (int i = threadIdx.x; i < a.ld; i += blockDim.x) {
    float x = 0.f;
    if (i < a.n_in) {
      x = a.x[i];
      if (a.mean) x = (x - a.mean[i]) * a.istd[i];
    }
    xs[i] = x;
  }
  __syncthreads();
  float acc = 0.f;
  if (o < a.n_out) {
    const uint4* row = reinterpret_cast<const uint4*>(a.W + (size_t)o * a.ld);
    const int nc = a.ld / 8;
#pragma unroll 4
    for (int c = lane; c < nc; c += 32) {
      const uint4 u = __ldg(row + c);
      const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
      const float4 x0 = xs4[2 * c], x1 = xs4[2 * c + 1];
      float2 f = __bfloat1622float2(h[0]);
      acc = fmaf(f.x, x0.x, acc);
      acc = fmaf(f.y, x0.y, acc);
      f = __bfloat1622float2(h[1]);
      acc = fmaf(f.x, x0.z, acc);
      acc = fmaf(f.y, x0.w, acc);
      f = __bfloat1622float2(h[2]);
      acc = fmaf(f.x, x1.x, acc);
      acc = fmaf(f.y, x1.y, acc);
      f = __bfloat1622float2(h[3]);
      acc = fmaf(f.x, x1.z, acc);
      acc = fmaf(f.y, x1.w, acc);
    }
  }
  for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
  if (lane == 0 && o < a.n_out) {
    float z = acc + a.bias[o];
    if (a.gelu) z = gelu_f(z);
    if (a.ring) {
      if (!isfinite(z)) {  // a diverged network must not corrupt the command
        atomicOr(a.fault, 1u);
        z = 0.f;
      }
      const long long t = *a.step;
      const float prev = a.ring[(size_t)((t - 1 + a.delay) % a.delay) * a.n_out + o];
      const float c = fmaf(a.gain ? a.gain[o] : 1.0f, z, prev);
      a.ring[(size_t)(t % a.delay) * a.n_out + o] = c;
      if (a.cmd_last) a.cmd_last[o] = c;
    }
    if (a.y) a.y[o] = z;
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

static pas_status gemv_chain(pas_mlp_t m, const float* x, float* y, const ReconArgs* integ, cudaStream_t st,
                             bool pdl) {
  for (int l = 0; l < m->L; ++l) {
    GemvArgs g = {};
    g.W = m->d_W[l];
    g.ld = m->ld[l];
    g.n_in = m->sz[l];
    g.n_out = m->sz[l + 1];
    g.bias = m->d_p + m->offb[l];
    g.x = l == 0 ? x : m->d_vec[(l - 1) & 1];
    const bool last = l == m->L - 1;
    g.y = last ? y : m->d_vec[l & 1];
    if (l == 0) {
      g.mean = m->d_mean;
      g.istd = m->d_istd;
    }
    g.gelu = last ? 0 : 1;
    if (last && integ) {
      g.gain = integ->gain;
      g.ring = integ->ring;
      g.delay = integ->delay;
      g.step = integ->step;
      g.cmd_last = integ->cmd_last;
      g.step_inc = integ->step_inc;
      g.done = m->d_gemv_done;
      g.fault = m->d_fault;
    }
    const int grid = (g.n_out + GEMV_ROWS - 1) / GEMV_ROWS;
    cudaError_t e = launch_k(mlp_gemv_kernel, dim3(grid), dim3(256), sizeof(float) * (size_t)g.ld, st,
                             pdl || l > 0, g);
    if (e != cudaSuccess) return set_error(m->ctx, PAS_ECUDA, "MLP layer %d launch: %s", l, cudaGetErrorString(e));
  }
  return PAS_OK;
}

pas_status mlp_loop_launch(pas_mlp_t m, const ReconArgs& integ, cudaStream_t st, bool pdl) {
  return gemv_chain(m, integ.s, integ.dmodes, &integ, st, pdl);
}

// ---------------------------------------------------------------- batched passes

static pas_status gemm_err(pas_mlp_t m, const char* what, cudaError_t e) {
  return set_error(m->ctx, PAS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

static pas_status mlp_layers_enqueue(pas_mlp_t m, int B, cudaStream_t st);

// Forward pass on the samples S[idx[*iter * B + b]] (idx null: the first B rows).
static pas_status mlp_forward_enqueue(pas_mlp_t m, int B, const float* S, int n_data, const int* idx,
                                      const int* iter, cudaStream_t st) {
  const int n_in = m->sz[0];
  dim3 tb(32, 8);
  cudaError_t e = launch_k(mlp_input_kernel, dim3((n_in + 31) / 32, (B + 31) / 32), tb, 0, st, false, S, n_data, idx,
                           iter, B, n_in, (const float*)m->d_mean, (const float*)m->d_istd, m->d_X, m->ld[0], m->d_Xt,
                           m->ldb, m->d_err);
  if (e != cudaSuccess) return gemm_err(m, "MLP input", e);
  return mlp_layers_enqueue(m, B, st);
}

// The forward GEMMs on the standardised inputs already in d_X: d_out [B][ld out].
static pas_status mlp_layers_enqueue(pas_mlp_t m, int B, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < m->L; ++l) {
    const __nv_bfloat16* A = l == 0 ? m->d_X : m->d_H[l - 1];
    GemmOp op;
    if (!gemm_prepare(&op, A, m->ld[l], m->d_W[l], m->ld[l], B, m->sz[l + 1], m->sz[l], m->ctx->sm_count))
      return set_error(m->ctx, PAS_ECUDA, "MLP forward layer %d: tensor map rejected", l);
    if (l < m->L - 1) {
      EpiHidden ep{m->d_p + m->offb[l], m->d_Z[l], m->d_H[l], m->d_Ht[l], m->ld[l + 1], m->ldb, m->sz[l + 1]};
      e = gemm_launch(op, ep, st, m->d_err, true);
    } else {
      EpiOut ep{m->d_p + m->offb[l], m->d_out, m->ld[l + 1], m->sz[l + 1]};
      e = gemm_launch(op, ep, st, m->d_err, true);
    }
    if (e != cudaSuccess) return gemm_err(m, "MLP forward GEMM", e);
  }
  return PAS_OK;
}

// A split layer's partials [splits][B][n_out] summed in range order, plus the bias; a
// hidden layer then stores Z, H and H^T as EpiHidden does, the output layer out as EpiOut.
__global__ void mlp_split_finish_kernel(const float* part, int splits, int B, int n_out, const float* bias, int hidden,
                                        float* Z, __nv_bfloat16* H, __nv_bfloat16* Ht, int ld, int ldt, float* out) {
  const size_t tot = (size_t)B * n_out;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(t / n_out), o = (int)(t - (size_t)b * n_out);
    float acc = 0.f;
    for (int z = 0; z < splits; ++z) acc += part[((size_t)z * B + b) * n_out + o];
    const float zv = acc + bias[o];
    if (hidden) {
      const float h = gelu_f(zv);
      Z[(size_t)b * ld + o] = zv;
      H[(size_t)b * ld + o] = __float2bfloat16_rn(h);
      Ht[(size_t)o * ldt + b] = __float2bfloat16_rn(h);
    } else {
      out[(size_t)b * ld + o] = zv;
    }
  }
}

// K ranges of a layer's product for B rows: about one CTA per SM when the layer has
// fewer output tiles than SMs (1: no split).
static int layer_splits(pas_mlp_t m, const GemmOp& op) {
  if (op.persist > 0) return 1;
  const int tiles = ((op.M + 127) / 128) * ((op.N + op.bn - 1) / op.bn);
  const int nk = (op.K + 63) / 64;
  return std::max(1, std::min(nk, m->ctx->sm_count / std::max(1, tiles)));
}

size_t mlp_split_workspace(pas_mlp_t m, int B) {
  size_t need = 0;
  for (int l = 0; l < m->L; ++l) {
    GemmOp op;
    op.M = B;
    op.N = m->sz[l + 1];
    op.K = m->sz[l];
    op.bn = gemm_pick_bn(B, op.N, m->ctx->sm_count);
    gemm_set_persist(&op, m->ctx->sm_count);
    const int sp = layer_splits(m, op);
    if (sp > 1) need = std::max(need, (size_t)sp * B * op.N);
  }
  return need;
}

pas_status mlp_batch_forward(pas_mlp_t m, int B, const float* const* d_slopes, float* part, size_t part_len,
                             cudaStream_t st) {
  if (B < 1 || B > m->max_batch) return set_error(m->ctx, PAS_EINVAL, "MLP batch forward: 1 <= B <= max_batch");
  const int n_in = m->sz[0];
  mlp_gather_input_kernel<<<dim3((n_in + 31) / 32, (B + 31) / 32), dim3(32, 8), 0, st>>>(
      d_slopes, B, n_in, m->d_mean, m->d_istd, m->d_X, m->ld[0], m->d_Xt, m->ldb);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return gemm_err(m, "MLP batch input", e);
  if (!part) return mlp_layers_enqueue(m, B, st);
  for (int l = 0; l < m->L; ++l) {
    const __nv_bfloat16* A = l == 0 ? m->d_X : m->d_H[l - 1];
    GemmOp op;
    if (!gemm_prepare(&op, A, m->ld[l], m->d_W[l], m->ld[l], B, m->sz[l + 1], m->sz[l], m->ctx->sm_count))
      return set_error(m->ctx, PAS_ECUDA, "MLP forward layer %d: tensor map rejected", l);
    const bool hidden = l < m->L - 1;
    const int sp = layer_splits(m, op);
    if (sp > 1 && (size_t)sp * B * m->sz[l + 1] <= part_len) {
      op.splits = sp;
      e = gemm_launch(op, EpiSplitPart{part, B, m->sz[l + 1]}, st, m->d_err, true);
      if (e == cudaSuccess) {
        const int n = B * m->sz[l + 1];
        mlp_split_finish_kernel<<<std::min(1024, (n + 255) / 256), 256, 0, st>>>(
            part, sp, B, m->sz[l + 1], m->d_p + m->offb[l], hidden ? 1 : 0, hidden ? m->d_Z[l] : nullptr,
            hidden ? m->d_H[l] : nullptr, hidden ? m->d_Ht[l] : nullptr, m->ld[l + 1], m->ldb, m->d_out);
        e = cudaGetLastError();
      }
    } else if (hidden) {
      EpiHidden ep{m->d_p + m->offb[l], m->d_Z[l], m->d_H[l], m->d_Ht[l], m->ld[l + 1], m->ldb, m->sz[l + 1]};
      e = gemm_launch(op, ep, st, m->d_err, true);
    } else {
      EpiOut ep{m->d_p + m->offb[l], m->d_out, m->ld[l + 1], m->sz[l + 1]};
      e = gemm_launch(op, ep, st, m->d_err, true);
    }
    if (e != cudaSuccess) return gemm_err(m, "MLP batch forward GEMM", e);
  }
  return PAS_OK;
}

int mlp_batch_forward_kernels(pas_mlp_t m, int B, size_t part_len) {
  int n = 1;  // the input gather
  for (int l = 0; l < m->L; ++l) {
    GemmOp op;
    op.M = B;
    op.N = m->sz[l + 1];
    op.K = m->sz[l];
    op.bn = gemm_pick_bn(B, op.N, m->ctx->sm_count);
    gemm_set_persist(&op, m->ctx->sm_count);
    const int sp = layer_splits(m, op);
    n += sp > 1 && (size_t)sp * B * op.N <= part_len ? 2 : 1;
  }
  return n;
}

// Loss, backward pass and bias gradients into d_g (loss into loss[*iter]).
static pas_status mlp_backward_enqueue(pas_mlp_t m, int B, const float* Y, int n_data, const int* idx,
                                       const int* iter, float* loss, cudaStream_t st) {
  const int L = m->L, n_out = m->sz[L];
  dim3 tb(32, 8);
  dim3 lg((n_out + 31) / 32, (B + 31) / 32);
  cudaError_t e = launch_k(mlp_loss_kernel, lg, tb, 0, st, true, (const float*)m->d_out, m->ld[L], Y, n_data, idx,
                           iter, B, n_out, m->d_dZ[L - 1], m->ld[L], m->d_dZt[L - 1], m->ldb, m->d_loss_part,
                           m->d_done, loss);
  if (e != cudaSuccess) return gemm_err(m, "MLP loss", e);
  for (int l = L - 1; l >= 0; --l) {
    // weight gradient dW_l = dZ_l^T H_{l-1}: M = out, N = in, K = B
    const __nv_bfloat16* Ht = l == 0 ? m->d_Xt : m->d_Ht[l - 1];
    GemmOp op;
    if (!gemm_prepare(&op, m->d_dZt[l], m->ldb, Ht, m->ldb, m->sz[l + 1], m->sz[l], B, m->ctx->sm_count))
      return set_error(m->ctx, PAS_ECUDA, "MLP weight-gradient layer %d: tensor map rejected", l);
    EpiF32 eg{m->d_g + m->offW[l], m->sz[l], m->sz[l]};
    e = gemm_launch(op, eg, st, m->d_err, true);
    if (e != cudaSuccess) return gemm_err(m, "MLP weight-gradient GEMM", e);
    if (l == 0) break;
    // input gradient dH_{l-1} = dZ_l W_l, times gelu'(Z_{l-1}): M = B, N = in, K = out
    GemmOp ob;
    if (!gemm_prepare(&ob, m->d_dZ[l], m->ld[l + 1], m->d_Wt[l], m->ld[l + 1], B, m->sz[l], m->sz[l + 1],
                      m->ctx->sm_count))
      return set_error(m->ctx, PAS_ECUDA, "MLP input-gradient layer %d: tensor map rejected", l);
    EpiBack eb{m->d_Z[l - 1], m->d_dZ[l - 1], m->d_dZt[l - 1], m->ld[l], m->ldb, m->sz[l]};
    e = gemm_launch(ob, eb, st, m->d_err, true);
    if (e != cudaSuccess) return gemm_err(m, "MLP input-gradient GEMM", e);
  }
  BiasGradArgs ba = {};
  ba.L = L;
  ba.ldt = m->ldb;
  ba.B = B;
  ba.g = m->d_g;
  ba.start[0] = 0;
  for (int l = 0; l < L; ++l) {
    ba.dZt[l] = m->d_dZt[l];
    ba.offb[l] = m->offb[l];
    ba.start[l + 1] = ba.start[l] + m->sz[l + 1];
  }
  const int warps = ba.start[L];
  e = launch_k(mlp_bias_grad_kernel, dim3((warps * 32 + 255) / 256), dim3(256), 0, st, true, ba);
  if (e != cudaSuccess) return gemm_err(m, "MLP bias gradient", e);
  return PAS_OK;
}

static AdamArgs adam_args(pas_mlp_t m, int update) {
  AdamArgs a = {};
  a.p = m->d_p;
  a.m = m->d_m;
  a.v = m->d_v;
  a.g = m->d_g;
  a.L = m->L;
  a.tile_start[0] = 0;
  a.bias_start[0] = 0;
  for (int l = 0; l < m->L; ++l) {
    a.out[l] = m->sz[l + 1];
    a.in[l] = m->sz[l];
    a.offW[l] = m->offW[l];
    a.offb[l] = m->offb[l];
    a.W[l] = m->d_W[l];
    a.Wt[l] = m->d_Wt[l];
    a.ldW[l] = m->ld[l];
    a.ldWt[l] = m->ld[l + 1];
    a.tile_start[l + 1] = a.tile_start[l] + ((m->sz[l + 1] + 31) / 32) * ((m->sz[l] + 31) / 32);
    a.bias_start[l + 1] = a.bias_start[l] + m->sz[l + 1];
  }
  a.update = update;
  a.t = m->d_t;
  a.b1 = 0.9f;
  a.b2 = 0.999f;
  a.eps = 1e-8f;
  a.done = m->d_done + 1;
  return a;
}

static pas_status adam_launch(pas_mlp_t m, const AdamArgs& a, cudaStream_t st, bool pdl = false) {
  const int blocks = a.tile_start[a.L] + (a.update ? (a.bias_start[a.L] + 255) / 256 : 0);
  cudaError_t e = launch_k(mlp_adam_kernel, dim3(blocks), dim3(32, 8), 0, st, pdl, a);
  if (e != cudaSuccess) return gemm_err(m, "MLP Adam", e);
  return PAS_OK;
}

static pas_status mlp_train_enqueue(pas_mlp_t m, int B, const float* S, const float* Y, int n_data, const int* idx,
                                    const float* lr, float* loss, cudaStream_t st) {
  pas_status s = mlp_forward_enqueue(m, B, S, n_data, idx, m->d_iter, st);
  if (s == PAS_OK) s = mlp_backward_enqueue(m, B, Y, n_data, idx, m->d_iter, loss, st);
  if (s != PAS_OK) return s;
  AdamArgs a = adam_args(m, 1);
  a.lr = lr;
  a.iter = m->d_iter;
  a.iter_inc = m->d_iter;
  return adam_launch(m, a, st, true);
}

// ---------------------------------------------------------------- training pairs

__global__ void scale_kernel(const float* in, float amp, float* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = amp * in[i];
}

}  // namespace pas

// ================================================================ C ABI

using pas::dev_alloc;
using pas::dev_free;

extern "C" {

void pas_mlp_destroy(pas_mlp_t m) {
  if (!m) return;
  if (m->train_exec) cudaGraphExecDestroy(m->train_exec);
  if (m->train_graph) cudaGraphDestroy(m->train_graph);
  void* ptrs[] = {m->d_p,   m->d_g,    m->d_m,     m->d_v,        m->d_t,         m->d_mean,  m->d_istd,
                  m->d_X,   m->d_Xt,   m->d_out,   m->d_loss_part, m->d_done,     m->d_zero,  m->d_iter,
                  m->d_loss1, m->d_lr1, m->d_err,  m->d_fault,    m->d_gemv_done, m->d_vec[0], m->d_vec[1]};
  for (void* p : ptrs) dev_free(p);
  for (int l = 0; l < PAS_MLP_MAX_LAYERS; ++l) {
    dev_free(m->d_W[l]);
    dev_free(m->d_Wt[l]);
    dev_free(m->d_Z[l]);
    dev_free(m->d_H[l]);
    dev_free(m->d_Ht[l]);
    dev_free(m->d_dZ[l]);
    dev_free(m->d_dZt[l]);
  }
  delete m;
}

pas_status pas_mlp_create(pas_ctx_t ctx, int32_t n_layers, const int32_t* sizes, int32_t max_batch,
                          pas_mlp_t* out) {
  if (!ctx || !sizes || !out) return pas::set_global_error(PAS_EINVAL, "pas_mlp_create: NULL argument");
  *out = nullptr;
  PAS_CHECK_ARG(ctx, n_layers >= 1 && n_layers <= PAS_MLP_MAX_LAYERS, "pas_mlp_create: 1 <= n_layers <= 8");
  PAS_CHECK_ARG(ctx, max_batch >= 1 && max_batch <= (1 << 20), "pas_mlp_create: 1 <= max_batch <= 2^20");
  for (int l = 0; l <= n_layers; ++l)
    PAS_CHECK_ARG(ctx, sizes[l] >= 1 && sizes[l] <= 65536, "pas_mlp_create: layer widths in [1, 65536]");
  pas_mlp_t m = new pas_mlp_s();
  m->ctx = ctx;
  m->L = n_layers;
  for (int l = 0; l <= n_layers; ++l) {
    m->sz[l] = sizes[l];
    m->ld[l] = (sizes[l] + 7) / 8 * 8;
  }
  m->max_batch = max_batch;
  m->ldb = (max_batch + 7) / 8 * 8;
  // internal parameter layout: every tensor starts on a 16-byte boundary
  size_t o = 0;
  for (int l = 0; l < n_layers; ++l) {
    m->offW[l] = o;
    o += ((size_t)sizes[l + 1] * sizes[l] + 3) / 4 * 4;
    m->offb[l] = o;
    o += ((size_t)sizes[l + 1] + 3) / 4 * 4;
  }
  m->n_params = o;
  pas_status st = PAS_OK;
  auto A = [&](void** p, size_t bytes) {
    if (st == PAS_OK) st = dev_alloc(ctx, p, bytes);
  };
  const size_t B = (size_t)max_batch;
  A((void**)&m->d_p, 4 * o);
  A((void**)&m->d_g, 4 * o);
  A((void**)&m->d_m, 4 * o);
  A((void**)&m->d_v, 4 * o);
  A((void**)&m->d_t, sizeof(long long));
  A((void**)&m->d_mean, 4 * (size_t)m->ld[0]);
  A((void**)&m->d_istd, 4 * (size_t)m->ld[0]);
  A((void**)&m->d_X, 2 * B * m->ld[0]);
  A((void**)&m->d_Xt, 2 * (size_t)m->sz[0] * m->ldb);
  A((void**)&m->d_out, 4 * B * m->ld[n_layers]);
  const size_t loss_blocks = ((size_t)(sizes[n_layers] + 31) / 32) * ((B + 31) / 32);
  A((void**)&m->d_loss_part, 4 * loss_blocks);
  A((void**)&m->d_done, 4 * sizeof(unsigned));
  A((void**)&m->d_zero, sizeof(int));
  A((void**)&m->d_iter, sizeof(int));
  A((void**)&m->d_loss1, sizeof(float));
  A((void**)&m->d_lr1, sizeof(float));
  A((void**)&m->d_err, sizeof(unsigned));
  A((void**)&m->d_fault, sizeof(unsigned));
  A((void**)&m->d_gemv_done, sizeof(unsigned));
  int widest = 0;
  for (int l = 0; l <= n_layers; ++l) widest = std::max(widest, m->ld[l]);
  A((void**)&m->d_vec[0], 4 * (size_t)widest);
  A((void**)&m->d_vec[1], 4 * (size_t)widest);
  for (int l = 0; l < n_layers; ++l) {
    A((void**)&m->d_W[l], 2 * (size_t)m->sz[l + 1] * m->ld[l]);
    A((void**)&m->d_Wt[l], 2 * (size_t)m->sz[l] * m->ld[l + 1]);
    A((void**)&m->d_dZ[l], 2 * B * m->ld[l + 1]);
    A((void**)&m->d_dZt[l], 2 * (size_t)m->sz[l + 1] * m->ldb);
    if (l < n_layers - 1) {
      A((void**)&m->d_Z[l], 4 * B * m->ld[l + 1]);
      A((void**)&m->d_H[l], 2 * B * m->ld[l + 1]);
      A((void**)&m->d_Ht[l], 2 * (size_t)m->sz[l + 1] * m->ldb);
    }
  }
  if (st != PAS_OK) {
    pas_mlp_destroy(m);
    return st;
  }
  cudaError_t e = cudaSuccess;
  auto Z = [&](void* p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMemset(p, 0, bytes);
  };
  Z(m->d_p, 4 * o);
  Z(m->d_g, 4 * o);
  Z(m->d_m, 4 * o);
  Z(m->d_v, 4 * o);
  Z(m->d_t, sizeof(long long));
  Z(m->d_mean, 4 * (size_t)m->ld[0]);
  Z(m->d_done, 4 * sizeof(unsigned));
  Z(m->d_zero, sizeof(int));
  Z(m->d_iter, sizeof(int));
  Z(m->d_err, sizeof(unsigned));
  Z(m->d_fault, sizeof(unsigned));
  Z(m->d_gemv_done, sizeof(unsigned));
  for (int l = 0; l < n_layers; ++l) {
    Z(m->d_W[l], 2 * (size_t)m->sz[l + 1] * m->ld[l]);
    Z(m->d_Wt[l], 2 * (size_t)m->sz[l] * m->ld[l + 1]);
  }
  if (e == cudaSuccess) {
    std::vector<float> ones(m->ld[0], 1.0f);
    e = cudaMemcpy(m->d_istd, ones.data(), 4 * ones.size(), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    pas_mlp_destroy(m);
    return pas::set_error(ctx, PAS_ECUDA, "pas_mlp_create: %s", cudaGetErrorString(e));
  }
  *out = m;
  return PAS_OK;
}

int64_t pas_mlp_n_params(pas_mlp_t m) {
  if (!m) return -1;
  int64_t n = 0;
  for (int l = 0; l < m->L; ++l) n += (int64_t)m->sz[l + 1] * m->sz[l] + m->sz[l + 1];
  return n;
}

// packed (user) offset of every tensor, in order W_0, b_0, W_1, ...
static void packed_tensors(pas_mlp_t m, std::vector<size_t>& internal, std::vector<size_t>& count) {
  for (int l = 0; l < m->L; ++l) {
    internal.push_back(m->offW[l]);
    count.push_back((size_t)m->sz[l + 1] * m->sz[l]);
    internal.push_back(m->offb[l]);
    count.push_back((size_t)m->sz[l + 1]);
  }
}

static pas_status copy_packed(pas_mlp_t m, float* dst_packed, const float* src_internal, cudaMemcpyKind kind) {
  std::vector<size_t> in, cnt;
  packed_tensors(m, in, cnt);
  size_t o = 0;
  for (size_t t = 0; t < in.size(); ++t) {
    PAS_CUDA_TRY(m->ctx, cudaMemcpyAsync(dst_packed + o, src_internal + in[t], 4 * cnt[t], kind, m->ctx->stream));
    o += cnt[t];
  }
  return PAS_OK;
}

pas_status pas_mlp_set_params(pas_mlp_t m, const float* h_params) {
  if (!m || !h_params) return pas::set_global_error(PAS_EINVAL, "pas_mlp_set_params: NULL argument");
  pas_ctx_t ctx = m->ctx;
  std::vector<size_t> in, cnt;
  packed_tensors(m, in, cnt);
  size_t o = 0;
  for (size_t t = 0; t < in.size(); ++t) {
    PAS_CUDA_TRY(ctx, cudaMemcpyAsync(m->d_p + in[t], h_params + o, 4 * cnt[t], cudaMemcpyHostToDevice, ctx->stream));
    o += cnt[t];
  }
  PAS_CUDA_TRY(ctx, cudaMemsetAsync(m->d_m, 0, 4 * m->n_params, ctx->stream));
  PAS_CUDA_TRY(ctx, cudaMemsetAsync(m->d_v, 0, 4 * m->n_params, ctx->stream));
  PAS_CUDA_TRY(ctx, cudaMemsetAsync(m->d_t, 0, sizeof(long long), ctx->stream));
  pas_status s = pas::adam_launch(m, pas::adam_args(m, 0), ctx->stream);
  if (s != PAS_OK) return s;
  PAS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return PAS_OK;
}

pas_status pas_mlp_get_params(pas_mlp_t m, float* h_params) {
  if (!m || !h_params) return pas::set_global_error(PAS_EINVAL, "pas_mlp_get_params: NULL argument");
  pas_status s = copy_packed(m, h_params, m->d_p, cudaMemcpyDeviceToHost);
  if (s != PAS_OK) return s;
  PAS_CUDA_TRY(m->ctx, cudaStreamSynchronize(m->ctx->stream));
  return PAS_OK;
}

pas_status pas_mlp_set_norm(pas_mlp_t m, const float* h_mean, const float* h_inv_std) {
  if (!m || !h_mean || !h_inv_std) return pas::set_global_error(PAS_EINVAL, "pas_mlp_set_norm: NULL argument");
  PAS_CUDA_TRY(m->ctx, cudaMemcpy(m->d_mean, h_mean, 4 * (size_t)m->sz[0], cudaMemcpyHostToDevice));
  PAS_CUDA_TRY(m->ctx, cudaMemcpy(m->d_istd, h_inv_std, 4 * (size_t)m->sz[0], cudaMemcpyHostToDevice));
  return PAS_OK;
}

pas_status pas_mlp_apply(pas_mlp_t m, const float* d_slopes, float* d_out) {
  if (!m || !d_slopes || !d_out) return pas::set_global_error(PAS_EINVAL, "pas_mlp_apply: NULL argument");
  return pas::gemv_chain(m, d_slopes, d_out, nullptr, m->ctx->stream, false);
}

pas_status pas_mlp_forward(pas_mlp_t m, int32_t batch, const float* d_S, float* d_out) {
  if (!m || !d_S || !d_out) return pas::set_global_error(PAS_EINVAL, "pas_mlp_forward: NULL argument");
  PAS_CHECK_ARG(m->ctx, batch >= 1 && batch <= m->max_batch, "pas_mlp_forward: 1 <= batch <= max_batch");
  cudaStream_t st = m->ctx->stream;
  pas_status s = pas::mlp_forward_enqueue(m, batch, d_S, batch, nullptr, m->d_zero, st);
  if (s != PAS_OK) return s;
  const int n_out = m->sz[m->L];
  PAS_CUDA_TRY(m->ctx, cudaMemcpy2DAsync(d_out, 4 * (size_t)n_out, m->d_out, 4 * (size_t)m->ld[m->L],
                                         4 * (size_t)n_out, batch, cudaMemcpyDeviceToDevice, st));
  return PAS_OK;
}

pas_status pas_mlp_gradients(pas_mlp_t m, int32_t batch, const float* d_S, const float* d_Y, float* d_grad,
                             float* h_loss) {
  if (!m || !d_S || !d_Y || !d_grad) return pas::set_global_error(PAS_EINVAL, "pas_mlp_gradients: NULL argument");
  PAS_CHECK_ARG(m->ctx, batch >= 1 && batch <= m->max_batch, "pas_mlp_gradients: 1 <= batch <= max_batch");
  cudaStream_t st = m->ctx->stream;
  pas_status s = pas::mlp_forward_enqueue(m, batch, d_S, batch, nullptr, m->d_zero, st);
  if (s == PAS_OK) s = pas::mlp_backward_enqueue(m, batch, d_Y, batch, nullptr, m->d_zero, m->d_loss1, st);
  if (s == PAS_OK) s = copy_packed(m, d_grad, m->d_g, cudaMemcpyDeviceToDevice);
  if (s != PAS_OK) return s;
  if (h_loss) {
    PAS_CUDA_TRY(m->ctx, cudaMemcpyAsync(h_loss, m->d_loss1, sizeof(float), cudaMemcpyDeviceToHost, st));
    PAS_CUDA_TRY(m->ctx, cudaStreamSynchronize(st));
  }
  return PAS_OK;
}

pas_status pas_mlp_train(pas_mlp_t m, const float* d_S, const float* d_Y, int32_t n_data, int32_t batch,
                         const int32_t* d_idx, const float* d_lr, int32_t n_steps, float* d_loss) {
  if (!m || !d_S || !d_Y || !d_idx || !d_lr || !d_loss)
    return pas::set_global_error(PAS_EINVAL, "pas_mlp_train: NULL argument");
  pas_ctx_t ctx = m->ctx;
  PAS_CHECK_ARG(ctx, batch >= 1 && batch <= m->max_batch, "pas_mlp_train: 1 <= batch <= max_batch");
  PAS_CHECK_ARG(ctx, n_data >= 1 && n_steps >= 0, "pas_mlp_train: n_data >= 1, n_steps >= 0");
  const void* key[6] = {d_S, d_Y, d_idx, d_lr, d_loss, (const void*)(intptr_t)n_data};
  if (m->train_exec && (batch != m->train_batch || memcmp(key, m->train_key, sizeof(key)) != 0)) {
    cudaGraphExecDestroy(m->train_exec);
    cudaGraphDestroy(m->train_graph);
    m->train_exec = nullptr;
    m->train_graph = nullptr;
  }
  if (!m->train_exec) {
    PAS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    PAS_CUDA_TRY(ctx, cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
    pas_status s = pas::mlp_train_enqueue(m, batch, d_S, d_Y, n_data, d_idx, d_lr, d_loss, ctx->capture_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->capture_stream, &g);
    if (s != PAS_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) return pas::set_error(ctx, PAS_ECUDA, "training capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&m->train_exec, g, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      return pas::set_error(ctx, PAS_ECUDA, "training instantiate: %s", cudaGetErrorString(e));
    }
    m->train_graph = g;
    m->train_batch = batch;
    memcpy(m->train_key, key, sizeof(key));
  }
  PAS_CUDA_TRY(ctx, cudaMemsetAsync(m->d_iter, 0, sizeof(int), ctx->stream));
  for (int t = 0; t < n_steps; ++t) PAS_CUDA_TRY(ctx, cudaGraphLaunch(m->train_exec, ctx->stream));
  return PAS_OK;
}

pas_status pas_mlp_check(pas_mlp_t m, uint32_t* h_fault) {
  if (!m) return pas::set_global_error(PAS_EINVAL, "pas_mlp_check: NULL argument");
  unsigned e = 0, f = 0;
  PAS_CUDA_TRY(m->ctx, cudaStreamSynchronize(m->ctx->stream));
  PAS_CUDA_TRY(m->ctx, cudaMemcpy(&e, m->d_err, sizeof(e), cudaMemcpyDeviceToHost));
  PAS_CUDA_TRY(m->ctx, cudaMemcpy(&f, m->d_fault, sizeof(f), cudaMemcpyDeviceToHost));
  PAS_CUDA_TRY(m->ctx, cudaMemset(m->d_err, 0, sizeof(unsigned)));
  PAS_CUDA_TRY(m->ctx, cudaMemset(m->d_fault, 0, sizeof(unsigned)));
  if (h_fault) *h_fault = f;
  if (e & pas::MLP_ERR_INDEX) return pas::set_error(m->ctx, PAS_EINVAL, "MLP: sample index out of range");
  if (e) return pas::set_error(m->ctx, PAS_ETIMEOUT, "MLP: tensor-core pipeline wait timed out (code %u)", e);
  return PAS_OK;
}

pas_status pas_mlp_pair(pas_pyr_t pyr, pas_dm_t dm, const float* d_opd, float amp, float* d_work, float* d_slopes,
                        float* d_coeffs) {
  if (!pyr || !dm || !d_opd || !d_work || !d_slopes || !d_coeffs)
    return pas::set_global_error(PAS_EINVAL, "pas_mlp_pair: NULL argument");
  pas_ctx_t ctx = dm->ctx;
  PAS_CHECK_ARG(ctx, pas::pyr_np(pyr) == dm->Np, "pas_mlp_pair: pyramid and DM pupil sizes differ");
  const int Np = dm->Np, n = Np * Np;
  cudaStream_t st = ctx->stream;
  pas::scale_kernel<<<(n + 255) / 256, 256, 0, st>>>(d_opd, amp, d_work, n);
  PAS_CUDA_TRY(ctx, cudaGetLastError());
  pas_status s = pas::pyr_launch(pyr, d_work, d_work + n, d_slopes, st, nullptr, true);
  if (s != PAS_OK) return s;
  return pas::dm_project_launch(dm, d_work, d_coeffs, st);
}

pas_status pas_gemm_bf16(pas_ctx_t ctx, int32_t M, int32_t N, int32_t K, const uint16_t* d_A, int32_t lda,
                         const uint16_t* d_B, int32_t ldb, float* d_C, int32_t ldc, int32_t tile_n,
                         uint32_t* d_err) {
  return pas_gemm_bf16_waits(ctx, M, N, K, d_A, lda, d_B, ldb, d_C, ldc, tile_n, pas::tc::WAIT_LIMIT, d_err);
}

pas_status pas_gemm_bf16_waits(pas_ctx_t ctx, int32_t M, int32_t N, int32_t K, const uint16_t* d_A, int32_t lda,
                               const uint16_t* d_B, int32_t ldb, float* d_C, int32_t ldc, int32_t tile_n,
                               uint32_t wait_limit, uint32_t* d_err) {
  if (!ctx || !d_A || !d_B || !d_C || !d_err) return pas::set_global_error(PAS_EINVAL, "pas_gemm_bf16: NULL argument");
  PAS_CHECK_ARG(ctx, M >= 1 && N >= 1 && K >= 1 && lda >= K && ldb >= K && ldc >= N,
                "pas_gemm_bf16: M, N, K >= 1, lda, ldb >= K, ldc >= N");
  PAS_CHECK_ARG(ctx, lda % 8 == 0 && ldb % 8 == 0, "pas_gemm_bf16: lda and ldb must be multiples of 8");
  PAS_CHECK_ARG(ctx, tile_n == 0 || tile_n == 16 || tile_n == 32 || tile_n == 64 || tile_n == 128 || tile_n == 256,
                "pas_gemm_bf16: tile_n in {0 (automatic), 16, 32, 64, 128, 256}");
  pas::GemmOp op;
  if (!pas::gemm_prepare(&op, reinterpret_cast<const __nv_bfloat16*>(d_A), lda,
                         reinterpret_cast<const __nv_bfloat16*>(d_B), ldb, M, N, K, ctx->sm_count))
    return pas::set_error(ctx, PAS_EINVAL, "pas_gemm_bf16: tensor map rejected (16-byte alignment)");
  if (tile_n) {  // a fixed tile width
    op.bn = tile_n;
    pas::gemm_set_persist(&op, ctx->sm_count);
    if (!pas::make_tmap_bf16(&op.b, d_B, (uint64_t)N, (uint64_t)K, (uint64_t)ldb, (uint32_t)tile_n))
      return pas::set_error(ctx, PAS_EINVAL, "pas_gemm_bf16: tensor map rejected");
  }
  pas::EpiF32 ep{d_C, ldc, N};
  cudaError_t e = pas::gemm_launch(op, ep, ctx->stream, d_err, false, wait_limit);
  if (e != cudaSuccess) return pas::set_error(ctx, PAS_ECUDA, "pas_gemm_bf16: %s", cudaGetErrorString(e));
  return PAS_OK;
}

}  // extern "C"
