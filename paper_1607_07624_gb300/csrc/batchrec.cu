// Batched reconstruction on the tensor cores: the loops of a batch that share one
// bfloat16 reconstructor R (n_m x n_s, rows scaled to max |R| = 1) get their modal
// updates from one product C = R S^T, S the B x n_s matrix of their slopes in
// bfloat16, with float32 accumulation in tensor memory (gemm.cuh). The epilogue applies
// each loop's integrator (c_t = c_{t-1} + g * scale_m * C[m][b], written into the loop's
// command ring), so the per-loop matrix-vector products disappear from the step: R is
// read once per step instead of B times.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "batchrec.cuh"
#include "gemm.cuh"
#include "mlp.cuh"

namespace pas {

struct BatchRecGroup {
  pas_ctx_t ctx = nullptr;
  pas_recon_t rec = nullptr;
  pas_mlp_t mlp = nullptr;       // a shared network instead of rec: one batched forward
  int B = 0;
  __nv_bfloat16* d_S = nullptr;  // [B][n_s_pad]
  float* d_part = nullptr;       // split product: [splits][n_m][B] partial sums (a network: its layers')
  size_t part_len = 0;           // floats of d_part
  void** d_ptrs = nullptr;       // the pointer arrays of BatchRecState, contiguous
  int* d_delay = nullptr;
  unsigned int* d_err = nullptr;
  BatchRecState st;
  GemmOp op;
};

// S[b][j] = bf16(s_b[j]) for j < n_s, 0 in the row padding.
__global__ void gather_slopes_bf16_kernel(const float* const* slopes, int n_s, int n_s_pad, int B,
                                          __nv_bfloat16* S) {
  const size_t tot = (size_t)B * n_s_pad;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(t / n_s_pad), j = (int)(t - (size_t)b * n_s_pad);
    S[t] = __float2bfloat16_rn(j < n_s ? slopes[b][j] : 0.f);
  }
}

__global__ void advance_steps_kernel(long long* const* step, int B) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) *step[b] += 1;
}

// A shared network's outputs out[b][m] (its last layer, float32) as each loop's modal
// update: the integrator of the single-vector chain's last layer, a non-finite output
// replaced by 0 with fault bit 0 set.
__global__ void mlp_batch_integrate_kernel(const float* out, int ldo, int n_m, int B, BatchRecState st,
                                           unsigned* fault) {
  const size_t tot = (size_t)B * n_m;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(t / n_m), m = (int)(t - (size_t)b * n_m);
    float z = out[(size_t)b * ldo + m];
    if (!isfinite(z)) {
      atomicOr(fault, 1u);
      z = 0.f;
    }
    const long long ts = *st.step[b];
    const int d = st.delay[b];
    float* ring = st.ring[b];
    const float prev = ring[(size_t)((ts - 1 + d) % d) * n_m + m];
    const float c = fmaf(st.gain[b][m], z, prev);
    ring[(size_t)(ts % d) * n_m + m] = c;
    st.cmd[b][m] = c;
    st.dmodes[b][m] = z;
  }
}

// Epilogue: rows are modes, columns are loops. The per-loop pointers, step counters
// and gains are read-only during the product: each group of 4 columns loads them level
// by level (pointers, then the values they point to), so a thread waits 3 memory
// latencies per 4 columns instead of one per dependent load of every column.
struct EpiBatchIntegrate {
  BatchRecState st;
  const float* scale;  // [n_m] per-row scale of the bf16 reconstructor
  int n_m, B;
  __device__ void store(int m, int col, const float (&v)[16]) const {
    constexpr int CH = 4;
    const float sc = __ldg(scale + m);
#pragma unroll
    for (int j0 = 0; j0 < 16; j0 += CH) {
      float* ring[CH];
      const float* gain[CH];
      const long long* stp[CH];
      int d[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int b = min(col + j0 + u, B - 1);
        ring[u] = st.ring[b];
        gain[u] = st.gain[b];
        stp[u] = st.step[b];
        d[u] = __ldg(st.delay + b);
      }
      long long t[CH];
      float g[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        t[u] = __ldg(stp[u]);
        g[u] = __ldg(gain[u] + m);
      }
      float prev[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) prev[u] = ring[u][(size_t)((t[u] - 1 + d[u]) % d[u]) * n_m + m];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int b = col + j0 + u;
        if (b < B) {
          const float dm = v[j0 + u] * sc;
          const float c = fmaf(g[u], dm, prev[u]);
          ring[u][(size_t)(t[u] % d[u]) * n_m + m] = c;
          st.cmd[b][m] = c;
          st.dmodes[b][m] = dm;
        }
      }
    }
  }
};

// Split reduction (few row tiles, long rows): each K range's product [n_m][B] goes to
// its own slice of the workspace (EpiSplitPart); this kernel adds the slices in range
// order and applies the integrator of EpiBatchIntegrate.
__global__ void split_integrate_kernel(const float* part, int splits, int n_m, int B, const float* scale,
                                       BatchRecState st) {
  const size_t tot = (size_t)n_m * B;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(t / B), b = (int)(t - (size_t)m * B);
    float acc = 0.f;
    for (int z = 0; z < splits; ++z) acc += part[((size_t)z * n_m + m) * B + b];
    const float dm = acc * scale[m];
    const long long ts = *st.step[b];
    const int d = st.delay[b];
    float* ring = st.ring[b];
    const float prev = ring[(size_t)((ts - 1 + d) % d) * n_m + m];
    const float c = fmaf(st.gain[b][m], dm, prev);
    ring[(size_t)(ts % d) * n_m + m] = c;
    st.cmd[b][m] = c;
    st.dmodes[b][m] = dm;
  }
}

static int pick_bn(int B) { return B <= 16 ? 16 : B <= 32 ? 32 : B <= 64 ? 64 : 128; }

// The group's per-loop pointer arrays on the device (g->st).
static pas_status group_pointers(BatchRecGroup* g, const float* const* slopes, float* const* ring,
                                 const float* const* gain, float* const* cmd, float* const* dmodes,
                                 long long* const* step, const int* delay) {
  const int B = g->B;
  pas_status s = dev_alloc(g->ctx, (void**)&g->d_ptrs, sizeof(void*) * 6 * (size_t)B);
  if (s == PAS_OK) s = dev_alloc(g->ctx, (void**)&g->d_delay, sizeof(int) * B);
  if (s == PAS_OK) s = dev_alloc(g->ctx, (void**)&g->d_err, sizeof(unsigned int));
  if (s != PAS_OK) return s;
  std::vector<void*> h(6 * (size_t)B);
  for (int b = 0; b < B; ++b) {
    h[0 * B + b] = const_cast<float*>(slopes[b]);
    h[1 * B + b] = ring[b];
    h[2 * B + b] = const_cast<float*>(gain[b]);
    h[3 * B + b] = cmd[b];
    h[4 * B + b] = dmodes[b];
    h[5 * B + b] = step[b];
  }
  cudaError_t e = cudaMemcpy(g->d_ptrs, h.data(), sizeof(void*) * h.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(g->d_delay, delay, sizeof(int) * B, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(g->d_err, 0, sizeof(unsigned int));
  if (e != cudaSuccess) return set_error(g->ctx, PAS_ECUDA, "batched reconstruction: %s", cudaGetErrorString(e));
  g->st.slopes = reinterpret_cast<const float* const*>(g->d_ptrs);
  g->st.ring = reinterpret_cast<float* const*>(g->d_ptrs + (size_t)B);
  g->st.gain = reinterpret_cast<const float* const*>(g->d_ptrs + 2 * (size_t)B);
  g->st.cmd = reinterpret_cast<float* const*>(g->d_ptrs + 3 * (size_t)B);
  g->st.dmodes = reinterpret_cast<float* const*>(g->d_ptrs + 4 * (size_t)B);
  g->st.step = reinterpret_cast<long long* const*>(g->d_ptrs + 5 * (size_t)B);
  g->st.delay = g->d_delay;
  return PAS_OK;
}

pas_status batch_mlp_create(pas_ctx_t ctx, pas_mlp_t mlp, int B, const float* const* slopes, float* const* ring,
                            const float* const* gain, float* const* cmd, float* const* dmodes,
                            long long* const* step, const int* delay, BatchRecGroup** out) {
  *out = nullptr;
  PAS_CHECK_ARG(ctx, mlp != nullptr, "batched inference: a network");
  PAS_CHECK_ARG(ctx, B >= 1 && B <= std::min(128, mlp->max_batch),
                "batched inference: 1 to min(128, the network's batch size) loops per group");
  BatchRecGroup* g = new BatchRecGroup();
  g->ctx = ctx;
  g->mlp = mlp;
  g->B = B;
  pas_status s = group_pointers(g, slopes, ring, gain, cmd, dmodes, step, delay);
  g->part_len = mlp_split_workspace(mlp, B);
  if (s == PAS_OK && g->part_len > 0) s = dev_alloc(ctx, (void**)&g->d_part, sizeof(float) * g->part_len);
  if (s != PAS_OK) {
    batch_rec_destroy(g);
    return s;
  }
  *out = g;
  return PAS_OK;
}

pas_status batch_rec_create(pas_ctx_t ctx, pas_recon_t rec, int B, const float* const* slopes, float* const* ring,
                            const float* const* gain, float* const* cmd, float* const* dmodes,
                            long long* const* step, const int* delay, BatchRecGroup** out) {
  *out = nullptr;
  PAS_CHECK_ARG(ctx, rec && rec->prec == PAS_BF16 && rec->d_Rb, "batched reconstruction: a bf16 reconstructor");
  PAS_CHECK_ARG(ctx, B >= 1 && B <= 128, "batched reconstruction: 1 to 128 loops per group");
  BatchRecGroup* g = new BatchRecGroup();
  g->ctx = ctx;
  g->rec = rec;
  g->B = B;
  pas_status s = dev_alloc(ctx, (void**)&g->d_S, sizeof(__nv_bfloat16) * (size_t)B * rec->n_s_pad);
  if (s == PAS_OK) s = group_pointers(g, slopes, ring, gain, cmd, dmodes, step, delay);
  if (s != PAS_OK) {
    batch_rec_destroy(g);
    return s;
  }
  // C[n_m][B] = R[n_m][n_s_pad] * S[B][n_s_pad]^T (both K-major, zero row padding)
  const int K = rec->n_s_pad;
  g->op.M = rec->n_modes;
  g->op.N = B;
  g->op.K = K;
  g->op.bn = pick_bn(B);
  if (!make_tmap_bf16(&g->op.a, rec->d_Rb, (uint64_t)rec->n_modes, (uint64_t)K, (uint64_t)K, 128) ||
      !make_tmap_bf16(&g->op.b, g->d_S, (uint64_t)B, (uint64_t)K, (uint64_t)K, (uint32_t)g->op.bn)) {
    batch_rec_destroy(g);
    return set_error(ctx, PAS_EINVAL, "batched reconstruction: tensor map rejected");
  }
  // fewer output tiles than SMs: split K so that about one CTA per SM streams R
  const int tiles = ((rec->n_modes + 127) / 128) * ((B + g->op.bn - 1) / g->op.bn);
  const int nk = (K + 63) / 64;
  g->op.splits = std::max(1, std::min(nk, ctx->sm_count / std::max(1, tiles)));
  if (g->op.splits > 1) {
    s = dev_alloc(ctx, (void**)&g->d_part, sizeof(float) * (size_t)g->op.splits * rec->n_modes * B);
    if (s != PAS_OK) {
      batch_rec_destroy(g);
      return s;
    }
  }
  *out = g;
  return PAS_OK;
}

pas_status batch_rec_launch(BatchRecGroup* g, cudaStream_t st) {
  if (g->mlp) {
    pas_mlp_t m = g->mlp;
    pas_status s = mlp_batch_forward(m, g->B, g->st.slopes, g->d_part, g->part_len, st);
    if (s != PAS_OK) return s;
    const int n_m = m->sz[m->L];
    const int blocks = (int)std::min<size_t>(1024, ((size_t)g->B * n_m + 255) / 256);
    mlp_batch_integrate_kernel<<<blocks, 256, 0, st>>>(m->d_out, m->ld[m->L], n_m, g->B, g->st, m->d_fault);
    advance_steps_kernel<<<(g->B + 127) / 128, 128, 0, st>>>(g->st.step, g->B);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(g->ctx, PAS_ECUDA, "batched inference launch: %s", cudaGetErrorString(e));
    return PAS_OK;
  }
  const int n_s = g->rec->n_slopes, K = g->rec->n_s_pad;
  const int blocks = (int)std::min<size_t>(1024, ((size_t)g->B * K + 255) / 256);
  gather_slopes_bf16_kernel<<<blocks, 256, 0, st>>>(g->st.slopes, n_s, K, g->B, g->d_S);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && g->op.splits > 1) {
    e = gemm_launch(g->op, EpiSplitPart{g->d_part, g->rec->n_modes, g->B}, st, g->d_err, false);
    if (e == cudaSuccess) {
      const int n = g->rec->n_modes * g->B;
      split_integrate_kernel<<<std::min(1024, (n + 255) / 256), 256, 0, st>>>(g->d_part, g->op.splits, g->rec->n_modes,
                                                                            g->B, g->rec->d_scale, g->st);
      e = cudaGetLastError();
    }
  } else if (e == cudaSuccess) {
    EpiBatchIntegrate ep{g->st, g->rec->d_scale, g->rec->n_modes, g->B};
    e = gemm_launch(g->op, ep, st, g->d_err, false);
  }
  if (e == cudaSuccess) {
    advance_steps_kernel<<<(g->B + 127) / 128, 128, 0, st>>>(g->st.step, g->B);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess)
    return set_error(g->ctx, PAS_ECUDA, "batched reconstruction launch: %s", cudaGetErrorString(e));
  return PAS_OK;
}

unsigned int* batch_rec_err(BatchRecGroup* g) { return g->mlp ? g->mlp->d_err : g->d_err; }

int batch_rec_kernels(BatchRecGroup* g) {
  if (g->mlp) return mlp_batch_forward_kernels(g->mlp, g->B, g->part_len) + 2;
  return g->op.splits > 1 ? 4 : 3;
}

void batch_rec_destroy(BatchRecGroup* g) {
  if (!g) return;
  dev_free(g->d_S);
  dev_free(g->d_part);
  dev_free(g->d_ptrs);
  dev_free(g->d_delay);
  dev_free(g->d_err);
  delete g;
}

}  // namespace pas
