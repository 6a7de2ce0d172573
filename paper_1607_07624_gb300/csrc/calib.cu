// One-off calibration on the GPU (the paper's example calibrates the reconstruction
// matrix before the run, Sec. Example; Table 1 modalrec): the push-pull interaction
// matrix measured through the sensor, its FP64 pseudo-inverse by a one-sided Jacobi
// SVD, and the FP64 products the set-up needs (Gram matrices and basis changes).
//
// Interaction matrix: column m = (s(+a M_m) - s(-a M_m)) / (2a), the sensor's
// noiseless slopes of the DM mode m pushed and pulled by a nm RMS.
//
// Pseudo-inverse: one-sided Jacobi (Hestenes 1958): pairs of columns (i, j) of the
// working copy W of A are rotated until every pair is orthogonal to working
// precision; the rotations accumulate in V, so A = W V^T with orthogonal columns of
// W, sigma_j = |W_j| and U_j = W_j / sigma_j. Then A^+ = V diag(1/sigma_j^2) W^T over
// the sigma_j >= rcond * sigma_max. Each round rotates n/2 disjoint pairs in parallel
// (one CTA per pair) in the round-robin order of the circle method, so a sweep of
// n - 1 rounds meets every pair once; sweeps repeat until one rotates no pair.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "atmo_dm.cuh"
#include "internal.h"
#include "pyr.cuh"
#include "sh.cuh"

namespace pas {

template <typename T>
__device__ __forceinline__ float basis_value(const T* MT, int n_m, int p, int m) {
  return (float)MT[((size_t)(p / RES_TILE) * n_m + m) * RES_TILE + (p % RES_TILE)];
}

// opd[pix[p]] = amp * M(p, m) over the pupil pixels (other pixels untouched).
template <typename T>
__global__ void push_mode_kernel(const T* MT, const int32_t* pix, int n_pix, int n_m, int m, float amp, float* opd) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_pix; p += gridDim.x * blockDim.x)
    opd[pix[p]] = amp * basis_value(MT, n_m, p, m);
}

// IM column: (s_plus - s_minus) / (2 amp) in FP64.
__global__ void im_column_kernel(const float* sp, const float* sm, int ns, double inv_2amp, double* col) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < ns; j += gridDim.x * blockDim.x)
    col[j] = ((double)sp[j] - (double)sm[j]) * inv_2amp;
}

__global__ void eye_kernel(double* V, int n) {
  const size_t tot = (size_t)n * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < tot; t += (size_t)gridDim.x * blockDim.x)
    V[t] = (t / n == t % n) ? 1.0 : 0.0;
}

// Sum over the CTA of three FP64 values (fixed order: warps, then warp 0).
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c, double* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (l == 0) {
    sh[3 * w] = a;
    sh[3 * w + 1] = b;
    sh[3 * w + 2] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0, y = 0, z = 0;
    for (int q = 0; q < nw; ++q) {
      x += sh[3 * q];
      y += sh[3 * q + 1];
      z += sh[3 * q + 2];
    }
    sh[0] = x;
    sh[1] = y;
    sh[2] = z;
  }
  __syncthreads();
  a = sh[0];
  b = sh[1];
  c = sh[2];
}

// One round of the circle method over n_pad (even) columns: CTA b takes the pair
// (r, n_pad - 1) for b = 0, else ((r + b) mod (n_pad - 1), (r - b) mod (n_pad - 1)).
// Columns >= n are padding (never rotated). W: m x n column-major; V: n x n.
__global__ void __launch_bounds__(256) jacobi_round_kernel(double* W, int m, double* V, int n, int n_pad, int r,
                                                           double tol, unsigned int* rotated) {
  __shared__ double sh[3 * 8];
  const int M = n_pad - 1, b = blockIdx.x;
  int i = b == 0 ? r : (r + b) % M;
  int j = b == 0 ? M : ((r - b) % M + M) % M;
  if (i > j) {
    const int t = i;
    i = j;
    j = t;
  }
  if (j >= n) return;  // a padding column
  double* wi = W + (size_t)i * m;
  double* wj = W + (size_t)j * m;
  double al = 0, be = 0, ga = 0;
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const double x = wi[k], y = wj[k];
    al = fma(x, x, al);
    be = fma(y, y, be);
    ga = fma(x, y, ga);
  }
  block_sum3(al, be, ga, sh);
  if (!(fabs(ga) > tol * sqrt(al * be)) || al == 0.0 || be == 0.0) return;
  // rotation making the pair orthogonal: t the smaller root of t^2 + 2 zeta t - 1 = 0
  const double zeta = (be - al) / (2.0 * ga);
  const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const double x = wi[k], y = wj[k];
    wi[k] = c * x - s * y;
    wj[k] = s * x + c * y;
  }
  double* vi = V + (size_t)i * n;
  double* vj = V + (size_t)j * n;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double x = vi[k], y = vj[k];
    vi[k] = c * x - s * y;
    vj[k] = s * x + c * y;
  }
  if (threadIdx.x == 0) atomicAdd(rotated, 1u);
}

__global__ void __launch_bounds__(256) col_norm2_kernel(const double* W, int m, double* out) {
  __shared__ double sh[3 * 8];
  const double* w = W + (size_t)blockIdx.x * m;
  double a = 0, b = 0, c = 0;
  for (int k = threadIdx.x; k < m; k += blockDim.x) a = fma(w[k], w[k], a);
  block_sum3(a, b, c, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = a;
}

// C[i * ldc + k] = sum_j X[i * sxi + j * sxj] * (w ? w[j] : 1) * Y[k * syk + j * syj]
// for i < ni, k < nk, j < nj: FP64, 64 x 64 output tiles, 256 threads x 4 x 4 outputs,
// 16 terms of j staged per round in shared memory.
__global__ void __launch_bounds__(256) gemm_f64_kernel(const double* X, long long sxi, long long sxj,
                                                       const double* Y, long long syk, long long syj,
                                                       const double* w, int ni, int nk, int nj, double* C,
                                                       long long ldc) {
  __shared__ double xs[16][64 + 1];
  __shared__ double ys[16][64 + 1];
  const int i0 = blockIdx.y * 64, k0 = blockIdx.x * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int j0 = 0; j0 < nj; j0 += 16) {
    for (int t = threadIdx.x; t < 16 * 64; t += 256) {
      // consecutive threads walk the output index when that stride is 1, else j
      int jj, ii;
      if (sxi == 1) {
        jj = t / 64;
        ii = t % 64;
      } else {
        ii = t / 16;
        jj = t % 16;
      }
      const int i = i0 + ii, j = j0 + jj;
      double v = 0.0;
      if (i < ni && j < nj) v = X[(long long)i * sxi + (long long)j * sxj] * (w ? w[j] : 1.0);
      xs[jj][ii] = v;
    }
    for (int t = threadIdx.x; t < 16 * 64; t += 256) {
      int jj, kk;
      if (syk == 1) {
        jj = t / 64;
        kk = t % 64;
      } else {
        kk = t / 16;
        jj = t % 16;
      }
      const int k = k0 + kk, j = j0 + jj;
      ys[jj][kk] = (k < nk && j < nj) ? Y[(long long)k * syk + (long long)j * syj] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < 16; ++jj) {
      double xv[4], yv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        xv[u] = xs[jj][ty + 16 * u];
        yv[u] = ys[jj][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(xv[u], yv[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = i0 + ty + 16 * u, k = k0 + tx + 16 * v;
      if (i < ni && k < nk) C[(long long)i * ldc + k] = acc[u][v];
    }
}

static pas_status gemm_f64(pas_ctx_t ctx, const double* X, long long sxi, long long sxj, const double* Y,
                           long long syk, long long syj, const double* w, int ni, int nk, int nj, double* C,
                           long long ldc, cudaStream_t st) {
  const dim3 grid((nk + 63) / 64, (ni + 63) / 64);
  if (grid.y > 65535u) return set_error(ctx, PAS_EINVAL, "FP64 product: %d output rows exceed the grid", ni);
  gemm_f64_kernel<<<grid, 256, 0, st>>>(X, sxi, sxj, Y, syk, syj, w, ni, nk, nj, C, ldc);
  return check_launch(ctx, "FP64 product");
}

}  // namespace pas

extern "C" {

pas_status pas_calib_interaction_matrix(pas_pyr_t pyr, pas_sh_t sh, pas_dm_t dm, double amp_nm, double* d_IM) {
  using namespace pas;
  if (!dm || !d_IM || (!pyr == !sh))
    return set_global_error(PAS_EINVAL, "pas_calib_interaction_matrix: need a DM, d_IM and one sensor");
  pas_ctx_t ctx = dm->ctx;
  PAS_CHECK_ARG(ctx, amp_nm > 0.0 && std::isfinite(amp_nm), "pas_calib_interaction_matrix: amp_nm must be > 0");
  const int Np = pyr ? pyr_np(pyr) : sh_np(sh);
  PAS_CHECK_ARG(ctx, Np == dm->Np, "pas_calib_interaction_matrix: sensor and DM pupils differ");
  const int ns = pyr ? 2 * pyr_n_valid(pyr) : sh_n_slopes(sh);
  const int side = pyr ? pyr_nd(pyr) : sh_frame_side(sh);
  cudaStream_t st = ctx->stream;
  float *opd = nullptr, *frame = nullptr, *sp = nullptr, *sm = nullptr;
  pas_status s = dev_alloc(ctx, (void**)&opd, sizeof(float) * (size_t)Np * Np);
  if (s == PAS_OK) s = dev_alloc(ctx, (void**)&frame, sizeof(float) * (size_t)side * side);
  if (s == PAS_OK) s = dev_alloc(ctx, (void**)&sp, sizeof(float) * ns);
  if (s == PAS_OK) s = dev_alloc(ctx, (void**)&sm, sizeof(float) * ns);
  cudaError_t e = cudaSuccess;
  if (s == PAS_OK) e = cudaMemsetAsync(opd, 0, sizeof(float) * (size_t)Np * Np, st);
  const int pb = std::min(1024, (dm->n_pix + 255) / 256), cb = std::min(1024, (ns + 255) / 256);
  for (int m = 0; m < dm->n_modes && s == PAS_OK && e == cudaSuccess; ++m) {
    for (int sgn = 0; sgn < 2 && s == PAS_OK; ++sgn) {
      const float a = (float)(sgn == 0 ? amp_nm : -amp_nm);
      if (dm->prec == PAS_BF16)
        push_mode_kernel<<<pb, 256, 0, st>>>(dm->d_MTb, dm->d_pix, dm->n_pix, dm->n_modes, m, a, opd);
      else
        push_mode_kernel<<<pb, 256, 0, st>>>(dm->d_MT, dm->d_pix, dm->n_pix, dm->n_modes, m, a, opd);
      float* out = sgn == 0 ? sp : sm;
      s = pyr ? pyr_measure_noiseless(pyr, opd, frame, out, st) : sh_measure_noiseless(sh, opd, frame, out, st);
    }
    if (s == PAS_OK) {
      im_column_kernel<<<cb, 256, 0, st>>>(sp, sm, ns, 0.5 / amp_nm, d_IM + (size_t)m * ns);
      e = cudaGetLastError();
    }
  }
  if (s == PAS_OK && e == cudaSuccess) e = cudaStreamSynchronize(st);
  dev_free(opd);
  dev_free(frame);
  dev_free(sp);
  dev_free(sm);
  if (s != PAS_OK) return s;
  if (e != cudaSuccess)
    return set_error(ctx, PAS_ECUDA, "pas_calib_interaction_matrix: %s", cudaGetErrorString(e));
  return PAS_OK;
}

pas_status pas_pinv_f64(pas_ctx_t ctx, const double* d_A, int32_t m, int32_t n, double rcond, double* d_P,
                        double* h_sv, int32_t* h_rank, int32_t* h_sweeps) {
  using namespace pas;
  if (!ctx || !d_A || !d_P) return set_global_error(PAS_EINVAL, "pas_pinv_f64: NULL argument");
  PAS_CHECK_ARG(ctx, n >= 1 && m >= n, "pas_pinv_f64: need m >= n >= 1");
  PAS_CHECK_ARG(ctx, rcond >= 0.0 && rcond < 1.0, "pas_pinv_f64: rcond in [0, 1)");
  cudaStream_t st = ctx->stream;
  const int n_pad = n + (n & 1);
  double *W = nullptr, *V = nullptr, *sig2 = nullptr, *wts = nullptr;
  unsigned int* rot = nullptr;
  pas_status s = dev_alloc(ctx, (void**)&W, sizeof(double) * (size_t)m * n);
  if (s == PAS_OK) s = dev_alloc(ctx, (void**)&V, sizeof(double) * (size_t)n * n);
  if (s == PAS_OK) s = dev_alloc(ctx, (void**)&sig2, sizeof(double) * n);
  if (s == PAS_OK) s = dev_alloc(ctx, (void**)&wts, sizeof(double) * n);
  if (s == PAS_OK) s = dev_alloc(ctx, (void**)&rot, sizeof(unsigned int));
  cudaError_t e = cudaSuccess;
  auto cleanup = [&]() {
    dev_free(W);
    dev_free(V);
    dev_free(sig2);
    dev_free(wts);
    dev_free(rot);
  };
  if (s != PAS_OK) {
    cleanup();
    return s;
  }
  e = cudaMemcpyAsync(W, d_A, sizeof(double) * (size_t)m * n, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) {
    eye_kernel<<<std::min(4096, (n * n + 255) / 256), 256, 0, st>>>(V, n);
    e = cudaGetLastError();
  }
  // rotate until a whole sweep leaves every pair alone: |W_i . W_j| <= tol |W_i| |W_j|
  const double tol = 8.0 * 2.220446049250313e-16 * std::sqrt((double)m);
  const int max_sweeps = 60;
  int sweeps = 0;
  unsigned int h_rot = 1;
  while (e == cudaSuccess && h_rot != 0 && sweeps < max_sweeps) {
    e = cudaMemsetAsync(rot, 0, sizeof(unsigned int), st);
    for (int r = 0; r < n_pad - 1 && e == cudaSuccess; ++r) {
      jacobi_round_kernel<<<n_pad / 2, 256, 0, st>>>(W, m, V, n, n_pad, r, tol, rot);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_rot, rot, sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    ++sweeps;
  }
  if (e == cudaSuccess && h_rot != 0) {
    cleanup();
    return set_error(ctx, PAS_ETIMEOUT, "pas_pinv_f64: Jacobi rotations did not settle in %d sweeps", max_sweeps);
  }
  std::vector<double> s2(n);
  if (e == cudaSuccess) {
    col_norm2_kernel<<<n, 256, 0, st>>>(W, m, sig2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(s2.data(), sig2, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cleanup();
    return set_error(ctx, PAS_ECUDA, "pas_pinv_f64: %s", cudaGetErrorString(e));
  }
  double smax = 0.0;
  for (int j = 0; j < n; ++j) smax = std::max(smax, std::sqrt(s2[j]));
  std::vector<double> w(n, 0.0);
  int rank = 0;
  for (int j = 0; j < n; ++j) {
    const double sj = std::sqrt(s2[j]);
    if (sj > 0.0 && sj >= rcond * smax) {
      w[j] = 1.0 / s2[j];
      ++rank;
    }
  }
  if (h_sv) {
    std::vector<double> sv(n);
    for (int j = 0; j < n; ++j) sv[j] = std::sqrt(s2[j]);
    std::sort(sv.begin(), sv.end(), [](double a, double b) { return a > b; });
    std::memcpy(h_sv, sv.data(), sizeof(double) * n);
  }
  if (h_rank) *h_rank = rank;
  if (h_sweeps) *h_sweeps = sweeps;
  e = cudaMemcpyAsync(wts, w.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st);
  // P[i][k] = sum_j V[i + j n] w_j W[k + j m]
  if (e == cudaSuccess) s = gemm_f64(ctx, V, 1, n, W, 1, m, wts, n, m, n, d_P, m, st);
  if (e == cudaSuccess && s == PAS_OK) e = cudaStreamSynchronize(st);
  cleanup();
  if (s != PAS_OK) return s;
  if (e != cudaSuccess) return set_error(ctx, PAS_ECUDA, "pas_pinv_f64: %s", cudaGetErrorString(e));
  return PAS_OK;
}

pas_status pas_gemm_f64(pas_ctx_t ctx, const double* d_X, int64_t sxi, int64_t sxj, const double* d_Y, int64_t syk,
                        int64_t syj, const double* d_w, int32_t ni, int32_t nk, int32_t nj, double* d_C,
                        int64_t ldc) {
  using namespace pas;
  if (!ctx || !d_X || !d_Y || !d_C) return set_global_error(PAS_EINVAL, "pas_gemm_f64: NULL argument");
  PAS_CHECK_ARG(ctx, ni >= 0 && nk >= 0 && nj >= 0 && ldc >= nk, "pas_gemm_f64: bad sizes");
  if (ni == 0 || nk == 0) return PAS_OK;
  return gemm_f64(ctx, d_X, sxi, sxj, d_Y, syk, syj, d_w, ni, nk, nj, d_C, ldc, ctx->stream);
}

}  // extern "C"
