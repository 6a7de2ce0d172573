// Context, error reporting, device allocation and the host pupil geometry.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "internal.h"

namespace {
thread_local std::string g_global_err;
int g_fail_alloc_after = 0;  // test hook, see pas_debug_fail_alloc_after
}  // namespace

namespace pas {

static std::string vformat(const char* fmt, va_list ap) {
  char buf[1024];
  vsnprintf(buf, sizeof(buf), fmt, ap);
  return std::string(buf);
}

pas_status set_error(pas_ctx_t ctx, pas_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  std::string m = vformat(fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = m;
  g_global_err = m;
  return st;
}

pas_status set_global_error(pas_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  g_global_err = vformat(fmt, ap);
  va_end(ap);
  return st;
}

pas_status dev_alloc(pas_ctx_t ctx, void** p, size_t bytes) {
  *p = nullptr;
  if (g_fail_alloc_after > 0) {
    if (--g_fail_alloc_after == 0)
      return set_error(ctx, PAS_ENOMEM, "injected allocation failure (%zu bytes)", bytes);
  }
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return set_error(ctx, PAS_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
  }
  return PAS_OK;
}

void dev_free(void* p) {
  if (p) cudaFree(p);
}

pas_status check_launch(pas_ctx_t ctx, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(ctx, PAS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
  return PAS_OK;
}

int64_t obstruction_threshold(int Np, double obs) {
  double t = obs * (double)Np;
  return (int64_t)std::ceil(t * t - 1e-9);
}

}  // namespace pas

extern "C" {

int pas_version(void) { return 101; }

pas_status pas_ctx_create(void* cuda_stream, pas_ctx_t* out) {
  if (!out) return pas::set_global_error(PAS_EINVAL, "pas_ctx_create: out is NULL");
  *out = nullptr;
  pas_ctx_t c = new pas_ctx_s();
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete c;
    cudaGetLastError();
    return pas::set_global_error(PAS_ECUDA, "pas_ctx_create: %s", cudaGetErrorString(e));
  }
  c->stream = (cudaStream_t)cuda_stream;
  *out = c;
  return PAS_OK;
}

void pas_ctx_destroy(pas_ctx_t ctx) {
  if (!ctx) return;
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  delete ctx;
}

pas_status pas_ctx_set_stream(pas_ctx_t ctx, void* cuda_stream) {
  if (!ctx) return pas::set_global_error(PAS_EINVAL, "pas_ctx_set_stream: NULL context");
  ctx->stream = (cudaStream_t)cuda_stream;
  return PAS_OK;
}

pas_status pas_ctx_synchronize(pas_ctx_t ctx) {
  if (!ctx) return pas::set_global_error(PAS_EINVAL, "pas_ctx_synchronize: NULL context");
  PAS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return PAS_OK;
}

const char* pas_last_error(pas_ctx_t ctx) { return ctx ? ctx->err.c_str() : g_global_err.c_str(); }
const char* pas_global_error(void) { return g_global_err.c_str(); }

void pas_debug_fail_alloc_after(int n) { g_fail_alloc_after = n < 0 ? 0 : n; }

pas_status pas_pupil_mask(int Np, double obs, uint8_t* mask, int32_t* n_pix) {
  if (Np <= 0 || !(obs >= 0.0 && obs < 1.0))
    return pas::set_global_error(PAS_EINVAL, "pas_pupil_mask: bad Np or obs");
  int64_t T = pas::obstruction_threshold(Np, obs);
  int32_t n = 0;
  for (int i = 0; i < Np; ++i)
    for (int j = 0; j < Np; ++j) {
      bool in = pas::in_pupil(i, j, Np, T);
      if (mask) mask[(size_t)i * Np + j] = in ? 1 : 0;
      n += in;
    }
  if (n_pix) *n_pix = n;
  return PAS_OK;
}

pas_status pas_pupil_pixels(int Np, double obs, int32_t* idx, int32_t cap, int32_t* n_pix) {
  if (Np <= 0 || !(obs >= 0.0 && obs < 1.0))
    return pas::set_global_error(PAS_EINVAL, "pas_pupil_pixels: bad Np or obs");
  int64_t T = pas::obstruction_threshold(Np, obs);
  int32_t n = 0;
  for (int i = 0; i < Np; ++i)
    for (int j = 0; j < Np; ++j)
      if (pas::in_pupil(i, j, Np, T)) {
        if (idx) {
          if (n >= cap) return pas::set_global_error(PAS_EINVAL, "pas_pupil_pixels: cap too small");
          idx[n] = i * Np + j;
        }
        ++n;
      }
  if (n_pix) *n_pix = n;
  return PAS_OK;
}

pas_status pas_valid_subaps(int Np, double obs, int n_sub, int32_t* valid, int32_t cap,
                            int32_t* n_valid) {
  if (Np <= 0 || n_sub <= 0 || n_sub > Np || !(obs >= 0.0 && obs < 1.0))
    return pas::set_global_error(PAS_EINVAL, "pas_valid_subaps: need 0 < n_sub <= Np and 0 <= obs < 1");
  // Sub-aperture (r, c) covers pupil pixels [r b, (r+1) b) x [c b, (c+1) b), b = Np / n_sub
  // not necessarily an integer. Scaled by n_sub every end is an integer, and the overlap
  // of pixel i with row r is o(i) = |[i n_sub, (i+1) n_sub) & [r Np, (r+1) Np)| in units of
  // 1/n_sub. Valid iff 2 * sum over pupil pixels of o_r(i) o_c(j) >= Np^2, i.e. twice the
  // pupil area reaches b^2 (for integer b: 2 * pixel count >= b^2).
  auto ovl = [&](int i, int s) -> int64_t {
    const int64_t lo = std::max((int64_t)i * n_sub, (int64_t)s * Np);
    const int64_t hi = std::min((int64_t)(i + 1) * n_sub, (int64_t)(s + 1) * Np);
    return hi > lo ? hi - lo : 0;
  };
  int64_t T = pas::obstruction_threshold(Np, obs);
  int32_t n = 0;
  for (int r = 0; r < n_sub; ++r) {
    const int i0 = (int)(((int64_t)r * Np) / n_sub), i1 = (int)(((int64_t)(r + 1) * Np + n_sub - 1) / n_sub);
    for (int c = 0; c < n_sub; ++c) {
      const int j0 = (int)(((int64_t)c * Np) / n_sub), j1 = (int)(((int64_t)(c + 1) * Np + n_sub - 1) / n_sub);
      int64_t A = 0;
      for (int i = i0; i < i1; ++i) {
        const int64_t oi = ovl(i, r);
        for (int j = j0; j < j1; ++j)
          if (pas::in_pupil(i, j, Np, T)) A += oi * ovl(j, c);
      }
      if (2 * A >= (int64_t)Np * Np) {
        if (valid) {
          if (n >= cap) return pas::set_global_error(PAS_EINVAL, "pas_valid_subaps: cap too small");
          valid[n] = r * n_sub + c;
        }
        ++n;
      }
    }
  }
  if (n_valid) *n_valid = n;
  return PAS_OK;
}

}  // extern "C"
