// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <cstdarg>
#include <cstdint>
#include <string>

#include "pas.h"

#define PAS_MAX_LAYERS 16

struct pas_ctx_s {
  cudaStream_t stream = nullptr;          // borrowed
  cudaStream_t capture_stream = nullptr;  // owned: graph capture only
  int device = 0;
  int sm_count = 0;
  std::string err;
};

namespace pas {

pas_status set_error(pas_ctx_t ctx, pas_status st, const char* fmt, ...);
pas_status set_global_error(pas_status st, const char* fmt, ...);
// cudaMalloc with the test fault-injection hook; on failure records PAS_ENOMEM.
pas_status dev_alloc(pas_ctx_t ctx, void** p, size_t bytes);
void dev_free(void* p);
// Raise (never lower) a kernel's dynamic shared-memory limit.
cudaError_t raise_dyn_smem(const void* func, size_t bytes);
// Check the last launch; records PAS_ECUDA with `what`.
pas_status check_launch(pas_ctx_t ctx, const char* what);

// Pupil geometry (integer-exact, host).
int64_t obstruction_threshold(int Np, double obs);
inline bool in_pupil(int i, int j, int Np, int64_t T) {
  int64_t a = 2 * (int64_t)i - Np + 1, b = 2 * (int64_t)j - Np + 1;
  int64_t d2 = a * a + b * b;
  return d2 <= (int64_t)Np * Np && d2 >= T;
}

}  // namespace pas

#define PAS_CHECK_ARG(ctx, cond, msg)                                   \
  do {                                                                  \
    if (!(cond)) return pas::set_error((ctx), PAS_EINVAL, "%s", (msg)); \
  } while (0)

#define PAS_CUDA_TRY(ctx, call)                                                        \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return pas::set_error((ctx), PAS_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)
