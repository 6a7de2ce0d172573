// Reconstructor object and kernel arguments (shared with the loop).
#pragma once
#include <cuda_bf16.h>

#include "internal.h"

namespace pas {

struct ReconArgs {
  const float* R = nullptr;             // [n_m][n_s_pad] float32
  const __nv_bfloat16* Rb = nullptr;    // [n_m][n_s_pad] bfloat16 (row-scaled)
  const float* scale = nullptr;         // [n_m]
  int n_m = 0, n_s = 0, n_s_pad = 0;
  const float* s = nullptr;             // [n_s] slopes
  float* dmodes = nullptr;              // [n_m] out (may be null)
  // integrator (active when ring != null)
  const float* gain = nullptr;          // [n_m] or null (gain 1)
  float* ring = nullptr;                // [delay][n_m]
  int delay = 1;
  const long long* step = nullptr;
  float* cmd_last = nullptr;            // [n_m] copy of the new command
  long long* step_inc = nullptr;        // advanced by one after the last CTA (or null)
  unsigned int* done = nullptr;         // CTA completion counter
  int n_int = 1;                        // > 1: new command only when (step + 1) mod n_int = 0
  unsigned int* err = nullptr;          // wait-timeout flags (bulk-copy kernel)
};

}  // namespace pas

struct pas_recon_s {
  pas_ctx_t ctx = nullptr;
  int n_modes = 0, n_slopes = 0, n_s_pad = 0;
  pas_precision prec = PAS_FP32;
  float* d_R = nullptr;
  __nv_bfloat16* d_Rb = nullptr;
  float* d_scale = nullptr;
  unsigned int* d_done = nullptr;
  unsigned int* d_err = nullptr;
  int rt_rows = 0, rt_slots = 0;        // TMA row pipeline: rows per CTA (0: not used), row slots
};

namespace pas {
pas_status recon_launch(pas_recon_t r, ReconArgs a, cudaStream_t st, bool pdl = false);
}
