// Shared declarations of the atmosphere / DM objects and their kernels.
#pragma once
#include <cuda_bf16.h>
#include "internal.h"

namespace pas {

// Pixels per basis block: the DM basis is stored [tile][mode][RES_TILE], one contiguous
// block per tile of RES_TILE pupil pixels (one residual CTA each).
constexpr int RES_TILE = 64;

struct AtmoArgs {
  const float* screens = nullptr;  // [L][S][S]
  int L = 0, S = 0, Np = 0;
  double vx[PAS_MAX_LAYERS] = {};
  double vy[PAS_MAX_LAYERS] = {};
  double ox[PAS_MAX_LAYERS] = {};  // footprint offsets of an off-axis source [px]
  double oy[PAS_MAX_LAYERS] = {};
  double sc[PAS_MAX_LAYERS] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};  // footprint scales
  int cone = 0;                    // some scale differs from 1 (a source at finite height)
};

struct ResArgs {
  AtmoArgs atmo;                   // L = 0: take opd_atm instead
  const float* opd_atm = nullptr;  // [Np][Np] or null (zero atmosphere)
  const float* MT = nullptr;       // [tiles][n_m][64] basis, one contiguous block per pixel tile
  const __nv_bfloat16* MTb = nullptr;  // the same in bfloat16 (a PAS_BF16 DM); MT then null
  const int* pix = nullptr;        // [n_pix] flat pupil pixel indices
  int n_pix = 0, n_pad = 0, n_m = 0, Np = 0;
  const float* cmd = nullptr;      // [n_m] command
  const float* cmd_ring = nullptr; // [delay][n_m]: slot step % delay used instead
  int delay = 1;
  const long long* d_step = nullptr;
  long long h_step = 0;
  float dm_sign = 1.0f;            // out = atm - dm_sign * M c
  float* out = nullptr;            // [Np][Np], pupil pixels written
  double2* wfe_part = nullptr;     // per-CTA (sum r, sum r^2) or null
};

// One loop of a batched residual (loops sharing one DM object).
struct ResBatchLoop {
  AtmoArgs atmo;                    // on-axis or off-axis source at infinity (no cone)
  const float* cmd_ring = nullptr;  // [delay][n_m]: slot step % delay is subtracted
  int delay = 1;
  const long long* d_step = nullptr;
  float* out = nullptr;             // [Np][Np], pupil pixels written
  double2* wfe_part = nullptr;      // [tiles] (sum r, sum r^2) or null
};

struct ResBatchArgs {
  const float* MT = nullptr;
  const __nv_bfloat16* MTb = nullptr;
  const int* pix = nullptr;
  int n_pix = 0, n_m = 0;
  const ResBatchLoop* loops = nullptr;  // [B] device array
  int B = 0, Bp = 0;                    // loops, padded to whole chunks
  const float* cmdg = nullptr;          // [n_m][Bp] gathered commands
  int Lmax = 0;                         // most layers of a loop
};

// B loops sharing `dm`: residual_j = atm_j - M c_j for all j from one pass over the
// basis per step (gather of the commands, then one kernel); every loop's residual
// and tile WFE partials equal those of its own residual kernel, bit for bit.
struct ResBatch;
bool res_batch_ok(const AtmoArgs& atmo);  // the loop's atmosphere can join a batched residual
pas_status res_batch_create(pas_ctx_t ctx, pas_dm_t dm, int B, const ResBatchLoop* loops, ResBatch** out);
pas_status res_batch_launch(ResBatch* r, cudaStream_t st);
void res_batch_destroy(ResBatch* r);

// pdl: launch as a programmatic dependent of the preceding kernel in `st`.
pas_status residual_launch(pas_ctx_t ctx, const ResArgs& a, cudaStream_t st, bool pdl = false);
// Number of CTAs (and of residual-WFE partials) of residual_launch for n_pix pixels.
int residual_tiles(int n_pix);
// coeffs = (1/n_pix) M^T opd over the pupil pixels (one CTA per mode).
pas_status dm_project_launch(pas_dm_t dm, const float* opd, float* coeffs, cudaStream_t st);

}  // namespace pas

struct pas_atmo_s {
  pas_ctx_t ctx = nullptr;
  pas::AtmoArgs args;
};

struct pas_dm_s {
  pas_ctx_t ctx = nullptr;
  int n_pix = 0, n_modes = 0, Np = 0, n_pad = 0;
  int64_t T_obs = 0;
  float* d_MT = nullptr;            // PAS_FP32 basis
  __nv_bfloat16* d_MTb = nullptr;   // PAS_BF16 basis
  pas_precision prec = PAS_FP32;
  int32_t* d_pix = nullptr;
};

namespace pas {
inline ResArgs make_res_args(pas_dm_t d) {
  ResArgs a;
  a.MT = d->d_MT;
  a.MTb = d->d_MTb;
  a.pix = d->d_pix;
  a.n_pix = d->n_pix;
  a.n_pad = d->n_pad;
  a.n_m = d->n_modes;
  a.Np = d->Np;
  return a;
}
}  // namespace pas
