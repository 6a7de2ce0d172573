// Shared declarations of the atmosphere / DM objects and their kernels.
#pragma once
#include <cuda.h>
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
  // TMA staging of the layer taps (sources at infinity): the screens' tensor map
  // (boxes of 2 rows x RES_BOX floats), the tile's pupil-row segments, the wait
  // bound and the atmosphere's error word. tma = 0: 4-byte asynchronous copies.
  CUtensorMap tmap;
  int tma = 0;
  const int4* seg = nullptr;       // [tiles][seg_max] (row i, first column, pixels, first tile pixel)
  int seg_max = 0;
  unsigned int* err = nullptr;
  uint32_t wait_limit = 0;
};

// Floats per row of a TMA box of the tap staging: a segment of at most RES_TILE pupil
// pixels needs RES_TILE + 1 columns from a start rounded down to 16 bytes.
constexpr int RES_BOX = RES_TILE + 4;
// Shared-memory stride of one box (2 rows): the destinations of tensor copies on 128
// bytes.
constexpr int RES_BOX_PITCH = 160;
// Most pupil-row segments of a tile with TMA staging (more: 4-byte copies).
constexpr int RES_SEG_MAX = 8;
// PAS_TAPS_AUTO stages by TMA for a float32 basis from this many modes up, where a
// tile's basis stream hides the boxes' latency. Measured on GB300 (TMA against the
// 4-byte copies): 408.9 against 409.0 us at 4000 modes with a float32 basis; 220.4
// against 216.2 us with a bf16 one (half the stream); 19.6 against 19.0 and 15.1
// against 14.9 us at 400 modes (one wave of short CTAs).
constexpr int RES_TMA_MIN_MODES = 1000;

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

// Tensor map of L screens of S x S floats for boxes of 2 rows x `box` floats (false if
// the encoder rejects it or is unavailable).
bool make_tmap_rows_f32(CUtensorMap* map, const float* base, uint64_t S, uint64_t L, uint32_t box);

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
  // the screens as a tensor of [L][S][S] floats for TMA boxes of two rows (when S is a
  // multiple of 4 no smaller than a box and the screens start on 16 bytes)
  CUtensorMap tmap;
  bool tma = false;
  unsigned int* d_err = nullptr;  // owned by the base object, shared by its views
  bool owns_err = false;
  uint32_t wait_limit = 1u << 22;
  int taps = PAS_TAPS_AUTO;       // pas_atmo_set_tap_staging
};

struct pas_dm_s {
  pas_ctx_t ctx = nullptr;
  int n_pix = 0, n_modes = 0, Np = 0, n_pad = 0;
  int64_t T_obs = 0;
  float* d_MT = nullptr;            // PAS_FP32 basis
  __nv_bfloat16* d_MTb = nullptr;   // PAS_BF16 basis
  pas_precision prec = PAS_FP32;
  int32_t* d_pix = nullptr;
  // per residual tile: its pupil-row segments (row, first column, pixels, first tile
  // pixel), seg_max per tile, unused entries with 0 pixels
  int4* d_seg = nullptr;
  int seg_max = 0;
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
  a.seg = d->d_seg;
  a.seg_max = d->seg_max;
  return a;
}

// The atmosphere of a residual: its layers, and the TMA staging of their taps when
// the screens allow it and the source is at infinity.
// taps, wait_limit: the staging mode and wait bound the caller took from the
// atmosphere when it was set up (a loop keeps those of its creation).
inline void res_args_set_atmo(ResArgs& a, pas_atmo_t at, int taps, uint32_t wait_limit) {
  a.atmo = at->args;
  const bool want =
      taps == PAS_TAPS_TMA || (taps == PAS_TAPS_AUTO && a.MT != nullptr && a.n_m >= RES_TMA_MIN_MODES);
  a.tma = want && at->tma && !at->args.cone && a.seg != nullptr ? 1 : 0;
  if (a.tma) a.tmap = at->tmap;
  a.err = at->d_err;
  a.wait_limit = wait_limit;
}
}  // namespace pas
