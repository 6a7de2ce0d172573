// Declarations shared between the pyramid and loop translation units.
#pragma once
#include "internal.h"

namespace pas {

struct FrameArgs {
  const float* part;    // [G][nd*nd]
  float* frame;         // [nd*nd]
  const int* valid;     // [nv]
  const float* sn;      // [2nv] or null
  float* slopes;        // [2nv] or null
  int G, nd, n_sub, nv, local_norm;
  float invK;
  // noise
  double photon_scale;  // photons / n_pupil_pixels (<= 0: off)
  double ron;
  unsigned long long seed;
  long long* frame_ctr;  // device counter
  int ctr_increment;
  // residual WFE of the loop (optional)
  const double2* wfe_part;  // [n_wfe_part] (sum, sum of squares)
  int n_wfe_part;
  double inv_npix;
  double* wfe_hist;
  int wfe_hist_len;
  const long long* step;
};

// Launch rows pass, cols pass and frame/slopes on `st`. `extra` (may be null)
// supplies the loop's frame counter and residual-WFE fields. `ev` (may be null):
// three events recorded before the rows, cols and frame kernels.
pas_status pyr_launch(pas_pyr_t y, const float* d_opd, float* d_frame, float* d_slopes,
                      cudaStream_t st, FrameArgs* extra, bool increment_ctr,
                      cudaEvent_t* ev = nullptr);
int pyr_n_pupil(pas_pyr_t y);
int pyr_nd(pas_pyr_t y);

}  // namespace pas
