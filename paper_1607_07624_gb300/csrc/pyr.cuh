// Declarations shared between the pyramid and loop translation units.
#pragma once
#include "internal.h"

namespace pas {

// What the loop adds to a pyramid measurement: the noise frame counter it owns
// and the residual-WFE finalisation of the step.
struct LoopExtra {
  long long* frame_ctr = nullptr;       // counter used for the noise (loop: the step)
  const double2* wfe_part = nullptr;    // per-CTA (sum r, sum r^2) of the residual
  int n_wfe_part = 0;
  double inv_npix = 0.0;
  double* wfe_hist = nullptr;
  int wfe_hist_len = 1;
  const long long* step = nullptr;
  // a detector integrating n_int steps per frame (n_int > 1, loops): the noiseless
  // frames add up in acc [frame pixels] and are read out at the steps t with
  // (t + 1) mod n_int = 0 (frame_ctr holds t)
  float* acc = nullptr;
  int n_int = 1;
};

// Launch rows pass, cols pass and frame/slopes on `st`. `extra` (may be null)
// supplies the loop's frame counter and residual-WFE fields. `ev` (may be null):
// three events recorded before the rows, columns and slopes kernels (the kernels are
// then launched without programmatic dependence). pdl_first: the rows pass itself
// follows a kernel programmatically.
pas_status pyr_launch(pas_pyr_t y, const float* d_opd, float* d_frame, float* d_slopes,
                      cudaStream_t st, const LoopExtra* extra, bool increment_ctr,
                      cudaEvent_t* ev = nullptr, bool pdl_first = false);
// Noiseless frame and slopes of d_opd on `st` (the sensor's reference subtracted),
// whatever noise the object is set to: calibration measurements.
pas_status pyr_measure_noiseless(pas_pyr_t y, const float* d_opd, float* d_frame, float* d_slopes, cudaStream_t st);
// Persistent batched launch of several pyramids' rows and columns passes (one
// launch per transform length; each task is one CTA of the pyramid's own launches,
// so the frames equal those measured alone). Per member: its OPD, frame and slopes
// buffers and loop fields (as pyr_launch takes them, counter not incremented).
struct PyrBatch;
constexpr long long PAS_BATCH_WAIT_DEFAULT = 1ll << 21;  // polls: about a second
pas_status pyr_batch_create(pas_ctx_t ctx, int n, const pas_pyr_t* y, const float* const* opd, float* const* frame,
                            float* const* slopes, const LoopExtra* extra, PyrBatch** out);
pas_status pyr_batch_launch(PyrBatch* b, cudaStream_t st, bool columns_only = false);
// Group g alone (its counters zeroed first); the groups are independent.
pas_status pyr_batch_launch_group(PyrBatch* b, int g, cudaStream_t st, bool columns_only = false);
int pyr_batch_group_of(const PyrBatch* b, int i);  // member i's group (transform length)
// h[8]: N, CTAs, threads per CTA, shared bytes, rows per rows task, sin chunk,
// rows tasks, columns tasks of group g
void pyr_batch_geometry(const PyrBatch* b, int g, int* h);
pas_status pyr_batch_slopes(PyrBatch* b, int i, cudaStream_t st, bool pdl);
int pyr_batch_n_groups(const PyrBatch* b);
unsigned int* pyr_batch_err(PyrBatch* b);
long long* pyr_batch_wait_limit(PyrBatch* b);
void pyr_batch_destroy(PyrBatch* b);
int pyr_n_valid(pas_pyr_t y);
int pyr_n_pupil(pas_pyr_t y);
int pyr_nd(pas_pyr_t y);
int pyr_np(pas_pyr_t y);

}  // namespace pas
