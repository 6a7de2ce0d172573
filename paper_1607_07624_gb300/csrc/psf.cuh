// PSF camera launches shared with the loop control.
#pragma once
#include "internal.h"

namespace pas {

// The camera's two passes on `st`: PSF of d_opd written to (accumulate = 0) or added to
// d_psf, its Strehl ratio to d_strehl (or nowhere). With d_step: nothing happens before
// step `start`, and the Strehl ratio of step t goes to d_strehl[t mod sr_len] (a camera
// inside a loop's step graph, the step counter read on the device).
pas_status psf_launch(pas_psf_t P, const float* d_opd, float* d_psf, int accumulate, double* d_strehl,
                      const long long* d_step, long long start, int sr_len, cudaStream_t st);
int psf_np(pas_psf_t P);

}  // namespace pas
