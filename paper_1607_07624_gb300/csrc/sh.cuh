// Declarations of the Shack-Hartmann sensor shared with the loop translation unit.
#pragma once
#include "internal.h"
#include "pyr.cuh"

namespace pas {

// Frame (may be null) and slopes of d_opd on `st`; `extra` (may be null): the loop's
// residual-WFE fields, closed by the kernel's first CTA. pdl: launched as a
// programmatic dependent of the preceding kernel.
pas_status sh_launch(pas_sh_t sh, const float* d_opd, float* d_frame, float* d_slopes, cudaStream_t st,
                     const LoopExtra* extra, bool pdl);
// Noiseless frame and slopes (calibration measurements), whatever the noise setting.
pas_status sh_measure_noiseless(pas_sh_t sh, const float* d_opd, float* d_frame, float* d_slopes, cudaStream_t st);
int sh_n_slopes(pas_sh_t sh);
int sh_frame_side(pas_sh_t sh);
int sh_np(pas_sh_t sh);

}  // namespace pas
