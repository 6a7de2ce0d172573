// Pupil phasor exp(2 pi i opd / lambda) of one OPD sample (the pyramid rows pass).
#pragma once
#include <cuda_runtime.h>

namespace pas {

// opd / lambda in cycles with 1/lambda = inv_hi + inv_lo (two floats): the product
// o * inv_hi is split exactly into hi + err, the whole part of hi removed, and the
// remaining phase in [-1/2, 1/2] cycles (plus the small terms) fed to sincospi.
__device__ __forceinline__ float2 opd_phasor(float o, float inv_hi, float inv_lo) {
  const float hi = __fmul_rn(o, inv_hi);
  const float err = __fmaf_rn(o, inv_hi, -hi);
  const float lo = __fmaf_rn(o, inv_lo, err);
  float sn, cs;
  sincospif(__fmul_rn(2.0f, __fadd_rn(__fsub_rn(hi, rintf(hi)), lo)), &sn, &cs);
  return make_float2(cs, sn);
}

}  // namespace pas
