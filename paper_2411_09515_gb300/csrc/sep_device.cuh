// Device helpers shared by the libsep kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sep.h"

namespace sep {

// Corrected value of pixel `col` of one frame (Section 1.2 and Eq. 1).
// Raw Jungfrau words: the two top bits select the gain level (code 0 -> 0,
// code 1 -> 1, codes 2 and 3 -> 2) and the low 14 bits are the ADC value;
// photons = RN32(RN32(adc - pedestal) / gain), IEEE round-to-nearest without
// fused or approximate operations. A per-pixel norm divides the result.
template <int DT, bool NORM>
__device__ __forceinline__ float pixel_value(const void* frame, int64_t col, int64_t npix, const float* ped,
                                             const float* gain, const float* norm) {
  float p;
  if (DT == SEP_DTYPE_U16_JF) {
    uint32_t u = __ldg(reinterpret_cast<const uint16_t*>(frame) + col);
    uint32_t code = u >> 14;
    int64_t lvl = code == 0 ? 0 : (code == 1 ? 1 : 2);
    float adc = (float)(u & 0x3FFFu);
    float x = __fsub_rn(adc, __ldg(ped + lvl * npix + col));
    p = __fdiv_rn(x, __ldg(gain + lvl * npix + col));
  } else {
    p = __ldg(reinterpret_cast<const float*>(frame) + col);
  }
  if (NORM) p = __fdiv_rn(p, __ldg(norm + col));
  return p;
}

template <int DT>
__device__ __forceinline__ const void* frame_ptr(const void* frames, int64_t f, int64_t npix) {
  if (DT == SEP_DTYPE_U16_JF) return reinterpret_cast<const uint16_t*>(frames) + f * npix;
  return reinterpret_cast<const float*>(frames) + f * npix;
}

}  // namespace sep
