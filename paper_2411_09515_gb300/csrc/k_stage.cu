// Staging of a batch: every pixel that the integration matrix uses is
// corrected once (Section 1.2, divided by its norm, Eq. 1) and written to
// its staging position, where the clip kernel reads it.
//
// One CTA per staging tile (kTileH x kTileW pixels of the image) and group
// of frames. Raw words and calibration planes are read in image order
// (consecutive threads on consecutive pixels); the tile's values are placed
// in shared memory at their rank inside the tile, then written out as one
// contiguous run. Each value is the same IEEE sequence as pixel_value():
// RN32(RN32(adc - pedestal) / gain), then RN32(. / norm).
#include <cuda_runtime.h>
#include <stdint.h>

#include "sep_device.cuh"
#include "sep_internal.h"

namespace sep {
namespace {

constexpr int kStageThreads = 256;
constexpr int kTilePix = kTileH * kTileW;
constexpr int kPerThread = kTilePix / kStageThreads;
static_assert(kTilePix % kStageThreads == 0, "tile size");

template <int DT, bool NORM>
__global__ void __launch_bounds__(kStageThreads) k_stage(StageArgs a) {
  __shared__ float tv[kTilePix];
  const int t = blockIdx.x;
  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)(t / a.tiles_x) * kTileH, c0 = (int64_t)(t % a.tiles_x) * kTileW;
  const int base = __ldg(a.tile_base + t), cnt = __ldg(a.tile_base + t + 1) - base;
  if (cnt == 0) return;
  int64_t pix[kPerThread];
  int rank[kPerThread];
  float p0[kPerThread], g0[kPerThread], nm[kPerThread];
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    const int idx = tid + k * kStageThreads;
    const int64_t r = r0 + idx / kTileW, c = c0 + idx % kTileW;
    rank[k] = -1;
    pix[k] = 0;
    p0[k] = 0.0f;
    g0[k] = 1.0f;
    nm[k] = 1.0f;
    if (r < a.rows && c < a.cols) {
      pix[k] = r * a.cols + c;
      rank[k] = __ldg(a.tile_rank + pix[k]);
      if (rank[k] >= 0) {
        if (DT == SEP_DTYPE_U16_JF) {
          p0[k] = __ldg(a.ped + pix[k]);
          g0[k] = __ldg(a.gain + pix[k]);
        }
        if (NORM) nm[k] = __ldg(a.norm + pix[k]);
      }
    }
  }
  const int f0 = blockIdx.y * a.frames_per_cta;
  const int f1 = min(f0 + a.frames_per_cta, a.n_frames);
  for (int f = f0; f < f1; ++f) {
    const void* frame = a.fptr ? (const void*)a.fptr[f] : frame_ptr<DT>(a.frames, f, a.npix);
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
      if (rank[k] < 0) continue;
      float x;
      if (DT == SEP_DTYPE_U16_JF) {
        const uint32_t u = __ldg(reinterpret_cast<const uint16_t*>(frame) + pix[k]);
        const uint32_t code = u >> 14;
        float ped = p0[k], gain = g0[k];
        if (code != 0) {   // gain levels 1 and 2
          const int64_t lvl = code == 1 ? 1 : 2;
          ped = __ldg(a.ped + lvl * a.npix + pix[k]);
          gain = __ldg(a.gain + lvl * a.npix + pix[k]);
        }
        x = __fdiv_rn(__fsub_rn((float)(u & 0x3FFFu), ped), gain);
      } else {
        x = __ldg(reinterpret_cast<const float*>(frame) + pix[k]);
      }
      if (NORM) x = __fdiv_rn(x, nm[k]);
      tv[rank[k]] = x;
    }
    __syncthreads();
    float* out = a.stage + (int64_t)f * a.npos + base;
    for (int j = tid; j < cnt; j += kStageThreads) out[j] = tv[j];
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_stage(const StageArgs& a, int32_t dtype, bool has_norm, cudaStream_t s) {
  if (a.n_frames <= 0) return cudaSuccess;
  const int n_tiles = a.tiles_x * a.tiles_y;
  dim3 grid(n_tiles, (a.n_frames + a.frames_per_cta - 1) / a.frames_per_cta);
  if (dtype == SEP_DTYPE_U16_JF) {
    if (has_norm) k_stage<SEP_DTYPE_U16_JF, true><<<grid, kStageThreads, 0, s>>>(a);
    else k_stage<SEP_DTYPE_U16_JF, false><<<grid, kStageThreads, 0, s>>>(a);
  } else {
    if (has_norm) k_stage<SEP_DTYPE_F32, true><<<grid, kStageThreads, 0, s>>>(a);
    else k_stage<SEP_DTYPE_F32, false><<<grid, kStageThreads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace sep
