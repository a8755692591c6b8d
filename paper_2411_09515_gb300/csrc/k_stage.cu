// Staging of a batch: every pixel that the integration matrix uses is
// corrected once (Section 1.2, divided by its norm, Eq. 1) and written to
// its staging position, where the clip kernel reads it.
//
// One CTA per staging tile (kTileH x kTileW pixels of the image) and group
// of frames. Threads read tile rows: each thread four consecutive pixels
// (one vector load where the row is aligned), two frames per step; the
// tile's values are placed in shared memory at their rank inside the tile,
// then written out as one contiguous run. Each value is the same IEEE sequence as pixel_value():
// RN32(RN32(adc - pedestal) / gain), then RN32(. / norm).
#include <cuda_runtime.h>
#include <stdint.h>

#include "sep_device.cuh"
#include "sep_internal.h"

namespace sep {
namespace {

constexpr int kTilePix = kTileH * kTileW;
constexpr int kStageThreads = kTilePix / 4;   // 4 consecutive pixels of one row a thread
constexpr int kRowThreads = kTileW / 4;       // threads covering one tile row
static_assert(kTileW % 4 == 0 && kStageThreads % 32 == 0 && kStageThreads <= 1024, "tile shape");

// Four consecutive raw words / values of one frame (VEC: one aligned vector load).
template <int DT, bool VEC>
__device__ __forceinline__ void load4(const void* frame, int64_t p, bool (&in)[4], uint32_t (&w)[4]) {
  if (DT == SEP_DTYPE_U16_JF) {
    const uint16_t* f = reinterpret_cast<const uint16_t*>(frame);
    if (VEC) {
      const uint2 v = __ldg(reinterpret_cast<const uint2*>(f + p));
      w[0] = v.x & 0xffffu; w[1] = v.x >> 16; w[2] = v.y & 0xffffu; w[3] = v.y >> 16;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) w[k] = in[k] ? __ldg(f + p + k) : 0u;
    }
  } else {
    const float* f = reinterpret_cast<const float*>(frame);
    if (VEC) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(f + p));
      w[0] = __float_as_uint(v.x); w[1] = __float_as_uint(v.y); w[2] = __float_as_uint(v.z); w[3] = __float_as_uint(v.w);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) w[k] = in[k] ? __float_as_uint(__ldg(f + p + k)) : 0u;
    }
  }
}

template <int DT, bool NORM, bool VEC>
__global__ void __launch_bounds__(kStageThreads) k_stage(StageArgs a) {
  __shared__ float tv[2][kTilePix];
  const int t = blockIdx.x;
  const int tid = threadIdx.x;
  const int base = __ldg(a.tile_base + t), cnt = __ldg(a.tile_base + t + 1) - base;
  if (t == 0 && tid == 0) {   // the NaN slot of padding entries, once per frame
    const int f1n = min((int)(blockIdx.y + 1) * a.frames_per_cta, a.n_frames);
    for (int f = blockIdx.y * a.frames_per_cta; f < f1n; ++f)
      a.stage[(int64_t)f * a.npos + a.nan_pos] = __int_as_float(0x7fc00000);
  }
  if (cnt == 0) return;
  const int64_t r = (int64_t)(t / a.tiles_x) * kTileH + tid / kRowThreads;
  const int64_t c = (int64_t)(t % a.tiles_x) * kTileW + 4 * (tid % kRowThreads);
  const int64_t p = r * a.cols + c;    // first of this thread's 4 pixels
  bool in[4];
  int rank[4];
  float p0[4], g0[4], nm[4];
  bool any = false;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    in[k] = r < a.rows && c + k < a.cols;
    rank[k] = in[k] ? __ldg(a.tile_rank + p + k) : -1;
    any = any || rank[k] >= 0;
    p0[k] = 0.0f;
    g0[k] = 1.0f;
    nm[k] = 1.0f;
    if (rank[k] >= 0) {
      if (DT == SEP_DTYPE_U16_JF) {
        p0[k] = __ldg(a.ped + p + k);
        g0[k] = __ldg(a.gain + p + k);
      }
      if (NORM) nm[k] = __ldg(a.norm + p + k);
    }
  }
  const int f0 = blockIdx.y * a.frames_per_cta;
  const int f1 = min(f0 + a.frames_per_cta, a.n_frames);
  // two frames per step: both frames' loads are in flight together
  for (int f = f0; f < f1; f += 2) {
    const int nf = min(2, f1 - f);
    uint32_t w[2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h < nf && any) {
        const void* frame = a.fptr ? (const void*)a.fptr[f + h] : frame_ptr<DT>(a.frames, f + h, a.npix);
        load4<DT, VEC>(frame, p, in, w[h]);
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h >= nf) continue;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (rank[k] < 0) continue;
        float x;
        if (DT == SEP_DTYPE_U16_JF) {
          const uint32_t u = w[h][k], code = u >> 14;
          float ped = p0[k], gain = g0[k];
          if (code != 0) {   // gain levels 1 and 2
            const int64_t lvl = code == 1 ? 1 : 2;
            ped = __ldg(a.ped + lvl * a.npix + p + k);
            gain = __ldg(a.gain + lvl * a.npix + p + k);
          }
          x = __fdiv_rn(__fsub_rn((float)(u & 0x3FFFu), ped), gain);
        } else {
          x = __uint_as_float(w[h][k]);
        }
        if (NORM) x = __fdiv_rn(x, nm[k]);
        tv[h][rank[k]] = x;
      }
    }
    __syncthreads();
    for (int h = 0; h < nf; ++h) {
      float* out = a.stage + (int64_t)(f + h) * a.npos + base;
      for (int j = tid; j < cnt; j += kStageThreads) out[j] = tv[h][j];
    }
    __syncthreads();
  }
}

template <int DT, bool NORM>
void launch_v(const StageArgs& a, dim3 grid, bool vec, cudaStream_t s) {
  if (vec) k_stage<DT, NORM, true><<<grid, kStageThreads, 0, s>>>(a);
  else k_stage<DT, NORM, false><<<grid, kStageThreads, 0, s>>>(a);
}

}  // namespace

cudaError_t launch_stage(const StageArgs& a, int32_t dtype, bool has_norm, cudaStream_t s) {
  if (a.n_frames <= 0) return cudaSuccess;
  const int n_tiles = a.tiles_x * a.tiles_y;
  dim3 grid(n_tiles, (a.n_frames + a.frames_per_cta - 1) / a.frames_per_cta);
  // vector loads need every thread's 4 pixels aligned: a column count that
  // is a multiple of 4 (tiles start at multiples of 128), frames contiguous
  // or listed at 16-byte aligned addresses
  bool vec = a.cols % 4 == 0;
  if (!a.fptr) vec = vec && ((uintptr_t)a.frames % 16 == 0);
  if (dtype == SEP_DTYPE_U16_JF) {
    if (has_norm) launch_v<SEP_DTYPE_U16_JF, true>(a, grid, vec && !a.fptr, s);
    else launch_v<SEP_DTYPE_U16_JF, false>(a, grid, vec && !a.fptr, s);
  } else {
    if (has_norm) launch_v<SEP_DTYPE_F32, true>(a, grid, vec && !a.fptr, s);
    else launch_v<SEP_DTYPE_F32, false>(a, grid, vec && !a.fptr, s);
  }
  return cudaGetLastError();
}

}  // namespace sep
