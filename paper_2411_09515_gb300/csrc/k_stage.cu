// Staging of a batch: every pixel of the image is corrected once per frame
// (Section 1.2, divided by its norm, Eq. 1) and its value is written to the
// slots of its matrix entries in the frame's staged row (slot e holds entry
// e's value, padding slots NaN), so the clip kernel reads each bin's values
// as one contiguous run.
//
// One CTA per image tile (kTileH x kTileW pixels) and group of frames.
// Threads read tile rows: each thread four consecutive pixels (one vector
// load where the row is aligned), two frames per step (four in the ring
// kernel); the corrected tile sits in shared memory by pixel, then the
// tile's list of (slot, pixel) pairs, ascending by slot, writes it out (the
// entries of one bin inside a tile occupy consecutive slots). Each value is
// the same IEEE sequence as pixel_value(): RN32(RN32(adc - pedestal) /
// gain), then RN32(. / norm).
#include <cuda_runtime.h>
#include <stdint.h>

#include "sep_device.cuh"
#include "sep_internal.h"

namespace sep {
namespace {

constexpr int kTilePix = kTileH * kTileW;
constexpr int kTileSlots = kTilePix + 4;   // the tile's values, then a NaN (padding slots read it)
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

// The tile's (slot, shared-memory index) pairs a thread writes: pairs tid +
// kStageThreads k for k < kScReg stay in registers for every frame, longer
// lists read the rest at each scatter. Padding pairs point at the NaN.
constexpr int kScReg = 8;

struct TileScatter {
  int slot[kScReg], loc[kScReg];
  int n;   // pairs held
  __device__ __forceinline__ void load(const StageArgs& a, int eb, int ne) {
    n = 0;
#pragma unroll
    for (int k = 0; k < kScReg; ++k) {
      const int j = threadIdx.x + kStageThreads * k;
      int2 sc = make_int2(0, kTilePix);
      if (j < ne) {
        sc = __ldg(a.tile_sc + eb + j);
        n = k + 1;
      }
      slot[k] = sc.x;
      loc[k] = sc.y >= 0 ? sc.y : kTilePix;
    }
  }
};

// Scatter of NF corrected tiles (tv[h]) of frames f .. f + NF - 1 (the
// first nf of them) to their entries' slots.
template <int NF>
__device__ __forceinline__ void scatter_tile(const StageArgs& a, const TileScatter& ts, const float (*tv)[kTileSlots],
                                             int eb, int ne, int64_t f, int nf) {
  float* out[NF];
#pragma unroll
  for (int h = 0; h < NF; ++h) out[h] = a.stage + (f + min(h, nf - 1)) * a.npos;
#pragma unroll
  for (int k = 0; k < kScReg; ++k) {
    if (k >= ts.n) break;
#pragma unroll
    for (int h = 0; h < NF; ++h)
      if (h < nf) out[h][ts.slot[k]] = tv[h][ts.loc[k]];
  }
  for (int j = threadIdx.x + kStageThreads * kScReg; j < ne; j += kStageThreads) {
    const int2 sc = __ldg(a.tile_sc + eb + j);
    const int l = sc.y >= 0 ? sc.y : kTilePix;
#pragma unroll
    for (int h = 0; h < NF; ++h)
      if (h < nf) out[h][sc.x] = tv[h][l];
  }
}

template <int DT, bool NORM, bool VEC>
__global__ void __launch_bounds__(kStageThreads) k_stage(StageArgs a) {
  __shared__ float tv[2][kTileSlots];
  const int t = blockIdx.x;
  const int tid = threadIdx.x;
  const int eb = __ldg(a.tile_ebase + t), ne = __ldg(a.tile_ebase + t + 1) - eb;
  if (ne == 0) return;
  if (tid < 2) tv[tid][kTilePix] = __int_as_float(0x7fc00000);
  TileScatter ts;
  ts.load(a, eb, ne);
  const int loc0 = (tid / kRowThreads) * kTileW + 4 * (tid % kRowThreads);   // this thread's pixels in the tile
  const int64_t r = (int64_t)(t / a.tiles_x) * kTileH + tid / kRowThreads;
  const int64_t c = (int64_t)(t % a.tiles_x) * kTileW + 4 * (tid % kRowThreads);
  const int64_t p = r * a.cols + c;    // first of this thread's 4 pixels
  bool in[4];
  float p0[4], g0[4], nm[4];
  bool any = false;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    in[k] = r < a.rows && c + k < a.cols;
    any = any || in[k];
    p0[k] = 0.0f;
    g0[k] = 1.0f;
    nm[k] = 1.0f;
    if (in[k]) {
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
        if (!in[k]) continue;
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
        tv[h][loc0 + k] = x;
      }
    }
    __syncthreads();
    scatter_tile<2>(a, ts, tv, eb, ne, f, nf);
    __syncthreads();
  }
}

// The aligned case with the frames' loads ahead of their use: each thread
// copies its four raw words (8 bytes; 16 for FP32 input) of the next frames
// into its own slots of a ring in shared memory (cp.async, no registers
// held), kRing frames ahead, and reads them back when their frame comes.
// A thread reads only what it copied itself, so the ring needs no barrier.
// Four frames per step share the two barriers around the write-out.
constexpr int kRing = 8;   // frames ahead (a multiple of the 4 frames of a step)

// Dynamic shared memory of k_stage_ring: four corrected tiles, then the ring.
template <int DT>
constexpr size_t ring_smem_bytes() {
  return sizeof(float) * 4 * kTileSlots + (size_t)kRing * kStageThreads * (DT == SEP_DTYPE_U16_JF ? 8 : 16);
}

template <int DT, bool NORM>
__global__ void __launch_bounds__(kStageThreads) k_stage_ring(StageArgs a) {
  constexpr int kVec = DT == SEP_DTYPE_U16_JF ? 8 : 16;   // bytes of 4 raw words
  extern __shared__ __align__(16) unsigned char stage_smem[];
  float(*tv)[kTileSlots] = reinterpret_cast<float(*)[kTileSlots]>(stage_smem);
  unsigned char(*ring)[kStageThreads * kVec] =
      reinterpret_cast<unsigned char(*)[kStageThreads * kVec]>(stage_smem + sizeof(float) * 4 * kTileSlots);
  const int t = blockIdx.x;
  const int tid = threadIdx.x;
  const int eb = __ldg(a.tile_ebase + t), ne = __ldg(a.tile_ebase + t + 1) - eb;
  if (ne == 0) return;
  if (tid < 4) tv[tid][kTilePix] = __int_as_float(0x7fc00000);
  TileScatter ts;
  ts.load(a, eb, ne);
  const int loc0 = (tid / kRowThreads) * kTileW + 4 * (tid % kRowThreads);   // this thread's pixels in the tile
  const int64_t r = (int64_t)(t / a.tiles_x) * kTileH + tid / kRowThreads;
  const int64_t c = (int64_t)(t % a.tiles_x) * kTileW + 4 * (tid % kRowThreads);
  const int64_t p = r * a.cols + c;    // first of this thread's 4 pixels
  // (columns are a multiple of 4: a thread's 4 pixels are all inside or all outside)
  const bool inside = r < a.rows && c < a.cols;
  float p0[4], g0[4], r0[4], nm[4];
  const bool any = inside;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    p0[k] = 0.0f;
    g0[k] = 1.0f;
    nm[k] = 1.0f;
    if (inside) {
      if (DT == SEP_DTYPE_U16_JF) {
        p0[k] = __ldg(a.ped + p + k);
        g0[k] = __ldg(a.gain + p + k);
      }
      if (NORM) nm[k] = __ldg(a.norm + p + k);
    }
    // level-0 reciprocal for the division below; 0 (= use the IEEE
    // division) outside the range where the correction step is exact
    const float ag = fabsf(g0[k]);
    r0[k] = ag >= 0x1p-100f && ag <= 0x1p100f ? __frcp_rn(g0[k]) : 0.0f;
  }
  const int f0 = blockIdx.y * a.frames_per_cta;
  const int nfr = min(f0 + a.frames_per_cta, a.n_frames) - f0;
  const unsigned slot0 = (unsigned)__cvta_generic_to_shared(&ring[0][tid * kVec]);
  // one commit group per frame (empty past the last frame or for idle threads)
  auto issue = [&](int j) {
    if (any && j < nfr) {
      const char* src = reinterpret_cast<const char*>(frame_ptr<DT>(a.frames, f0 + j, a.npix)) +
                        p * (DT == SEP_DTYPE_U16_JF ? 2 : 4);
      const unsigned dst = slot0 + (unsigned)((j % kRing) * kStageThreads * kVec);
      if (kVec == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
      else
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
#pragma unroll
  for (int j = 0; j < kRing; ++j) issue(j);
  for (int j = 0; j < nfr; j += 4) {
    const int nf = min(4, nfr - j);
    // groups 0 .. j + kRing - 1 issued: frames j .. j + 3 have landed
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kRing - 4) : "memory");
    uint32_t w[4][4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const unsigned char* sl = &ring[(j + h) % kRing][tid * kVec];
      if (DT == SEP_DTYPE_U16_JF) {
        const uint2 v = *reinterpret_cast<const uint2*>(sl);
        w[h][0] = v.x & 0xffffu; w[h][1] = v.x >> 16; w[h][2] = v.y & 0xffffu; w[h][3] = v.y >> 16;
      } else {
        const uint4 v = *reinterpret_cast<const uint4*>(sl);
        w[h][0] = v.x; w[h][1] = v.y; w[h][2] = v.z; w[h][3] = v.w;
      }
    }
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      if (h >= nf) continue;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (!inside) continue;
        float x;
        if (DT == SEP_DTYPE_U16_JF) {
          const uint32_t u = w[h][k], code = u >> 14;
          const float d0 = __fsub_rn((float)(u & 0x3FFFu), p0[k]);
          const float q0 = __fmul_rn(d0, r0[k]);
          const float aq = fabsf(q0);
          if (code == 0 && r0[k] != 0.0f && ((aq >= 0x1p-125f && aq <= 0x1p125f) || d0 == 0.0f)) {
            // RN((adc - ped) / gain) without a division: with r = RN(1/gain)
            // and q = RN(d r), the residual e = d - q gain is exact under a
            // fused multiply-add, and RN(q + e r) is the correctly rounded
            // quotient (Markstein's correction, IBM J. Res. Dev. 34(1), 1990);
            // the range tests keep gain, quotient and residual normal,
            // elsewhere the IEEE division runs
            x = __fmaf_rn(__fmaf_rn(-q0, g0[k], d0), r0[k], q0);
          } else {
            float ped = p0[k], gain = g0[k];
            if (code != 0) {   // gain levels 1 and 2
              const int64_t lvl = code == 1 ? 1 : 2;
              ped = __ldg(a.ped + lvl * a.npix + p + k);
              gain = __ldg(a.gain + lvl * a.npix + p + k);
            }
            x = __fdiv_rn(__fsub_rn((float)(u & 0x3FFFu), ped), gain);
          }
        } else {
          x = __uint_as_float(w[h][k]);
        }
        if (NORM) x = __fdiv_rn(x, nm[k]);
        tv[h][loc0 + k] = x;
      }
    }
    // the slots just read are refilled (this thread's own words, already in registers)
    issue(j + kRing);
    issue(j + kRing + 1);
    issue(j + kRing + 2);
    issue(j + kRing + 3);
    __syncthreads();
    scatter_tile<4>(a, ts, tv, eb, ne, (int64_t)(f0 + j), nf);
    __syncthreads();
  }
}

template <int DT, bool NORM>
cudaError_t launch_v(const StageArgs& a, dim3 grid, bool vec, cudaStream_t s) {
  if (vec) {
    constexpr size_t smem = ring_smem_bytes<DT>();
    if (smem > 48 * 1024) {
      // opt in once per device (the attribute only needs to be set before
      // the first launch; later calls find it set)
      static bool set[64] = {};
      int dev = 0;
      if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
      if (!set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_stage_ring<DT, NORM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        set[dev] = true;
      }
    }
    k_stage_ring<DT, NORM><<<grid, kStageThreads, smem, s>>>(a);
  } else {
    k_stage<DT, NORM, false><<<grid, kStageThreads, 0, s>>>(a);
  }
  return cudaGetLastError();
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
  if (dtype == SEP_DTYPE_U16_JF)
    return has_norm ? launch_v<SEP_DTYPE_U16_JF, true>(a, grid, vec && !a.fptr, s)
                    : launch_v<SEP_DTYPE_U16_JF, false>(a, grid, vec && !a.fptr, s);
  return has_norm ? launch_v<SEP_DTYPE_F32, true>(a, grid, vec && !a.fptr, s)
                  : launch_v<SEP_DTYPE_F32, false>(a, grid, vec && !a.fptr, s);
}

}  // namespace sep
