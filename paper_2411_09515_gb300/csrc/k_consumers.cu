// The two consumers of the separated background (Sections 3 and 4):
// sparsification (compact the kept pixels of each frame, ascending index)
// and peak picking (local maxima among kept pixels with enough kept
// neighbours), both driven by a per-frame kept-pixel bitmap (1 bit / pixel).
#include <cuda_runtime.h>
#include <stdint.h>

#include "sep_device.cuh"
#include "sep_internal.h"

namespace sep {
namespace {

// Exclusive scan of one int per thread over a block of NT threads.
template <int NT>
__device__ __forceinline__ int block_exclusive_scan(int x, int* total, int* sh) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) sh[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int v = lane < NW ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    if (lane < NW) sh[lane] = v;
  }
  __syncthreads();
  const int base = warp > 0 ? sh[warp - 1] : 0;
  *total = sh[NW - 1];
  __syncthreads();
  return base + inc - x;
}

__global__ void k_thresholds(const float* mean, const float* sigma, float k_pick, int64_t n, float* thr) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) thr[i] = __double2float_rd((double)mean[i] + (double)k_pick * (double)sigma[i]);
}

// One thread per pixel, one warp per bitmap word: every word is written.
template <int DT, bool NORM>
__global__ void k_mark(PixArgs p, int32_t nbins, const float* thr, uint32_t* bitmap, int64_t words) {
  const int64_t f = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool keep = false;
  if (i < p.npix) {
    int32_t b = __ldg(p.bop + i);
    if (b >= 0) {
      float v = pixel_value<DT, NORM>(frame_ptr<DT>(p.frames, f, p.npix), i, p.npix, p.ped, p.gain, p.norm);
      keep = v > __ldg(thr + f * nbins + b);
    }
  }
  uint32_t m = __ballot_sync(0xffffffffu, keep);
  if ((threadIdx.x & 31) == 0 && (i >> 5) < words) bitmap[f * words + (i >> 5)] = m;
}

constexpr int kCompactThreads = 1024;
constexpr int kWordsPerThread = 8;

// One CTA per frame: walk the bitmap in tiles, write kept pixels in order.
template <int DT, bool NORM>
__global__ void __launch_bounds__(kCompactThreads) k_compact(PixArgs p, const uint32_t* bitmap, int64_t words,
                                                             int32_t* idx, float* val, int64_t cap,
                                                             int32_t* n_kept, int32_t* status) {
  __shared__ int sh[kCompactThreads / 32];
  const int64_t f = blockIdx.x;
  const uint32_t* bm = bitmap + f * words;
  const void* frame = frame_ptr<DT>(p.frames, f, p.npix);
  int64_t total = 0;
  for (int64_t base = 0; base < words; base += (int64_t)kCompactThreads * kWordsPerThread) {
    const int64_t w0 = base + (int64_t)threadIdx.x * kWordsPerThread;
    uint32_t wv[kWordsPerThread];
    int cnt = 0;
    if (w0 + kWordsPerThread <= words) {
      const uint4* q = reinterpret_cast<const uint4*>(bm + w0);
      uint4 a = q[0], b = q[1];
      wv[0] = a.x; wv[1] = a.y; wv[2] = a.z; wv[3] = a.w;
      wv[4] = b.x; wv[5] = b.y; wv[6] = b.z; wv[7] = b.w;
    } else {
#pragma unroll
      for (int j = 0; j < kWordsPerThread; ++j) wv[j] = (w0 + j < words) ? bm[w0 + j] : 0u;
    }
#pragma unroll
    for (int j = 0; j < kWordsPerThread; ++j) cnt += __popc(wv[j]);
    int tile_total;
    int off = block_exclusive_scan<kCompactThreads>(cnt, &tile_total, sh);
    int64_t pos = total + off;
#pragma unroll
    for (int j = 0; j < kWordsPerThread; ++j) {
      uint32_t m = wv[j];
      while (m) {
        int bit = __ffs(m) - 1;
        m &= m - 1u;
        int64_t i = (w0 + j) * 32 + bit;
        if (pos < cap) {
          idx[f * cap + pos] = (int32_t)i;
          val[f * cap + pos] = pixel_value<DT, NORM>(frame, i, p.npix, p.ped, p.gain, p.norm);
        }
        ++pos;
      }
    }
    total += tile_total;
  }
  if (threadIdx.x == 0) {
    n_kept[f] = (int32_t)total;
    if (total > cap) atomicOr(status, SEP_DEV_CAPACITY);
  }
}

// Indices outside the detector are ignored (a caller's list is not trusted).
__global__ void k_scatter_list(const int32_t* idx, const int32_t* n_kept, int64_t kcap, int64_t npix,
                               uint32_t* bitmap, int64_t words) {
  const int64_t f = blockIdx.y;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t n = n_kept[f];
  if (n > kcap) n = kcap;
  if (k < n) {
    int32_t i = idx[f * kcap + k];
    if (i >= 0 && i < npix) atomicOr(bitmap + f * words + (i >> 5), 1u << (i & 31));
  }
}

constexpr int kPeakThreads = 256;

__device__ __forceinline__ bool is_kept(const uint32_t* bm, int64_t j) { return (bm[j >> 5] >> (j & 31)) & 1u; }

// One CTA per frame: each thread tests one kept pixel; peaks are written in
// ascending index order through a block scan per tile.
template <int DT, bool NORM>
__global__ void __launch_bounds__(kPeakThreads) k_peaks(PixArgs p, int32_t nbins, const float* mean,
                                                        const float* sigma, const uint32_t* bitmap, int64_t words,
                                                        const int32_t* idx, const int32_t* n_kept, int64_t kcap, int32_t patch,
                                                        int32_t min_count, sep_peak* peaks, int64_t pcap,
                                                        int32_t* n_peaks, int32_t* status) {
  __shared__ int sh[kPeakThreads / 32];
  const int64_t f = blockIdx.x;
  const uint32_t* bm = bitmap + f * words;
  const void* frame = frame_ptr<DT>(p.frames, f, p.npix);
  const float* mu = mean + f * nbins;
  const float* sd = sigma + f * nbins;
  int64_t n = n_kept[f];
  if (n > kcap) n = kcap;
  const int h = patch >> 1;
  int64_t total = 0;
  for (int64_t base = 0; base < n; base += kPeakThreads) {
    const int64_t k = base + threadIdx.x;
    int flag = 0;
    sep_peak rec;
    const int64_t i = k < n ? idx[f * kcap + k] : -1;
    if (i >= 0 && i < p.npix && __ldg(p.bop + i) >= 0) {
      const float vi = pixel_value<DT, NORM>(frame, i, p.npix, p.ped, p.gain, p.norm);
      const int r0 = (int)(i / p.cols), c0 = (int)(i - (int64_t)r0 * p.cols);
      const int rlo = max(r0 - h, 0), rhi = min(r0 + h, p.rows - 1);
      const int clo = max(c0 - h, 0), chi = min(c0 + h, p.cols - 1);
      int nk = 0;
      for (int r = rlo; r <= rhi; ++r)
        for (int c = clo; c <= chi; ++c) nk += is_kept(bm, (int64_t)r * p.cols + c);
      bool ok = nk >= min_count;
      // the maximum of the patch over valid pixels; ties go to the lowest index
      for (int r = rlo; ok && r <= rhi; ++r)
        for (int c = clo; ok && c <= chi; ++c) {
          const int64_t j = (int64_t)r * p.cols + c;
          if (j == i || __ldg(p.bop + j) < 0) continue;
          const float vj = pixel_value<DT, NORM>(frame, j, p.npix, p.ped, p.gain, p.norm);
          if (!(vi > vj || (vi == vj && i < j))) ok = false;
        }
      if (ok) {
        float I = 0.f, sy = 0.f, sx = 0.f, s2 = 0.f;
        for (int r = rlo; r <= rhi; ++r)
          for (int c = clo; c <= chi; ++c) {
            const int64_t j = (int64_t)r * p.cols + c;
            if (!is_kept(bm, j)) continue;
            const int32_t bj = __ldg(p.bop + j);
            const float vj = j == i ? vi : pixel_value<DT, NORM>(frame, j, p.npix, p.ped, p.gain, p.norm);
            const float w = vj - __ldg(mu + bj);
            const float s = __ldg(sd + bj);
            I += w;
            sy += w * ((float)r + 0.5f);
            sx += w * ((float)c + 0.5f);
            s2 += s * s;
          }
        rec.idx = (int32_t)i;
        rec.I = I;
        rec.y = sy / I;
        rec.x = sx / I;
        rec.sigma = sqrtf(s2);
        rec.npix = nk;
        flag = 1;
      }
    }
    int tile_total;
    int off = block_exclusive_scan<kPeakThreads>(flag, &tile_total, sh);
    if (flag && total + off < pcap) peaks[f * pcap + total + off] = rec;
    total += tile_total;
  }
  if (threadIdx.x == 0) {
    n_peaks[f] = (int32_t)total;
    if (total > pcap) atomicOr(status, SEP_DEV_CAPACITY);
  }
}

}  // namespace

cudaError_t launch_thresholds(const float* mean, const float* sigma, float k_pick, int64_t n, float* thr,
                              cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_thresholds<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(mean, sigma, k_pick, n, thr);
  return cudaGetLastError();
}

cudaError_t launch_mark(const PixArgs& p, int32_t n_frames, int32_t nbins, const float* thr, uint32_t* bitmap,
                        int64_t words, cudaStream_t s) {
  if (n_frames <= 0) return cudaSuccess;
  dim3 grid((unsigned)((words * 32 + 255) / 256), (unsigned)n_frames);
  const bool nrm = p.norm != nullptr;
  if (p.dtype == SEP_DTYPE_U16_JF) {
    if (nrm) k_mark<SEP_DTYPE_U16_JF, true><<<grid, 256, 0, s>>>(p, nbins, thr, bitmap, words);
    else k_mark<SEP_DTYPE_U16_JF, false><<<grid, 256, 0, s>>>(p, nbins, thr, bitmap, words);
  } else {
    if (nrm) k_mark<SEP_DTYPE_F32, true><<<grid, 256, 0, s>>>(p, nbins, thr, bitmap, words);
    else k_mark<SEP_DTYPE_F32, false><<<grid, 256, 0, s>>>(p, nbins, thr, bitmap, words);
  }
  return cudaGetLastError();
}

cudaError_t launch_compact(const PixArgs& p, int32_t n_frames, const uint32_t* bitmap, int64_t words, int32_t* idx,
                           float* val, int64_t cap, int32_t* n_kept, int32_t* status, cudaStream_t s) {
  if (n_frames <= 0) return cudaSuccess;
  const bool nrm = p.norm != nullptr;
  if (p.dtype == SEP_DTYPE_U16_JF) {
    if (nrm) k_compact<SEP_DTYPE_U16_JF, true><<<n_frames, kCompactThreads, 0, s>>>(p, bitmap, words, idx, val, cap, n_kept, status);
    else k_compact<SEP_DTYPE_U16_JF, false><<<n_frames, kCompactThreads, 0, s>>>(p, bitmap, words, idx, val, cap, n_kept, status);
  } else {
    if (nrm) k_compact<SEP_DTYPE_F32, true><<<n_frames, kCompactThreads, 0, s>>>(p, bitmap, words, idx, val, cap, n_kept, status);
    else k_compact<SEP_DTYPE_F32, false><<<n_frames, kCompactThreads, 0, s>>>(p, bitmap, words, idx, val, cap, n_kept, status);
  }
  return cudaGetLastError();
}

cudaError_t launch_scatter_list(int32_t n_frames, const int32_t* idx, const int32_t* n_kept, int64_t kcap,
                                int64_t npix, uint32_t* bitmap, int64_t words, cudaStream_t s) {
  if (n_frames <= 0 || kcap <= 0) return cudaSuccess;
  dim3 grid((unsigned)((kcap + 255) / 256), (unsigned)n_frames);
  k_scatter_list<<<grid, 256, 0, s>>>(idx, n_kept, kcap, npix, bitmap, words);
  return cudaGetLastError();
}

cudaError_t launch_peaks(const PixArgs& p, int32_t n_frames, int32_t nbins, const float* mean, const float* sigma,
                         const uint32_t* bitmap, int64_t words, const int32_t* idx,
                         const int32_t* n_kept, int64_t kcap, int32_t patch, int32_t min_count, sep_peak* peaks,
                         int64_t pcap, int32_t* n_peaks, int32_t* status, cudaStream_t s) {
  if (n_frames <= 0) return cudaSuccess;
  const bool nrm = p.norm != nullptr;
#define SEP_PEAK_ARGS p, nbins, mean, sigma, bitmap, words, idx, n_kept, kcap, patch, min_count, peaks, pcap, n_peaks, status
  if (p.dtype == SEP_DTYPE_U16_JF) {
    if (nrm) k_peaks<SEP_DTYPE_U16_JF, true><<<n_frames, kPeakThreads, 0, s>>>(SEP_PEAK_ARGS);
    else k_peaks<SEP_DTYPE_U16_JF, false><<<n_frames, kPeakThreads, 0, s>>>(SEP_PEAK_ARGS);
  } else {
    if (nrm) k_peaks<SEP_DTYPE_F32, true><<<n_frames, kPeakThreads, 0, s>>>(SEP_PEAK_ARGS);
    else k_peaks<SEP_DTYPE_F32, false><<<n_frames, kPeakThreads, 0, s>>>(SEP_PEAK_ARGS);
  }
#undef SEP_PEAK_ARGS
  return cudaGetLastError();
}

}  // namespace sep
