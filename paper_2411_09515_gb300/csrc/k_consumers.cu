// The two consumers of the separated background (Sections 3 and 4):
// sparsification (compact the kept pixels of each frame, ascending index)
// and peak picking (local maxima among kept pixels with enough kept
// neighbours), both driven by a per-frame kept-pixel bitmap (1 bit / pixel).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "sep_device.cuh"
#include "sep_internal.h"

namespace sep {
namespace {

// Value of pixel i of launch frame f: the staged copy when the call staged
// the batch, else recomputed from the frame (the same IEEE sequence).
template <int DT, bool NORM>
__device__ __forceinline__ float value_of(const PixArgs& p, const void* frame, int64_t f, int64_t i) {
  if (p.stage) return __ldg(p.stage + f * p.npos + __ldg(p.pos_of + i));
  return pixel_value<DT, NORM>(frame, i, p.npix, p.ped, p.gain, p.norm);
}

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

// Staged values back to image order; pixels without a position get NaN.
__global__ void k_unstage(const float* stage, int64_t stride, const int32_t* pos_of, int64_t npix, float* out) {
  const int64_t f = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npix) return;
  const int32_t q = __ldg(pos_of + i);
  out[f * npix + i] = q >= 0 ? __ldg(stage + f * stride + q) : __int_as_float(0x7fc00000);
}

constexpr int kCompactThreads = 1024;
constexpr int kWordsPerThread = 8;
constexpr int64_t kTileWords = (int64_t)kCompactThreads * kWordsPerThread;   // bitmap words per CTA
constexpr int kEmitList = 8192;   // kept pixels a CTA lists in shared memory at once

// Phase 1 of the ordered compaction: kept pixels per tile of the bitmap.
__global__ void __launch_bounds__(256) k_count_bits(const uint32_t* bitmap, int64_t words, int32_t* tile_cnt,
                                                    int32_t n_tiles) {
  const int64_t f = blockIdx.y;
  const int64_t w0 = (int64_t)blockIdx.x * kTileWords;
  const uint32_t* bm = bitmap + f * words;
  int cnt = 0;
  for (int64_t w = w0 + 4 * (int64_t)threadIdx.x; w < w0 + kTileWords && w < words; w += 4 * 256) {
    // words is a multiple of 8, so a 4-word vector never runs past the frame
    const uint4 q = *reinterpret_cast<const uint4*>(bm + w);
    cnt += __popc(q.x) + __popc(q.y) + __popc(q.z) + __popc(q.w);
  }
  __shared__ int sh[8];
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int i = 0; i < 8; ++i) t += sh[i];
    tile_cnt[f * n_tiles + blockIdx.x] = t;
  }
}

// Phase 2: each CTA writes its tile's kept pixels (ascending) after the
// pixels of all earlier tiles of the frame; values are recomputed from the
// frame exactly as the clip kernel computed them.
template <int DT, bool NORM>
__global__ void __launch_bounds__(kCompactThreads) k_emit_kept(PixArgs p, const uint32_t* bitmap, int64_t words,
                                                               const int32_t* tile_cnt, int32_t n_tiles, int32_t* idx,
                                                               float* val, int64_t cap, int32_t* n_kept,
                                                               int32_t* status) {
  __shared__ int sh[kCompactThreads / 32];
  __shared__ int64_t base_s;
  const int64_t f = blockIdx.y;
  const int tile = blockIdx.x;
  if (threadIdx.x < 32) {
    int64_t before = 0, all = 0;
    for (int t = threadIdx.x; t < n_tiles; t += 32) {
      const int c = tile_cnt[f * n_tiles + t];
      all += c;
      if (t < tile) before += c;
    }
    for (int o = 16; o > 0; o >>= 1) {
      before += __shfl_xor_sync(0xffffffffu, before, o);
      all += __shfl_xor_sync(0xffffffffu, all, o);
    }
    if (threadIdx.x == 0) {
      base_s = before;
      if (tile == 0) {
        n_kept[p.fidx ? p.fidx[f] : f] = (int32_t)all;
        if (all > cap) atomicOr(status, SEP_DEV_CAPACITY);
      }
    }
  }
  __syncthreads();
  const int64_t base = base_s;
  if (base >= cap) return;
  const uint32_t* bm = bitmap + f * words;
  const void* frame = p.fptr ? (const void*)p.fptr[f] : frame_ptr<DT>(p.frames, f, p.npix);
  const int64_t g = p.fidx ? p.fidx[f] : f;   // output row of this frame
  const int64_t w0 = (int64_t)tile * kTileWords + (int64_t)threadIdx.x * kWordsPerThread;
  uint32_t wv[kWordsPerThread];
  if (w0 + kWordsPerThread <= words) {
    const uint4* q = reinterpret_cast<const uint4*>(bm + w0);
    const uint4 a = q[0], b = q[1];
    wv[0] = a.x; wv[1] = a.y; wv[2] = a.z; wv[3] = a.w;
    wv[4] = b.x; wv[5] = b.y; wv[6] = b.z; wv[7] = b.w;
  } else {
#pragma unroll
    for (int j = 0; j < kWordsPerThread; ++j) wv[j] = (w0 + j < words) ? bm[w0 + j] : 0u;
  }
  int cnt = 0;
#pragma unroll
  for (int j = 0; j < kWordsPerThread; ++j) cnt += __popc(wv[j]);
  int tile_total;
  const int first = block_exclusive_scan<kCompactThreads>(cnt, &tile_total, sh);   // this thread's first, in the tile
  // The tile's kept pixels go through a shared list, kEmitList at a time:
  // each thread lists its own pixels at their ranks, then consecutive
  // threads take consecutive entries, so the value loads of the whole list
  // are in flight together and the stores are coalesced.
  __shared__ int32_t lst[kEmitList];
  const int64_t n_tile = (int64_t)tile_total < cap - base ? (int64_t)tile_total : cap - base;
  for (int r0 = 0; r0 < n_tile; r0 += kEmitList) {
    if (first < r0 + kEmitList && first + cnt > r0) {
      int rank = first;
#pragma unroll
      for (int j = 0; j < kWordsPerThread; ++j) {
        uint32_t m = wv[j];
        while (m) {
          const int bit = __ffs(m) - 1;
          m &= m - 1u;
          if (rank >= r0 && rank < r0 + kEmitList) lst[rank - r0] = (int32_t)((w0 + j) * 32 + bit);
          ++rank;
        }
      }
    }
    __syncthreads();
    const int nr = (int)(n_tile - r0 < kEmitList ? n_tile - r0 : kEmitList);
    for (int k = threadIdx.x; k < nr; k += kCompactThreads) {
      const int64_t pos = base + r0 + k;
      const int32_t i = lst[k];
      idx[g * cap + pos] = i;
      val[g * cap + pos] = value_of<DT, NORM>(p, frame, f, i);
    }
    __syncthreads();
  }
}

// Densification (Section 3): the background level of every binned pixel
// (its bin's mean, or RN(mean + RN(sigma z)) with the caller's deviates z),
// fill where a pixel has no bin; one thread per pixel.
// Level of pixel i in a per-bin profile p (bin level, or the radial
// interpolation between the bins a and a + 1 with weight t on the upper).
__device__ __forceinline__ float profile_at(const float* p, int32_t b, const int32_t* ia, const float* it, int64_t i,
                                            int32_t nbins) {
  if (!ia) return __ldg(p + b);
  const int32_t a = __ldg(ia + i);
  const float t = __ldg(it + i);
  const float hi = a + 1 < nbins ? __ldg(p + a + 1) : 0.0f;
  return __fadd_rn(__fmul_rn(__fsub_rn(1.0f, t), __ldg(p + a)), __fmul_rn(t, hi));
}

__global__ void __launch_bounds__(256) k_dense_background(const int32_t* bop, int64_t npix, int32_t nbins,
                                                          const float* mean, const float* sigma,
                                                          const float* noise, float fill, const int32_t* ia,
                                                          const float* it, float* out) {
  const int64_t f = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npix) return;
  const int32_t b = __ldg(bop + i);
  float x = fill;
  if (b >= 0) {
    x = profile_at(mean + f * nbins, b, ia, it, i, nbins);
    if (noise)
      x = __fadd_rn(x, __fmul_rn(profile_at(sigma + f * nbins, b, ia, it, i, nbins), __ldg(noise + f * npix + i)));
  }
  out[f * npix + i] = x;
}

// The same, four consecutive pixels a thread (vector loads and stores; the
// pixel count is a multiple of 4 and the rows are 16-byte aligned).
__global__ void __launch_bounds__(256) k_dense_background4(const int32_t* bop, int64_t npix, int32_t nbins,
                                                           const float* mean, const float* sigma,
                                                           const float* noise, float fill, const int32_t* ia,
                                                           const float* it, float* out) {
  const int64_t f = blockIdx.y;
  const int64_t i = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= npix) return;
  const int4 b = __ldg(reinterpret_cast<const int4*>(bop + i));
  const int bb[4] = {b.x, b.y, b.z, b.w};
  const float* mu = mean + f * nbins;
  float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  if (noise) {
    const float4 zz = __ldg(reinterpret_cast<const float4*>(noise + f * npix + i));
    z[0] = zz.x; z[1] = zz.y; z[2] = zz.z; z[3] = zz.w;
  }
  float x[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    x[k] = fill;
    if (bb[k] >= 0) {
      x[k] = profile_at(mu, bb[k], ia, it, i + k, nbins);
      if (noise) x[k] = __fadd_rn(x[k], __fmul_rn(profile_at(sigma + f * nbins, bb[k], ia, it, i + k, nbins), z[k]));
    }
  }
  *reinterpret_cast<float4*>(out + f * npix + i) = make_float4(x[0], x[1], x[2], x[3]);
}

// Kept pixels against the smooth background (Section 3): the threshold of
// pixel i is RD(mu(x_i) + k_pick sigma(x_i)) with the frame's profile
// interpolated at the pixel centre. One thread per pixel, one warp per
// bitmap word: every word is written.
template <int DT, bool NORM>
__global__ void __launch_bounds__(256) k_mark_interp(PixArgs p, int32_t nbins, const float* mean, const float* sigma,
                                                     float k_pick, uint32_t* bitmap, int64_t words) {
  const int64_t f = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool keep = false;
  if (i < p.npix) {
    const int32_t b = __ldg(p.bop + i);
    if (b >= 0) {
      const int64_t row = p.orow ? p.orow[f] : f * (int64_t)nbins;
      const float m = profile_at(mean + row, b, p.ia, p.it, i, nbins);
      const float sd = profile_at(sigma + row, b, p.ia, p.it, i, nbins);
      const void* frame = p.fptr ? (const void*)p.fptr[f] : frame_ptr<DT>(p.frames, f, p.npix);
      const float v = value_of<DT, NORM>(p, frame, f, i);
      keep = v > __double2float_rd((double)m + (double)k_pick * (double)sd);
    }
  }
  const uint32_t mk = __ballot_sync(0xffffffffu, keep);
  if ((threadIdx.x & 31) == 0 && (i >> 5) < words) bitmap[f * words + (i >> 5)] = mk;
}

// ... then the recorded values of the kept pixels.
__global__ void __launch_bounds__(256) k_dense_scatter(const int32_t* idx, const float* val, int64_t cap,
                                                       const int32_t* n_kept, int64_t npix, float* out) {
  const int64_t f = blockIdx.y;
  int64_t n = n_kept[f];
  n = n < 0 ? 0 : (n > cap ? cap : n);
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = idx[f * cap + k];
    if (i >= 0 && i < npix) out[f * npix + i] = val[f * cap + k];
  }
}

// Veto (Section 4): the frames with at least min_peaks peaks, ascending, by
// one CTA scanning the counts in tiles of its size.
__global__ void __launch_bounds__(1024) k_veto(int32_t n_frames, const int32_t* n_peaks, int32_t min_peaks,
                                               int32_t* list, int32_t* n_pass) {
  __shared__ int sh[32];
  int base = 0;
  for (int f0 = 0; f0 < n_frames; f0 += 1024) {
    const int f = f0 + threadIdx.x;
    const int pass = f < n_frames && n_peaks[f] >= min_peaks;
    int total;
    const int pos = base + block_exclusive_scan<1024>(pass, &total, sh);
    if (pass) list[pos] = f;
    base += total;
  }
  if (threadIdx.x == 0) *n_pass = base;
}

// Row j of dst = row list[j] of src for j < *n_pass (32-bit words; 16-byte
// vectors when rows and bases allow).
template <bool VEC>
__global__ void __launch_bounds__(256) k_compact_rows(const int32_t* list, const int32_t* n_pass, int64_t row_words,
                                                      const uint32_t* src, uint32_t* dst) {
  const int64_t j = blockIdx.y;
  if (j >= *n_pass) return;
  const int64_t r = list[j];
  if (r < 0 || r >= gridDim.y) return;   // (a caller's list is not trusted)
  const uint32_t* s = src + r * row_words;
  uint32_t* d = dst + j * row_words;
  if (VEC) {
    const int64_t n4 = row_words >> 2;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += (int64_t)gridDim.x * blockDim.x)
      reinterpret_cast<uint4*>(d)[q] = __ldg(reinterpret_cast<const uint4*>(s) + q);
  } else {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < row_words;
         q += (int64_t)gridDim.x * blockDim.x)
      d[q] = __ldg(s + q);
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
constexpr int kPeakChunk = 256;          // kept entries per flag chunk (8 flag words)
constexpr int kPeakCtasPerFrame = 64;
constexpr int kPeakList = 4096;         // peaks a record CTA lists in shared memory at once

__device__ __forceinline__ bool is_kept(const uint32_t* bm, int64_t j) { return (bm[j >> 5] >> (j & 31)) & 1u; }

// Is kept pixel i a peak (Section 4)? At least min_count kept pixels in the
// patch, and i the maximum of the patch's valid pixels (ties: lowest index).
// (the pixel's own value is loaded only once the bitmap has shown enough
// kept pixels: most kept pixels are isolated and fail on the count alone)
template <int DT, bool NORM>
__device__ __forceinline__ bool peak_test(const PixArgs& p, const void* frame, int64_t f, const uint32_t* bm, int64_t i,
                                          int h, int32_t min_count) {
  const int r0 = (int)(i / p.cols), c0 = (int)(i - (int64_t)r0 * p.cols);
  const int rlo = max(r0 - h, 0), rhi = min(r0 + h, p.rows - 1);
  const int clo = max(c0 - h, 0), chi = min(c0 + h, p.cols - 1);
  int nk = 0;
  for (int r = rlo; r <= rhi; ++r)
    for (int c = clo; c <= chi; ++c) nk += is_kept(bm, (int64_t)r * p.cols + c);
  if (nk < min_count) return false;
  const float vi = value_of<DT, NORM>(p, frame, f, i);
  for (int r = rlo; r <= rhi; ++r)
    for (int c = clo; c <= chi; ++c) {
      const int64_t j = (int64_t)r * p.cols + c;
      if (j == i || __ldg(p.bop + j) < 0) continue;
      const float vj = value_of<DT, NORM>(p, frame, f, j);
      if (!(vi > vj || (vi == vj && i < j))) return false;
    }
  return true;
}

// Phase 1: one flag bit per kept-list entry, and peaks per chunk of 256.
template <int DT, bool NORM>
__global__ void __launch_bounds__(kPeakThreads) k_peak_flags(PixArgs p, const uint32_t* bitmap, int64_t words,
                                                             const int32_t* idx, const int32_t* n_kept, int64_t kcap,
                                                             int32_t patch, int32_t min_count, uint32_t* flags,
                                                             int32_t* chunk_cnt, int32_t n_chunks) {
  const int64_t f = blockIdx.y;
  const uint32_t* bm = bitmap + f * words;
  const void* frame = p.fptr ? (const void*)p.fptr[f] : frame_ptr<DT>(p.frames, f, p.npix);
  const int64_t g = p.fidx ? p.fidx[f] : f;
  int64_t n = n_kept[g];
  if (n > kcap) n = kcap;
  const int h = patch >> 1;
  for (int64_t ch = blockIdx.x; ch * kPeakChunk < n; ch += gridDim.x) {
    const int64_t k = ch * kPeakChunk + threadIdx.x;
    bool peak = false;
    const int64_t i = k < n ? idx[g * kcap + k] : -1;
    if (i >= 0 && i < p.npix && __ldg(p.bop + i) >= 0) peak = peak_test<DT, NORM>(p, frame, f, bm, i, h, min_count);
    const uint32_t m = __ballot_sync(0xffffffffu, peak);
    if ((threadIdx.x & 31) == 0) flags[f * ((int64_t)n_chunks * 8) + ch * 8 + (threadIdx.x >> 5)] = m;
    const int c = __syncthreads_count(peak);
    if (threadIdx.x == 0) chunk_cnt[f * n_chunks + ch] = c;
  }
}

// Phase 2 (one CTA per frame): prefix over chunk counts, then every flagged
// entry writes its record at its rank: ascending pixel order, since the
// kept list ascends.
template <int DT, bool NORM, bool INTERP>
__global__ void __launch_bounds__(1024) k_peak_emit(PixArgs p, int32_t nbins, const float* mean, const float* sigma,
                                                    const uint32_t* bitmap, int64_t words, const int32_t* idx,
                                                    const int32_t* n_kept, int64_t kcap, int32_t patch,
                                                    const uint32_t* flags, int32_t* chunk_cnt, int32_t n_chunks,
                                                    sep_peak* peaks, int64_t pcap, int32_t* n_peaks,
                                                    int32_t* status) {
  __shared__ int sh[32];
  const int64_t f = blockIdx.x;
  const int64_t g = p.fidx ? p.fidx[f] : f;
  int64_t n = n_kept[g];
  if (n > kcap) n = kcap;
  const int nch = (int)((n + kPeakChunk - 1) / kPeakChunk);
  // chunk counts become chunk offsets, in place (a count <= kcap < 2^31)
  int32_t* chunk_base = chunk_cnt + f * n_chunks;
  int64_t total = 0;
  for (int c0 = 0; c0 < nch; c0 += 1024) {
    const int c = c0 + threadIdx.x;
    const int x = c < nch ? chunk_base[c] : 0;
    int tt;
    const int off = block_exclusive_scan<1024>(x, &tt, sh);
    if (c < nch) chunk_base[c] = (int32_t)(total + off);
    total += tt;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    n_peaks[g] = (int32_t)total;
    if (total > pcap) atomicOr(status, SEP_DEV_CAPACITY);
  }
  const uint32_t* bm = bitmap + f * words;
  const void* frame = p.fptr ? (const void*)p.fptr[f] : frame_ptr<DT>(p.frames, f, p.npix);
  const int64_t row = p.orow ? p.orow[f] : f * (int64_t)nbins;
  const float* mu = mean + row;
  const float* sd = sigma + row;
  const int h = patch >> 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t* fl = flags + f * ((int64_t)n_chunks * 8);
  // the flagged entries go through a shared list, kPeakList at a time: a
  // warp per chunk and a lane per flag bit list them at their ranks, then a
  // thread per listed peak writes its record (all patches in flight together)
  __shared__ int32_t plist[kPeakList];
  const int64_t n_out = total < pcap ? total : pcap;
  for (int64_t r0 = 0; r0 < n_out; r0 += kPeakList) {
    for (int c = warp; c < nch; c += 32) {
      int64_t rank = chunk_base[c];
      if (rank >= r0 + kPeakList) continue;
      for (int wd = 0; wd < 8; ++wd) {
        const uint32_t m = fl[c * 8 + wd];
        if (m == 0) continue;
        if ((m >> lane) & 1u) {
          const int64_t pos = rank + __popc(m & ((1u << lane) - 1u));
          if (pos >= r0 && pos < r0 + kPeakList) plist[pos - r0] = c * kPeakChunk + wd * 32 + lane;
        }
        rank += __popc(m);
      }
    }
    __syncthreads();
    const int nr = (int)(n_out - r0 < kPeakList ? n_out - r0 : kPeakList);
    for (int t = threadIdx.x; t < nr; t += 1024) {
      const int64_t pos = r0 + t;
      const int64_t i = idx[g * kcap + plist[t]];
      const int rr0 = (int)(i / p.cols), cc0 = (int)(i - (int64_t)rr0 * p.cols);
      const int rlo = max(rr0 - h, 0), rhi = min(rr0 + h, p.rows - 1);
      const int clo = max(cc0 - h, 0), chi = min(cc0 + h, p.cols - 1);
      float I = 0.f, sy = 0.f, sx = 0.f, s2 = 0.f;
      int nk = 0;
      for (int r = rlo; r <= rhi; ++r)
        for (int cc = clo; cc <= chi; ++cc) {
          const int64_t j = (int64_t)r * p.cols + cc;
          if (!is_kept(bm, j)) continue;
          const int32_t bj = __ldg(p.bop + j);
          const float vj = value_of<DT, NORM>(p, frame, f, j);
          // background of the pixel's bin, or the profile at its centre
          const float w = vj - (INTERP ? profile_at(mu, bj, p.ia, p.it, j, nbins) : __ldg(mu + bj));
          const float sdv = INTERP ? profile_at(sd, bj, p.ia, p.it, j, nbins) : __ldg(sd + bj);
          ++nk;
          I += w;
          sy += w * ((float)r + 0.5f);
          sx += w * ((float)cc + 0.5f);
          s2 += sdv * sdv;
        }
      sep_peak rec;
      rec.idx = (int32_t)i;
      rec.I = I;
      rec.y = sy / I;
      rec.x = sx / I;
      rec.sigma = sqrtf(s2);
      rec.npix = nk;
      peaks[g * pcap + pos] = rec;
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_thresholds(const float* mean, const float* sigma, float k_pick, int64_t n, float* thr,
                              cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_thresholds<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(mean, sigma, k_pick, n, thr);
  return cudaGetLastError();
}

cudaError_t launch_unstage(const float* stage, int64_t stride, const int32_t* pos_of, int64_t npix, int32_t n_frames,
                           float* out, cudaStream_t s) {
  if (n_frames <= 0 || npix <= 0) return cudaSuccess;
  dim3 grid((unsigned)((npix + 255) / 256), (unsigned)n_frames);
  k_unstage<<<grid, 256, 0, s>>>(stage, stride, pos_of, npix, out);
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

cudaError_t launch_mark_interp(const PixArgs& p, int32_t n_frames, int32_t nbins, const float* mean,
                               const float* sigma, float k_pick, uint32_t* bitmap, int64_t words, cudaStream_t s) {
  if (n_frames <= 0) return cudaSuccess;
  dim3 grid((unsigned)((words * 32 + 255) / 256), (unsigned)n_frames);
  const bool nrm = p.norm != nullptr;
#define SEP_MARK_ARGS p, nbins, mean, sigma, k_pick, bitmap, words
  if (p.dtype == SEP_DTYPE_U16_JF) {
    if (nrm) k_mark_interp<SEP_DTYPE_U16_JF, true><<<grid, 256, 0, s>>>(SEP_MARK_ARGS);
    else k_mark_interp<SEP_DTYPE_U16_JF, false><<<grid, 256, 0, s>>>(SEP_MARK_ARGS);
  } else {
    if (nrm) k_mark_interp<SEP_DTYPE_F32, true><<<grid, 256, 0, s>>>(SEP_MARK_ARGS);
    else k_mark_interp<SEP_DTYPE_F32, false><<<grid, 256, 0, s>>>(SEP_MARK_ARGS);
  }
#undef SEP_MARK_ARGS
  return cudaGetLastError();
}

int32_t compact_tiles(int64_t words) { return (int32_t)((words + kTileWords - 1) / kTileWords); }
int32_t peak_chunks(int64_t kcap) { return (int32_t)((kcap + kPeakChunk - 1) / kPeakChunk); }

cudaError_t launch_compact(const PixArgs& p, int32_t n_frames, const uint32_t* bitmap, int64_t words, int32_t* idx,
                           float* val, int64_t cap, int32_t* n_kept, int32_t* scratch, int32_t* status,
                           cudaStream_t s) {
  if (n_frames <= 0) return cudaSuccess;
  const int32_t nt = compact_tiles(words);
  dim3 grid((unsigned)nt, (unsigned)n_frames);
  k_count_bits<<<grid, 256, 0, s>>>(bitmap, words, scratch, nt);
  const bool nrm = p.norm != nullptr;
#define SEP_EMIT_ARGS p, bitmap, words, scratch, nt, idx, val, cap, n_kept, status
  if (p.dtype == SEP_DTYPE_U16_JF) {
    if (nrm) k_emit_kept<SEP_DTYPE_U16_JF, true><<<grid, kCompactThreads, 0, s>>>(SEP_EMIT_ARGS);
    else k_emit_kept<SEP_DTYPE_U16_JF, false><<<grid, kCompactThreads, 0, s>>>(SEP_EMIT_ARGS);
  } else {
    if (nrm) k_emit_kept<SEP_DTYPE_F32, true><<<grid, kCompactThreads, 0, s>>>(SEP_EMIT_ARGS);
    else k_emit_kept<SEP_DTYPE_F32, false><<<grid, kCompactThreads, 0, s>>>(SEP_EMIT_ARGS);
  }
#undef SEP_EMIT_ARGS
  return cudaGetLastError();
}

cudaError_t launch_densify(const int32_t* bop, int64_t npix, int32_t nbins, int32_t n_frames, const float* mean,
                           const float* sigma, const int32_t* idx, const float* val, int64_t cap,
                           const int32_t* n_kept, const float* noise, float fill, const int32_t* interp_a,
                           const float* interp_t, float* out, cudaStream_t s) {
  if (n_frames <= 0 || npix <= 0) return cudaSuccess;
  const bool vec = npix % 4 == 0 && (uintptr_t)out % 16 == 0 && (!noise || (uintptr_t)noise % 16 == 0) &&
                   (uintptr_t)bop % 16 == 0;
  if (vec) {
    dim3 g1((unsigned)((npix / 4 + 255) / 256), (unsigned)n_frames);
    k_dense_background4<<<g1, 256, 0, s>>>(bop, npix, nbins, mean, sigma, noise, fill, interp_a, interp_t, out);
  } else {
    dim3 g1((unsigned)((npix + 255) / 256), (unsigned)n_frames);
    k_dense_background<<<g1, 256, 0, s>>>(bop, npix, nbins, mean, sigma, noise, fill, interp_a, interp_t, out);
  }
  if (cap > 0) {
    dim3 g2((unsigned)std::min<int64_t>((cap + 255) / 256, 64), (unsigned)n_frames);
    k_dense_scatter<<<g2, 256, 0, s>>>(idx, val, cap, n_kept, npix, out);
  }
  return cudaGetLastError();
}

cudaError_t launch_veto(int32_t n_frames, const int32_t* n_peaks, int32_t min_peaks, int32_t* list, int32_t* n_pass,
                        cudaStream_t s) {
  k_veto<<<1, 1024, 0, s>>>(n_frames, n_peaks, min_peaks, list, n_pass);
  return cudaGetLastError();
}

cudaError_t launch_compact_rows(int32_t n_frames, const int32_t* list, const int32_t* n_pass, int64_t row_bytes,
                                const void* src, void* dst, cudaStream_t s) {
  if (n_frames <= 0 || row_bytes <= 0) return cudaSuccess;
  const int64_t words = row_bytes / 4;
  const bool vec = words % 4 == 0 && (uintptr_t)src % 16 == 0 && (uintptr_t)dst % 16 == 0;
  const int64_t per = vec ? words / 4 : words;
  dim3 grid((unsigned)std::min<int64_t>(std::max<int64_t>((per + 255) / 256, 1), 64), (unsigned)n_frames);
  if (vec)
    k_compact_rows<true><<<grid, 256, 0, s>>>(list, n_pass, words, static_cast<const uint32_t*>(src),
                                               static_cast<uint32_t*>(dst));
  else
    k_compact_rows<false><<<grid, 256, 0, s>>>(list, n_pass, words, static_cast<const uint32_t*>(src),
                                                static_cast<uint32_t*>(dst));
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
                         const uint32_t* bitmap, int64_t words, const int32_t* idx, const int32_t* n_kept, int64_t kcap,
                         int32_t patch, int32_t min_count, sep_peak* peaks, int64_t pcap, int32_t* n_peaks,
                         int32_t* scratch, int32_t* status, cudaStream_t s) {
  if (n_frames <= 0) return cudaSuccess;
  const int32_t nch = peak_chunks(kcap);
  uint32_t* flags = reinterpret_cast<uint32_t*>(scratch);
  int32_t* cnt = scratch + (int64_t)n_frames * nch * 8;
  dim3 g1((unsigned)std::min<int32_t>(std::max<int32_t>(nch, 1), kPeakCtasPerFrame), (unsigned)n_frames);
  const bool nrm = p.norm != nullptr;
  const bool itp = p.ia != nullptr && p.it != nullptr;
#define SEP_FLAG_ARGS p, bitmap, words, idx, n_kept, kcap, patch, min_count, flags, cnt, nch
#define SEP_PEMIT_ARGS p, nbins, mean, sigma, bitmap, words, idx, n_kept, kcap, patch, flags, cnt, nch, peaks, pcap, n_peaks, status
#define SEP_PEMIT(DT, NR)                                                              \
  if (itp) k_peak_emit<DT, NR, true><<<n_frames, 1024, 0, s>>>(SEP_PEMIT_ARGS);      \
  else k_peak_emit<DT, NR, false><<<n_frames, 1024, 0, s>>>(SEP_PEMIT_ARGS)
  if (p.dtype == SEP_DTYPE_U16_JF) {
    if (nrm) {
      k_peak_flags<SEP_DTYPE_U16_JF, true><<<g1, kPeakThreads, 0, s>>>(SEP_FLAG_ARGS);
      SEP_PEMIT(SEP_DTYPE_U16_JF, true);
    } else {
      k_peak_flags<SEP_DTYPE_U16_JF, false><<<g1, kPeakThreads, 0, s>>>(SEP_FLAG_ARGS);
      SEP_PEMIT(SEP_DTYPE_U16_JF, false);
    }
  } else {
    if (nrm) {
      k_peak_flags<SEP_DTYPE_F32, true><<<g1, kPeakThreads, 0, s>>>(SEP_FLAG_ARGS);
      SEP_PEMIT(SEP_DTYPE_F32, true);
    } else {
      k_peak_flags<SEP_DTYPE_F32, false><<<g1, kPeakThreads, 0, s>>>(SEP_FLAG_ARGS);
      SEP_PEMIT(SEP_DTYPE_F32, false);
    }
  }
#undef SEP_PEMIT
#undef SEP_FLAG_ARGS
#undef SEP_PEMIT_ARGS
  return cudaGetLastError();
}

// scratch words needed by launch_compact and launch_peaks for F frames
int64_t consumer_scratch_words(int32_t n_frames, int64_t words, int64_t kcap) {
  const int64_t a = (int64_t)n_frames * compact_tiles(words);
  const int64_t b = (int64_t)n_frames * peak_chunks(kcap) * 9;
  return a > b ? a : b;
}

}  // namespace sep
