// sep_sparsify_noalloc: sparsification that allocates nothing.
//
// sep_sparsify keeps its scratch (a kept-pixel bitmap, per-bin thresholds and
// per-tile counts) in buffers owned by the context, grown with cudaMalloc on
// first use or when a larger batch arrives. Some callers must not allocate
// when they call: a real-time acquisition thread that must never block on
// the device allocator, or a process whose device memory is fixed after
// start-up. This variant runs the same checks and kernels with its scratch
// in one statically allocated device array instead.
//
// The array (kNoallocScratchBytes) lives in every GPU that loads the library
// until the process exits. All calls share it and it keeps the last call's
// contents; this path writes every scratch word it reads, so nothing needs
// clearing. Calls that overlap on the GPU (different streams, or host
// threads) race on the array and must be serialised by the caller.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>
#include <string>

#include "sep_internal.h"

namespace {

constexpr size_t kNoallocScratchBytes = (size_t)16 << 20;   // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Device address of g_noalloc_scratch for each device (a host variable named
// g_noalloc_scratch is only a host-side stand-in, never a device address).
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" sep_status sep_sparsify_noalloc(sep_ctx* ctx, const sep_csr* csr, const sep_calib* calib,
                                           const void* frames_dev, int32_t dtype, int32_t n_frames,
                                           const sep_params* params, const float* mean_dev, const float* sigma_dev,
                                           int32_t* idx_dev, float* val_dev, int64_t capacity, int32_t* n_kept_dev,
                                           sep_stream stream) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
  if (!ctx) return SEP_ERR_ARG;
  auto fail = [&](sep_status st, const std::string& m) {
    ctx->err = m;
    return st;
  };
  if (ctx->device < 0 || ctx->device >= kMaxDevices) return fail(SEP_ERR_ARG, "device index too large");
  // the checks of sep_sparsify, which also make the context's device current
  const sep_status st = sep::check_call(ctx, csr, calib, frames_dev, dtype, n_frames, params);
  if (st != SEP_OK) return st;
  if (capacity < 0) return fail(SEP_ERR_ARG, "capacity < 0");
  if (n_frames > 0 && (!mean_dev || !sigma_dev || !n_kept_dev || (capacity > 0 && (!idx_dev || !val_dev))))
    return fail(SEP_ERR_ARG, "NULL argument");
  if (n_frames == 0) return SEP_OK;

  // scratch layout: bitmap [F][words] | thresholds [F][nbins] | tile counts
  int64_t words = (csr->npix + 31) / 32;
  words = (words + 7) & ~(int64_t)7;
  const size_t bm_bytes = align256((size_t)(words * n_frames) * 4);
  const size_t thr_bytes = align256((size_t)n_frames * (size_t)csr->h.nbins * 4);
  const size_t aux_bytes = align256((size_t)sep::consumer_scratch_words(n_frames, words, 0) * 4);
  const size_t need = bm_bytes + thr_bytes + aux_bytes;
  if (need > kNoallocScratchBytes)
    return fail(SEP_ERR_ARG, "batch needs " + std::to_string(need) + " bytes of scratch; the static array holds " +
                                 std::to_string(kNoallocScratchBytes) + " (use fewer frames per call)");

  cudaError_t e = cudaSuccess;
  void* base;
  {
    // first call on a device: look up the array's device address (no allocation)
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[ctx->device]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return fail(SEP_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_addr[ctx->device] = p;
    }
    base = g_scratch_addr[ctx->device];
  }
  unsigned char* b = static_cast<unsigned char*>(base);
  uint32_t* bitmap = reinterpret_cast<uint32_t*>(b);
  float* thr = reinterpret_cast<float*>(b + bm_bytes);
  int32_t* aux = reinterpret_cast<int32_t*>(b + bm_bytes + thr_bytes);

  sep::PixArgs p;
  p.frames = frames_dev;
  p.npix = csr->npix;
  p.rows = csr->h.rows;
  p.cols = csr->h.cols;
  p.dtype = dtype;
  p.ped = dtype == SEP_DTYPE_U16_JF ? calib->d_ped : nullptr;
  p.gain = dtype == SEP_DTYPE_U16_JF ? calib->d_gain : nullptr;
  p.norm = csr->d_norm;
  p.bop = csr->d_bop;
  cudaStream_t s = (cudaStream_t)stream;
  // the mark kernel writes every bitmap word and the count kernel every tile
  // count, so no scratch word is read before this call writes it
  if (params->interpolate) {
    p.ia = csr->d_interp_a;
    p.it = csr->d_interp_t;
    e = sep::launch_mark_interp(p, n_frames, csr->h.nbins, mean_dev, sigma_dev, params->k_pick, bitmap, words, s);
  } else {
    e = sep::launch_thresholds(mean_dev, sigma_dev, params->k_pick, (int64_t)n_frames * csr->h.nbins, thr, s);
    if (e == cudaSuccess) e = sep::launch_mark(p, n_frames, csr->h.nbins, thr, bitmap, words, s);
  }
  if (e == cudaSuccess)
    e = sep::launch_compact(p, n_frames, bitmap, words, idx_dev, val_dev, capacity, n_kept_dev, aux, ctx->d_status, s);
  if (e != cudaSuccess) return fail(SEP_ERR_CUDA, std::string("sparsify (static scratch): ") + cudaGetErrorString(e));
  return SEP_OK;
}
