// C ABI of libsep: argument checking, device buffers owned by the handles,
// launch sequencing and CUDA-graph capture of whole batches.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "sep_internal.h"

using sep::HostCsr;

namespace {

#define SEP_VERSION_STRING "libsep 0.1 (sm_103a)"

sep_status fail(sep_ctx* ctx, sep_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}

sep_status cuda_fail(sep_ctx* ctx, cudaError_t e, const char* where) {
  if (ctx) ctx->err = std::string(where) + ": " + cudaGetErrorString(e);
  return SEP_ERR_CUDA;
}

#define SEP_CUDA(ctx, call)                                   \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call); \
  } while (0)

template <class T>
sep_status upload(sep_ctx* ctx, T** dst, const T* src, size_t n) {
  *dst = nullptr;
  if (n == 0) return SEP_OK;
  cudaError_t e = cudaMalloc((void**)dst, n * sizeof(T));
  if (e != cudaSuccess) return fail(ctx, SEP_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  e = cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy");
  return SEP_OK;
}

int64_t bitmap_words(int64_t npix) {
  int64_t w = (npix + 31) / 32;
  return (w + 7) & ~(int64_t)7;   // 32-byte multiple: vector loads per frame stay aligned
}

sep_status ensure_scratch(sep_ctx* ctx, int64_t bitmap_total, int64_t thr_total, int64_t aux_total = 0) {
  if ((size_t)aux_total > ctx->aux_len) {
    if (ctx->d_aux) cudaFree(ctx->d_aux);
    ctx->d_aux = nullptr;
    ctx->aux_len = 0;
    cudaError_t e = cudaMalloc((void**)&ctx->d_aux, (size_t)aux_total * 4);
    if (e != cudaSuccess) return fail(ctx, SEP_ERR_OOM, "consumer scratch allocation failed");
    ctx->aux_len = (size_t)aux_total;
  }
  if ((size_t)bitmap_total > ctx->bitmap_words) {
    if (ctx->d_bitmap) cudaFree(ctx->d_bitmap);
    ctx->d_bitmap = nullptr;
    ctx->bitmap_words = 0;
    cudaError_t e = cudaMalloc((void**)&ctx->d_bitmap, (size_t)bitmap_total * 4);
    if (e != cudaSuccess) return fail(ctx, SEP_ERR_OOM, "kept-pixel bitmap allocation failed");
    ctx->bitmap_words = (size_t)bitmap_total;
  }
  if ((size_t)thr_total > ctx->thr_len) {
    if (ctx->d_thr) cudaFree(ctx->d_thr);
    ctx->d_thr = nullptr;
    ctx->thr_len = 0;
    cudaError_t e = cudaMalloc((void**)&ctx->d_thr, (size_t)thr_total * 4);
    if (e != cudaSuccess) return fail(ctx, SEP_ERR_OOM, "threshold scratch allocation failed");
    ctx->thr_len = (size_t)thr_total;
  }
  return SEP_OK;
}

sep_status check_params(sep_ctx* ctx, const sep_params* p) {
  if (!p) return fail(ctx, SEP_ERR_ARG, "params is NULL");
  if (p->n_iter < 0 || p->n_iter > 1000) return fail(ctx, SEP_ERR_ARG, "n_iter out of range [0, 1000]");
  if (!(p->k_clip > 0.0f) || !isfinite(p->k_clip)) return fail(ctx, SEP_ERR_ARG, "k_clip must be finite and > 0");
  if (!(p->k_pick >= 0.0f) || !isfinite(p->k_pick)) return fail(ctx, SEP_ERR_ARG, "k_pick must be finite and >= 0");
  if (p->patch < 1 || p->patch > 15 || (p->patch & 1) == 0) return fail(ctx, SEP_ERR_ARG, "patch must be odd in [1, 15]");
  if (p->min_count < 1) return fail(ctx, SEP_ERR_ARG, "min_count must be >= 1");
  if (p->precision < SEP_PREC_PLAIN || p->precision > SEP_PREC_FP64MERGE) return fail(ctx, SEP_ERR_ARG, "unknown precision");
  for (int i = 0; i < 4; ++i)
    if (p->reserved[i] != 0) return fail(ctx, SEP_ERR_ARG, "reserved params must be 0");
  return SEP_OK;
}

sep_status check_common(sep_ctx* ctx, const sep_csr* csr, const sep_calib* calib, const void* frames, int32_t dtype,
                        int32_t n_frames, const sep_params* params) {
  if (!ctx) return SEP_ERR_ARG;
  if (!csr) return fail(ctx, SEP_ERR_ARG, "csr is NULL");
  if (csr->ctx != ctx) return fail(ctx, SEP_ERR_STATE, "csr belongs to another context");
  if (n_frames < 0) return fail(ctx, SEP_ERR_ARG, "n_frames < 0");
  if (n_frames > 0 && !frames) return fail(ctx, SEP_ERR_ARG, "frames is NULL");
  if (dtype == SEP_DTYPE_U16_JF) {
    if (!calib) return fail(ctx, SEP_ERR_ARG, "raw Jungfrau frames need a calibration");
    if (calib->ctx != ctx) return fail(ctx, SEP_ERR_STATE, "calibration belongs to another context");
    if (calib->npix != csr->npix) return fail(ctx, SEP_ERR_ARG, "calibration size differs from the detector");
  } else if (dtype != SEP_DTYPE_F32) {
    return fail(ctx, SEP_ERR_ARG, "unknown dtype");
  }
  sep_status st = check_params(ctx, params);
  if (st != SEP_OK) return st;
  SEP_CUDA(ctx, cudaSetDevice(ctx->device));
  return SEP_OK;
}

sep::PixArgs pix_args(const sep_csr* csr, const sep_calib* calib, const void* frames, int32_t dtype) {
  sep::PixArgs p;
  p.frames = frames;
  p.npix = csr->npix;
  p.rows = csr->h.rows;
  p.cols = csr->h.cols;
  p.dtype = dtype;
  p.ped = calib && dtype == SEP_DTYPE_U16_JF ? calib->d_ped : nullptr;
  p.gain = calib && dtype == SEP_DTYPE_U16_JF ? calib->d_gain : nullptr;
  p.norm = csr->d_norm;
  p.bop = csr->d_bop;
  return p;
}

sep_status check_bin_fits(sep_ctx* ctx, const sep_csr* csr) {
  int optin = 0;
  SEP_CUDA(ctx, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
  const size_t need = sep::clip_smem_bytes(csr->h.max_row, csr->has_norm) + 1024;  // + static shared memory
  if (need > (size_t)optin) {
    char buf[160];
    snprintf(buf, sizeof buf, "largest bin (%d entries) needs %zu bytes of shared memory, device allows %d",
             csr->h.max_row, need, optin);
    return fail(ctx, SEP_ERR_CSR, buf);
  }
  return SEP_OK;
}

int frames_per_cta(const sep_ctx* ctx, int32_t n_frames, int32_t nbins) {
  // enough CTAs to fill the GPU several times over, at most 8 frames per CTA
  int64_t target = (int64_t)ctx->num_sms * 16;
  int64_t fpc = ((int64_t)n_frames * nbins) / std::max<int64_t>(target, 1);
  return (int)std::min<int64_t>(std::max<int64_t>(fpc, 1), 8);
}

sep::ClipArgs clip_args(sep_ctx* ctx, const sep_csr* csr, const sep_calib* calib, const void* frames, int32_t dtype,
                        int32_t n_frames, const sep_params* pr, float* mean, float* sigma, int32_t* count,
                        float* bounds, int32_t* iters, uint32_t* bitmap, int64_t words) {
  sep::ClipArgs a;
  a.rowptr = csr->d_rowptr;
  a.grp = csr->d_grp;
  a.cal0 = calib && dtype == SEP_DTYPE_U16_JF ? calib->d_cal0 : nullptr;
  a.ent = csr->d_ent;
  a.w = csr->d_w;
  a.norm = csr->d_norm;
  a.frames = frames;
  a.npix = csr->npix;
  a.nbins = csr->h.nbins;
  a.n_frames = n_frames;
  a.frames_per_cta = frames_per_cta(ctx, n_frames, csr->h.nbins);
  a.cap = std::max(csr->h.max_row, 1);
  a.ped = calib && dtype == SEP_DTYPE_U16_JF ? calib->d_ped : nullptr;
  a.gain = calib && dtype == SEP_DTYPE_U16_JF ? calib->d_gain : nullptr;
  a.n_iter = pr->n_iter;
  a.k_clip = pr->k_clip;
  a.k_pick = pr->k_pick;
  a.mean = mean;
  a.sigma = sigma;
  a.count = count;
  a.bounds = bounds;
  a.iters = iters;
  a.bitmap = bitmap;
  a.words = words;
  return a;
}

}  // namespace

extern "C" {

const char* sep_version(void) { return SEP_VERSION_STRING; }

sep_status sep_ctx_create(int32_t device, sep_ctx** out) {
  if (!out) return SEP_ERR_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return SEP_ERR_ARG;
  sep_ctx* c = new (std::nothrow) sep_ctx();
  if (!c) return SEP_ERR_OOM;
  c->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_status, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int32_t));
  if (e != cudaSuccess) {
    if (c->d_status) cudaFree(c->d_status);
    delete c;
    return SEP_ERR_CUDA;
  }
  *out = c;
  return SEP_OK;
}

void sep_ctx_destroy(sep_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  for (auto& kv : ctx->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->d_bitmap) cudaFree(ctx->d_bitmap);
  if (ctx->d_thr) cudaFree(ctx->d_thr);
  if (ctx->d_aux) cudaFree(ctx->d_aux);
  delete ctx;
}

const char* sep_last_error(const sep_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

sep_status sep_get_device_status(sep_ctx* ctx, sep_stream stream, int32_t* status_out) {
  if (!ctx || !status_out) return SEP_ERR_ARG;
  SEP_CUDA(ctx, cudaSetDevice(ctx->device));
  int32_t v = 0;
  SEP_CUDA(ctx, cudaMemcpyAsync(&v, ctx->d_status, sizeof v, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  SEP_CUDA(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof v, (cudaStream_t)stream));
  SEP_CUDA(ctx, cudaStreamSynchronize((cudaStream_t)stream));
  *status_out = v;
  return SEP_OK;
}

sep_status sep_build_csr(sep_ctx* ctx, const sep_geometry* geom, const uint8_t* mask_host, const float* norm_host,
                         sep_csr** out) {
  if (!geom || !out) return fail(ctx, SEP_ERR_ARG, "geometry and out must not be NULL");
  *out = nullptr;
  sep_csr* c = new (std::nothrow) sep_csr();
  if (!c) return fail(ctx, SEP_ERR_OOM, "host allocation failed");
  std::string why;
  try {
    why = sep::build_csr_host(*geom, mask_host, norm_host, &c->h);
  } catch (const std::bad_alloc&) {
    delete c;
    return fail(ctx, SEP_ERR_OOM, "host allocation failed while building the matrix");
  }
  if (!why.empty()) {
    delete c;
    return fail(ctx, SEP_ERR_ARG, why);
  }
  c->ctx = ctx;
  c->npix = (int64_t)c->h.rows * c->h.cols;
  c->nnz = (int64_t)c->h.ent.size();
  c->has_norm = norm_host != nullptr;
  if (!ctx) {  // host-only matrix: inspection only
    *out = c;
    return SEP_OK;
  }
  sep_status st;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(ctx, e, "cudaSetDevice");
  }
  if ((st = upload(ctx, &c->d_rowptr, c->h.rowptr.data(), c->h.rowptr.size())) != SEP_OK ||
      (st = upload(ctx, &c->d_ent, c->h.ent.data(), c->h.ent.size())) != SEP_OK ||
      (st = upload(ctx, &c->d_bop, c->h.bop.data(), c->h.bop.size())) != SEP_OK ||
      (st = upload(ctx, &c->d_grp, c->h.grp.data(), c->h.grp.size())) != SEP_OK ||
      (c->has_norm && (st = upload(ctx, &c->d_w, c->h.w.data(), c->h.w.size())) != SEP_OK) ||
      (c->has_norm && (st = upload(ctx, &c->d_norm, norm_host, (size_t)c->npix)) != SEP_OK)) {
    sep_csr_destroy(c);
    return st;
  }
  *out = c;
  return SEP_OK;
}

void sep_csr_destroy(sep_csr* csr) {
  if (!csr) return;
  if (!csr->ctx) {  // host-only matrix
    delete csr;
    return;
  }
  cudaSetDevice(csr->ctx->device);
  cudaFree(csr->d_rowptr);
  cudaFree(csr->d_ent);
  cudaFree(csr->d_w);
  cudaFree(csr->d_norm);
  cudaFree(csr->d_bop);
  cudaFree(csr->d_grp);
  delete csr;
}

sep_status sep_csr_info(const sep_csr* csr, int64_t* npix, int32_t* nbins, int64_t* nnz, int32_t* max_row,
                        double* range) {
  if (!csr) return SEP_ERR_ARG;
  if (npix) *npix = csr->npix;
  if (nbins) *nbins = csr->h.nbins;
  if (nnz) *nnz = csr->nnz;
  if (max_row) *max_row = csr->h.max_row;
  if (range) {
    range[0] = csr->h.lo;
    range[1] = csr->h.hi;
  }
  return SEP_OK;
}

sep_status sep_csr_export(const sep_csr* csr, int32_t* rowptr, int32_t* col, float* coef, int32_t* bin_of_pixel,
                          float* bin_centers) {
  if (!csr) return SEP_ERR_ARG;
  const HostCsr& h = csr->h;
  if (rowptr) memcpy(rowptr, h.rowptr.data(), h.rowptr.size() * 4);
  if (col)
    for (size_t e = 0; e < h.ent.size(); ++e)
      col[e] = (h.ent[e] & sep::kPad) ? -1 : (int32_t)(h.ent[e] & sep::kColMask);
  if (coef) memcpy(coef, h.coef.data(), h.coef.size() * 4);
  if (bin_of_pixel) memcpy(bin_of_pixel, h.bop.data(), h.bop.size() * 4);
  if (bin_centers) memcpy(bin_centers, h.centers.data(), h.centers.size() * 4);
  return SEP_OK;
}

sep_status sep_calib_create(sep_ctx* ctx, const sep_csr* csr, const float* ped_host, const float* gain_host,
                            sep_calib** out) {
  if (!ctx) return SEP_ERR_ARG;
  if (!csr || !ped_host || !gain_host || !out) return fail(ctx, SEP_ERR_ARG, "NULL argument");
  if (csr->ctx != ctx) return fail(ctx, SEP_ERR_STATE, "csr belongs to another context");
  *out = nullptr;
  SEP_CUDA(ctx, cudaSetDevice(ctx->device));
  sep_calib* c = new (std::nothrow) sep_calib();
  if (!c) return fail(ctx, SEP_ERR_OOM, "host allocation failed");
  c->ctx = ctx;
  c->csr = csr;
  c->npix = csr->npix;
  sep_status st;
  if ((st = upload(ctx, &c->d_ped, ped_host, (size_t)(3 * c->npix))) != SEP_OK ||
      (st = upload(ctx, &c->d_gain, gain_host, (size_t)(3 * c->npix))) != SEP_OK) {
    sep_calib_destroy(c);
    return st;
  }
  // level-0 pedestal and gain copied into matrix-row order: the clip kernel
  // reads them with the entries (coalesced) instead of gathering by pixel
  try {
    const sep::HostCsr& h = csr->h;
    std::vector<float2> cal0(h.ent.size());
    for (size_t e = 0; e < h.ent.size(); ++e) {
      if (h.ent[e] & sep::kPad) {
        cal0[e] = make_float2(0.0f, 1.0f);
      } else {
        const size_t col = h.ent[e] & sep::kColMask;
        cal0[e] = make_float2(ped_host[col], gain_host[col]);
      }
    }
    if ((st = upload(ctx, &c->d_cal0, cal0.data(), cal0.size())) != SEP_OK) {
      sep_calib_destroy(c);
      return st;
    }
  } catch (const std::bad_alloc&) {
    sep_calib_destroy(c);
    return fail(ctx, SEP_ERR_OOM, "host allocation failed");
  }
  *out = c;
  return SEP_OK;
}

void sep_calib_destroy(sep_calib* calib) {
  if (!calib) return;
  if (calib->ctx) cudaSetDevice(calib->ctx->device);
  cudaFree(calib->d_ped);
  cudaFree(calib->d_gain);
  cudaFree(calib->d_cal0);
  delete calib;
}

sep_status sep_integrate_clip(sep_ctx* ctx, const sep_csr* csr, const sep_calib* calib, const void* frames_dev,
                              int32_t dtype, int32_t n_frames, const sep_params* params, float* mean_dev,
                              float* sigma_dev, int32_t* count_dev, float* bounds_dev, int32_t* iters_dev,
                              sep_stream stream) {
  sep_status st = check_common(ctx, csr, calib, frames_dev, dtype, n_frames, params);
  if (st != SEP_OK) return st;
  if (n_frames > 0 && (!mean_dev || !sigma_dev || !count_dev)) return fail(ctx, SEP_ERR_ARG, "NULL output");
  if ((st = check_bin_fits(ctx, csr)) != SEP_OK) return st;
  if (n_frames == 0) return SEP_OK;
  sep::ClipArgs a = clip_args(ctx, csr, calib, frames_dev, dtype, n_frames, params, mean_dev, sigma_dev, count_dev,
                              bounds_dev, iters_dev, nullptr, 0);
  cudaError_t e = sep::launch_integrate_clip(a, dtype, csr->h.split > 1, csr->has_norm, params->precision, 0,
                                             (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "integrate_clip launch");
  return SEP_OK;
}

sep_status sep_sparsify(sep_ctx* ctx, const sep_csr* csr, const sep_calib* calib, const void* frames_dev,
                        int32_t dtype, int32_t n_frames, const sep_params* params, const float* mean_dev,
                        const float* sigma_dev, int32_t* idx_dev, float* val_dev, int64_t capacity,
                        int32_t* n_kept_dev, sep_stream stream) {
  sep_status st = check_common(ctx, csr, calib, frames_dev, dtype, n_frames, params);
  if (st != SEP_OK) return st;
  if (capacity < 0) return fail(ctx, SEP_ERR_ARG, "capacity < 0");
  if (n_frames > 0 && (!mean_dev || !sigma_dev || !n_kept_dev || (capacity > 0 && (!idx_dev || !val_dev))))
    return fail(ctx, SEP_ERR_ARG, "NULL argument");
  if (n_frames == 0) return SEP_OK;
  const int64_t words = bitmap_words(csr->npix);
  if ((st = ensure_scratch(ctx, words * n_frames, (int64_t)n_frames * csr->h.nbins,
                           sep::consumer_scratch_words(n_frames, words, capacity))) != SEP_OK)
    return st;
  cudaStream_t s = (cudaStream_t)stream;
  sep::PixArgs p = pix_args(csr, calib, frames_dev, dtype);
  cudaError_t e = sep::launch_thresholds(mean_dev, sigma_dev, params->k_pick, (int64_t)n_frames * csr->h.nbins,
                                         ctx->d_thr, s);
  if (e == cudaSuccess) e = sep::launch_mark(p, n_frames, csr->h.nbins, ctx->d_thr, ctx->d_bitmap, words, s);
  if (e == cudaSuccess)
    e = sep::launch_compact(p, n_frames, ctx->d_bitmap, words, idx_dev, val_dev, capacity, n_kept_dev, ctx->d_aux,
                            ctx->d_status, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sparsify launch");
  return SEP_OK;
}

sep_status sep_peakfind(sep_ctx* ctx, const sep_csr* csr, const sep_calib* calib, const void* frames_dev,
                        int32_t dtype, int32_t n_frames, const sep_params* params, const float* mean_dev,
                        const float* sigma_dev, const int32_t* idx_dev, const int32_t* n_kept_dev,
                        int64_t kept_capacity, sep_peak* peaks_dev, int64_t capacity, int32_t* n_peaks_dev,
                        sep_stream stream) {
  sep_status st = check_common(ctx, csr, calib, frames_dev, dtype, n_frames, params);
  if (st != SEP_OK) return st;
  if (capacity < 0 || kept_capacity < 0) return fail(ctx, SEP_ERR_ARG, "capacity < 0");
  if (n_frames > 0 && (!mean_dev || !sigma_dev || !n_kept_dev || !n_peaks_dev || (kept_capacity > 0 && !idx_dev) ||
                       (capacity > 0 && !peaks_dev)))
    return fail(ctx, SEP_ERR_ARG, "NULL argument");
  if (n_frames == 0) return SEP_OK;
  const int64_t words = bitmap_words(csr->npix);
  if ((st = ensure_scratch(ctx, words * n_frames, 0, sep::consumer_scratch_words(n_frames, words, kept_capacity))) !=
      SEP_OK)
    return st;
  cudaStream_t s = (cudaStream_t)stream;
  sep::PixArgs p = pix_args(csr, calib, frames_dev, dtype);
  cudaError_t e = cudaMemsetAsync(ctx->d_bitmap, 0, (size_t)(words * n_frames) * 4, s);
  if (e == cudaSuccess)
    e = sep::launch_scatter_list(n_frames, idx_dev, n_kept_dev, kept_capacity, csr->npix, ctx->d_bitmap, words, s);
  if (e == cudaSuccess)
    e = sep::launch_peaks(p, n_frames, csr->h.nbins, mean_dev, sigma_dev, ctx->d_bitmap, words, idx_dev, n_kept_dev,
                          kept_capacity, params->patch, params->min_count, peaks_dev, capacity, n_peaks_dev,
                          ctx->d_aux, ctx->d_status, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "peakfind launch");
  return SEP_OK;
}

sep_status sep_process_batch(sep_ctx* ctx, const sep_csr* csr, const sep_calib* calib, const void* frames_dev,
                             int32_t dtype, int32_t n_frames, const sep_params* params, float* mean_dev,
                             float* sigma_dev, int32_t* count_dev, int32_t* idx_dev, float* val_dev,
                             int64_t kept_capacity, int32_t* n_kept_dev, sep_peak* peaks_dev, int64_t peak_capacity,
                             int32_t* n_peaks_dev, int32_t use_graph, sep_stream stream) {
  sep_status st = check_common(ctx, csr, calib, frames_dev, dtype, n_frames, params);
  if (st != SEP_OK) return st;
  if (kept_capacity < 0 || peak_capacity < 0) return fail(ctx, SEP_ERR_ARG, "capacity < 0");
  if (n_frames > 0 && (!mean_dev || !sigma_dev || !count_dev || !n_kept_dev || !n_peaks_dev ||
                       (kept_capacity > 0 && (!idx_dev || !val_dev)) || (peak_capacity > 0 && !peaks_dev)))
    return fail(ctx, SEP_ERR_ARG, "NULL argument");
  if ((st = check_bin_fits(ctx, csr)) != SEP_OK) return st;
  if (n_frames == 0) return SEP_OK;
  const int64_t words = bitmap_words(csr->npix);
  if ((st = ensure_scratch(ctx, words * n_frames, 0, sep::consumer_scratch_words(n_frames, words, kept_capacity))) !=
      SEP_OK)
    return st;
  cudaStream_t s = (cudaStream_t)stream;

  auto enqueue = [&](int mode) -> cudaError_t {
    sep::ClipArgs a = clip_args(ctx, csr, calib, frames_dev, dtype, n_frames, params, mean_dev, sigma_dev, count_dev,
                                nullptr, nullptr, ctx->d_bitmap, words);
    sep::PixArgs p = pix_args(csr, calib, frames_dev, dtype);
    cudaError_t e = cudaMemsetAsync(ctx->d_bitmap, 0, (size_t)(words * n_frames) * 4, s);
    if (e == cudaSuccess)
      e = sep::launch_integrate_clip(a, dtype, csr->h.split > 1, csr->has_norm, params->precision, mode, s);
    if (e == cudaSuccess)
      e = sep::launch_compact(p, n_frames, ctx->d_bitmap, words, idx_dev, val_dev, kept_capacity, n_kept_dev,
                              ctx->d_aux, ctx->d_status, s);
    if (e == cudaSuccess)
      e = sep::launch_peaks(p, n_frames, csr->h.nbins, mean_dev, sigma_dev, ctx->d_bitmap, words, idx_dev,
                            n_kept_dev, kept_capacity, params->patch, params->min_count, peaks_dev, peak_capacity,
                            n_peaks_dev, ctx->d_aux, ctx->d_status, s);
    return e;
  };

  if (!use_graph || s == nullptr) {
    cudaError_t e = enqueue(0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "process_batch launch");
    return SEP_OK;
  }
  // one executable graph per distinct set of launch arguments
  std::vector<uint64_t> key = {(uint64_t)(uintptr_t)csr, (uint64_t)(uintptr_t)calib, (uint64_t)(uintptr_t)frames_dev,
                               (uint64_t)dtype, (uint64_t)n_frames, (uint64_t)(uintptr_t)mean_dev,
                               (uint64_t)(uintptr_t)sigma_dev, (uint64_t)(uintptr_t)count_dev,
                               (uint64_t)(uintptr_t)idx_dev, (uint64_t)(uintptr_t)val_dev, (uint64_t)kept_capacity,
                               (uint64_t)(uintptr_t)n_kept_dev, (uint64_t)(uintptr_t)peaks_dev,
                               (uint64_t)peak_capacity, (uint64_t)(uintptr_t)n_peaks_dev,
                               (uint64_t)(uintptr_t)ctx->d_bitmap, (uint64_t)(uintptr_t)ctx->d_aux,
                               (uint64_t)(uintptr_t)s};
  {
    uint32_t pw[sizeof(sep_params) / 4];
    memcpy(pw, params, sizeof(sep_params));
    for (uint32_t w : pw) key.push_back(w);
  }
  auto it = ctx->graphs.find(key);
  if (it == ctx->graphs.end()) {
    if (ctx->graphs.size() >= 16) {   // drop the least recently used
      auto lru = ctx->graphs.begin();
      for (auto j = ctx->graphs.begin(); j != ctx->graphs.end(); ++j)
        if (j->second.last_use < lru->second.last_use) lru = j;
      cudaGraphExecDestroy(lru->second.exec);
      cudaGraphDestroy(lru->second.graph);
      ctx->graphs.erase(lru);
    }
    // the kernel attribute is set before the capture, which then records launches only
    sep::ClipArgs a0 = clip_args(ctx, csr, calib, frames_dev, dtype, n_frames, params, mean_dev, sigma_dev, count_dev,
                                 nullptr, nullptr, ctx->d_bitmap, words);
    cudaError_t e = sep::launch_integrate_clip(a0, dtype, csr->h.split > 1, csr->has_norm, params->precision, 1, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel attribute");
    sep_graph_entry g;
    SEP_CUDA(ctx, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    e = enqueue(2);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail(ctx, e != cudaSuccess ? e : e2, "process_batch capture");
    }
    g.graph = graph;
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(graph);
      return cuda_fail(ctx, e, "cudaGraphInstantiate");
    }
    it = ctx->graphs.emplace(key, g).first;
  }
  it->second.last_use = ++ctx->use_clock;
  SEP_CUDA(ctx, cudaGraphLaunch(it->second.exec, s));
  return SEP_OK;
}

}  // extern "C"
