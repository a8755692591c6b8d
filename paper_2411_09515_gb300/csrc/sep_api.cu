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

// Row stride of a frame's staged values: one slot per matrix entry, rounded
// up to 32 floats so every frame's row starts 128-byte aligned (vector loads).
int64_t stage_stride(const sep_csr* csr) { return ((int64_t)csr->h.ent.size() + 31) & ~(int64_t)31; }

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

// Staged values of a batch: floats [total] (grown on demand, never inside a capture).
sep_status ensure_stage(sep_ctx* ctx, int64_t total) {
  if ((size_t)total > ctx->stage_len) {
    if (ctx->d_stage) cudaFree(ctx->d_stage);
    ctx->d_stage = nullptr;
    ctx->stage_len = 0;
    cudaError_t e = cudaMalloc((void**)&ctx->d_stage, (size_t)total * 4);
    if (e != cudaSuccess) return fail(ctx, SEP_ERR_OOM, "staging buffer allocation failed");
    ctx->stage_len = (size_t)total;
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
  if (p->precision < SEP_PREC_PLAIN || p->precision > SEP_PREC_DWORD) return fail(ctx, SEP_ERR_ARG, "unknown precision");
  if (p->surrogate < 0 || p->surrogate > 8) return fail(ctx, SEP_ERR_ARG, "surrogate must be in [0, 8]");
  if (p->surrogate > 0 && p->precision != SEP_PREC_DWORD)
    return fail(ctx, SEP_ERR_ARG, "the surrogate runs in precision SEP_PREC_DWORD only");
  if (p->cutoff != SEP_CUTOFF_FIXED && p->cutoff != SEP_CUTOFF_CHAUVENET)
    return fail(ctx, SEP_ERR_ARG, "cutoff must be SEP_CUTOFF_FIXED or SEP_CUTOFF_CHAUVENET");
  if (p->cutoff == SEP_CUTOFF_CHAUVENET && p->surrogate > 0)
    return fail(ctx, SEP_ERR_ARG, "the surrogate predicts fixed-cut-off clipping only");
  if (p->error_model != SEP_ERROR_AZIMUTHAL && p->error_model != SEP_ERROR_POISSON &&
      p->error_model != SEP_ERROR_HYBRID)
    return fail(ctx, SEP_ERR_ARG, "error_model must be SEP_ERROR_AZIMUTHAL, _POISSON or _HYBRID");
  if (!(p->dark_var >= 0.0f) || !isfinite(p->dark_var)) return fail(ctx, SEP_ERR_ARG, "dark_var must be finite and >= 0");
  if (p->error_model != SEP_ERROR_AZIMUTHAL && p->surrogate > 0)
    return fail(ctx, SEP_ERR_ARG, "the surrogate predicts azimuthal-model clipping only");
  if (p->interpolate != 0 && p->interpolate != 1) return fail(ctx, SEP_ERR_ARG, "interpolate must be 0 or 1");
  return SEP_OK;
}

sep_status check_common(sep_ctx* ctx, const sep_csr* csr, const sep_calib* calib, const void* frames, int32_t dtype,
                        int32_t n_frames, const sep_params* params, bool chunked = false) {
  if (!ctx) return SEP_ERR_ARG;
  if (!csr) return fail(ctx, SEP_ERR_ARG, "csr is NULL");
  if (csr->ctx != ctx) return fail(ctx, SEP_ERR_STATE, "csr belongs to another context");
  if (n_frames < 0) return fail(ctx, SEP_ERR_ARG, "n_frames < 0");
  if (n_frames > SEP_MAX_FRAMES && !chunked) return fail(ctx, SEP_ERR_ARG, "n_frames above SEP_MAX_FRAMES");
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
  if (params->error_model != SEP_ERROR_AZIMUTHAL && csr->has_norm)
    return fail(ctx, SEP_ERR_ARG, "the Poisson and hybrid models take frames without a norm");
  if (params->surrogate > 0 && !csr->model) return fail(ctx, SEP_ERR_STATE, "surrogate requested but no model attached");
  if (params->surrogate > 0 && csr->model->ctx != ctx) return fail(ctx, SEP_ERR_STATE, "model belongs to another context");
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

// The consumers' background at the pixel centre (params->interpolate).
void set_interp(sep::PixArgs& p, const sep_csr* csr, const sep_params* params) {
  if (params->interpolate) {
    p.ia = csr->d_interp_a;
    p.it = csr->d_interp_t;
  }
}

sep_status check_bin_fits(sep_ctx* ctx, const sep_csr* csr) {
  // the clip kernel keeps an entry's index inside its row in 16 bits and, with
  // per-entry weights, the longest row's weights in shared memory
  if (csr->h.max_row >= 65536) {
    char buf[120];
    snprintf(buf, sizeof buf, "largest bin has %d entries; at most 65535 are supported", csr->h.max_row);
    return fail(ctx, SEP_ERR_CSR, buf);
  }
  int optin = 0;
  SEP_CUDA(ctx, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
  const size_t need = sep::clip_smem_bytes(csr->h.max_row, csr->weighted) + sep::kClipStaticSmem;
  if (need > (size_t)optin) {
    char buf[160];
    snprintf(buf, sizeof buf, "largest bin (%d entries) needs %zu bytes of shared memory, device allows %d",
             csr->h.max_row, need, optin);
    return fail(ctx, SEP_ERR_CSR, buf);
  }
  return SEP_OK;
}

void free_plan(sep_csr* csr) {
  for (auto& c : csr->plan) cudaFree(c.d_bins);
  csr->plan.clear();
}

// Partition the bins by row length at the given thresholds (ascending); class
// i holds rows with thr[i-1] < n <= thr[i], the last class everything longer.
sep_status make_plan(sep_ctx* ctx, sep_csr* csr, int32_t n_classes, const int32_t* thresholds, const int32_t* tpb) {
  if (n_classes < 1 || n_classes > 4) return fail(ctx, SEP_ERR_ARG, "1 to 4 classes");
  for (int i = 0; i < n_classes; ++i) {
    if (tpb[i] != 32 && tpb[i] != 64 && tpb[i] != 128 && tpb[i] != 256)
      return fail(ctx, SEP_ERR_ARG, "threads per block: 32, 64, 128 or 256");
    if (i + 1 < n_classes && (thresholds[i] < 1 || (i > 0 && thresholds[i] <= thresholds[i - 1])))
      return fail(ctx, SEP_ERR_ARG, "thresholds must ascend");
  }
  std::vector<std::vector<int32_t>> bins(n_classes);
  const auto& rp = csr->h.rowptr;
  for (int32_t b = 0; b < csr->h.nbins; ++b) {
    const int32_t n = rp[b + 1] - rp[b];
    int c = 0;
    while (c + 1 < n_classes && n > thresholds[c]) ++c;
    bins[c].push_back(b);
  }
  free_plan(csr);
  for (int c = 0; c < n_classes; ++c) {
    sep_clip_class k;
    k.tpb = tpb[c];
    k.threshold = c + 1 < n_classes ? thresholds[c] : 0;
    if (bins[c].empty()) continue;
    std::stable_sort(bins[c].begin(), bins[c].end(),
                     [&](int32_t x, int32_t y) { return rp[x + 1] - rp[x] > rp[y + 1] - rp[y]; });
    k.n_bins = (int32_t)bins[c].size();
    k.cap = std::max(rp[bins[c][0] + 1] - rp[bins[c][0]], 4);
    sep_status st = upload(ctx, &k.d_bins, bins[c].data(), bins[c].size());
    if (st != SEP_OK) {
      free_plan(csr);
      return st;
    }
    csr->plan.push_back(k);
  }
  csr->plan_version += 1;
  return SEP_OK;
}

// block size of the clip kernel without a plan (one warp per item)
constexpr int32_t kDefaultTpb = 32;

int frames_per_cta(const sep_ctx* ctx, int32_t n_frames, int32_t nbins, int32_t tpb = 32) {
  // enough CTAs to fill the GPU several times over, at most 4 frames per
  // warp; the clip kernel gives each warp of a CTA its own frames, so a
  // CTA takes a multiple of its warps
  const int64_t target = (int64_t)ctx->num_sms * 16;
  int64_t fpc = ((int64_t)n_frames * nbins) / std::max<int64_t>(target, 1);
  fpc = std::min<int64_t>(std::max<int64_t>(fpc, 1), 4);
  const int64_t w = std::max(tpb / 32, 1);
  return (int)(((fpc + w - 1) / w) * w);
}

sep::ClipArgs clip_args(sep_ctx* ctx, const sep_csr* csr, const float* stage, int32_t n_frames, const sep_params* pr,
                        float* mean, float* sigma, int32_t* count, float* bounds, int32_t* iters, float* thr_out) {
  sep::ClipArgs a;
  a.bin_list = nullptr;
  a.rowptr = csr->d_rowptr;
  a.grp = csr->d_grp;
  a.ent = csr->d_ent;
  a.w = csr->d_w;
  a.stage = stage;
  a.cpix = csr->d_cpix;
  a.npos = stage_stride(csr);
  a.nbins = csr->h.nbins;
  a.n_frames = n_frames;
  a.frames_per_cta = frames_per_cta(ctx, n_frames, csr->h.nbins);
  a.cap = std::max(csr->h.max_row, 1);
  a.n_iter = pr->n_iter;
  a.k_clip = pr->k_clip;
  a.cutoff = pr->cutoff;
  a.error_model = pr->error_model;
  a.dark_var = pr->dark_var;
  a.k_pick = pr->k_pick;
  a.mean = mean;
  a.sigma = sigma;
  a.count = count;
  a.bounds = bounds;
  a.iters = iters;
  a.thr_out = thr_out;
  if (ctx->clip_stats_on) a.clip_stats = ctx->d_clip_stats;
  if (pr->surrogate > 0 && csr->model) {
    a.mlp_w = csr->model->d_wbt;
    a.mlp_norm = csr->model->d_norm;
    a.surr_stats = ctx->d_surr;
  }
  return a;
}

// Correction + staging of n frames (contiguous at `frames`, or listed in
// fptr) into stage [n][stage_stride].
cudaError_t enqueue_stage(sep_ctx* ctx, const sep_csr* csr, const sep_calib* calib, const void* frames,
                          const uint64_t* fptr, int32_t dtype, int32_t n, float* stage, cudaStream_t s) {
  sep::StageArgs g;
  g.frames = frames;
  g.fptr = fptr;
  g.npix = csr->npix;
  g.npos = stage_stride(csr);
  g.rows = csr->h.rows;
  g.cols = csr->h.cols;
  g.tiles_x = csr->h.tiles_x;
  g.tiles_y = csr->h.tiles_y;
  g.n_frames = n;
  g.frames_per_cta = std::min(n, 32);   // calibration and ranks are read once per CTA
  g.ped = calib && dtype == SEP_DTYPE_U16_JF ? calib->d_ped : nullptr;
  g.gain = calib && dtype == SEP_DTYPE_U16_JF ? calib->d_gain : nullptr;
  g.norm = csr->d_norm;
  g.tile_ebase = csr->d_tile_ebase;
  g.tile_sc = csr->d_tile_sc;
  g.stage = stage;
  return sep::launch_stage(g, dtype, csr->has_norm, s);
}

// Launch the clip kernel for every size class of the plan: one class on the
// caller's stream, several as parallel branches (fork / join through events,
// which a stream capture records as graph edges).
cudaError_t enqueue_clip(sep_ctx* ctx, const sep_csr* csr, sep::ClipArgs a, int32_t precision, int mode,
                         cudaStream_t s, bool allow_fork = true) {
  const bool split = csr->h.split > 1;
  // each launch its own work-queue counter (launches of a call run concurrently)
  auto take_queue = [&]() { return ctx->d_queue + (ctx->queue_next++ % sep_ctx::kQueueSlots); };
  if (csr->plan.empty()) {
    a.queue = take_queue();
    a.bin_list = nullptr;
    a.cap = std::max(csr->h.max_row, 4);
    a.frames_per_cta = frames_per_cta(ctx, a.n_frames, csr->h.nbins, kDefaultTpb);
    return sep::launch_integrate_clip(a, csr->h.nbins, kDefaultTpb, split, csr->weighted, precision, mode, s);
  }
  const int nc = (int)csr->plan.size();
  if (nc == 1 || mode == 1 || !allow_fork) {
    for (const auto& k : csr->plan) {
      a.queue = take_queue();
      a.bin_list = k.d_bins;
      a.cap = k.cap;
      a.frames_per_cta = frames_per_cta(ctx, a.n_frames, k.n_bins, k.tpb);
      cudaError_t e = sep::launch_integrate_clip(a, k.n_bins, k.tpb, split, csr->weighted, precision, mode, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  cudaError_t e = cudaEventRecord(ctx->ev_fork, s);
  for (int i = 0; i < nc && e == cudaSuccess; ++i) {
    const auto& k = csr->plan[i];
    cudaStream_t si = i == 0 ? s : ctx->aux[i];
    if (i > 0) e = cudaStreamWaitEvent(si, ctx->ev_fork, 0);
    a.queue = take_queue();
    a.bin_list = k.d_bins;
    a.cap = k.cap;
    a.frames_per_cta = frames_per_cta(ctx, a.n_frames, k.n_bins, k.tpb);
    if (e == cudaSuccess)
      e = sep::launch_integrate_clip(a, k.n_bins, k.tpb, split, csr->weighted, precision, mode, si);
    if (e == cudaSuccess && i > 0) e = cudaEventRecord(ctx->ev_join[i], si);
  }
  for (int i = 1; i < nc && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(s, ctx->ev_join[i], 0);
  return e;
}

}  // namespace

namespace sep {
sep_status check_call(sep_ctx* ctx, const sep_csr* csr, const sep_calib* calib, const void* frames, int32_t dtype,
                      int32_t n_frames, const sep_params* params) {
  return check_common(ctx, csr, calib, frames, dtype, n_frames, params);
}
}  // namespace sep

extern "C" {

const char* sep_version(void) { return SEP_VERSION_STRING; }

sep_status sep_ctx_create(int32_t device, sep_ctx** out) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
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
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_surr, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(c->d_surr, 0, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_clip_stats, SEP_CLIP_STATS * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(c->d_clip_stats, 0, SEP_CLIP_STATS * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_queue, sep_ctx::kQueueSlots * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(c->d_queue, 0, sep_ctx::kQueueSlots * sizeof(int32_t));
  for (int i = 1; i < 4 && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&c->aux[i], cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
  for (int i = 1; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&c->ev_join[i], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    if (c->d_status) cudaFree(c->d_status);
    if (c->d_surr) cudaFree(c->d_surr);
    if (c->d_clip_stats) cudaFree(c->d_clip_stats);
    if (c->d_queue) cudaFree(c->d_queue);
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
  if (ctx->d_surr) cudaFree(ctx->d_surr);
  if (ctx->d_clip_stats) cudaFree(ctx->d_clip_stats);
  if (ctx->d_queue) cudaFree(ctx->d_queue);
  if (ctx->d_bitmap) cudaFree(ctx->d_bitmap);
  if (ctx->d_thr) cudaFree(ctx->d_thr);
  if (ctx->d_aux) cudaFree(ctx->d_aux);
  if (ctx->d_stage) cudaFree(ctx->d_stage);
  if (ctx->d_pipe) cudaFree(ctx->d_pipe);
  for (int j = 0; j < sep_ctx::kCopyStreams; ++j)
    if (ctx->s_in[j]) cudaStreamDestroy(ctx->s_in[j]);
  if (ctx->s_out) cudaStreamDestroy(ctx->s_out);
  for (int i = 0; i < sep_ctx::kSlots; ++i) {
    for (int j = 0; j < sep_ctx::kCopyStreams; ++j)
      if (ctx->ev_in[i][j]) cudaEventDestroy(ctx->ev_in[i][j]);
    if (ctx->ev_done[i]) cudaEventDestroy(ctx->ev_done[i]);
    if (ctx->ev_out[i]) cudaEventDestroy(ctx->ev_out[i]);
  }
  if (ctx->ev_start) cudaEventDestroy(ctx->ev_start);
  if (ctx->d_desc) cudaFree(ctx->d_desc);
  if (ctx->h_desc) cudaFreeHost(ctx->h_desc);
  for (int i = 1; i < 4; ++i) {
    if (ctx->aux[i]) cudaStreamDestroy(ctx->aux[i]);
    if (ctx->ev_join[i]) cudaEventDestroy(ctx->ev_join[i]);
  }
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  delete ctx;
}

const char* sep_last_error(const sep_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

sep_status sep_get_device_status(sep_ctx* ctx, sep_stream stream, int32_t* status_out) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
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
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
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
  c->weighted = c->has_norm || c->h.split == 0;
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
      (st = upload(ctx, &c->d_cpix, c->h.cpix.data(), c->h.cpix.size())) != SEP_OK ||
      (st = upload(ctx, &c->d_interp_a, c->h.interp_a.data(), c->h.interp_a.size())) != SEP_OK ||
      (st = upload(ctx, &c->d_interp_t, c->h.interp_t.data(), c->h.interp_t.size())) != SEP_OK ||
      (st = upload(ctx, &c->d_bop, c->h.bop.data(), c->h.bop.size())) != SEP_OK ||
      (st = upload(ctx, &c->d_grp, c->h.grp.data(), c->h.grp.size())) != SEP_OK ||
      (st = upload(ctx, &c->d_pos_of, c->h.slot_of.data(), c->h.slot_of.size())) != SEP_OK ||
      (st = upload(ctx, &c->d_tile_ebase, c->h.tile_ebase.data(), c->h.tile_ebase.size())) != SEP_OK ||
      (st = upload(ctx, &c->d_tile_sc, reinterpret_cast<const int2*>(c->h.tile_sc.data()),
                   c->h.tile_sc.size() / 2)) != SEP_OK ||
      (c->weighted && (st = upload(ctx, &c->d_w, c->h.w.data(), c->h.w.size())) != SEP_OK) ||
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
  free_plan(csr);
  cudaFree(csr->d_rowptr);
  cudaFree(csr->d_ent);
  cudaFree(csr->d_cpix);
  cudaFree(csr->d_interp_a);
  cudaFree(csr->d_interp_t);
  cudaFree(csr->d_w);
  cudaFree(csr->d_norm);
  cudaFree(csr->d_bop);
  cudaFree(csr->d_grp);
  cudaFree(csr->d_pos_of);
  cudaFree(csr->d_tile_ebase);
  cudaFree(csr->d_tile_sc);
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

sep_status sep_csr_staging(const sep_csr* csr, int32_t* perm_inv, int64_t* npos) {
  if (!csr) return SEP_ERR_ARG;
  if (perm_inv) memcpy(perm_inv, csr->h.perm_inv.data(), csr->h.perm_inv.size() * 4);
  if (npos) *npos = csr->h.npos;
  return SEP_OK;
}

sep_status sep_csr_interp(const sep_csr* csr, int32_t* lower_bin, float* weight) {
  if (!csr) return SEP_ERR_ARG;
  const size_t n = (size_t)csr->npix;
  if (csr->h.interp_a.size() != n || csr->h.interp_t.size() != n) return SEP_ERR_CSR;
  if (lower_bin) memcpy(lower_bin, csr->h.interp_a.data(), n * sizeof(int32_t));
  if (weight) memcpy(weight, csr->h.interp_t.data(), n * sizeof(float));
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

sep_status sep_csr_validate(const int32_t* rowptr, const int32_t* col, const float* coef, const int32_t* bin_of_pixel,
                            int32_t nbins, int64_t nnz, int64_t npix, int64_t calib_npix, char* msg, int32_t msg_len) {
  std::string why;
  try {
    why = sep::validate_matrix(rowptr, col, coef, bin_of_pixel, nbins, nnz, npix);
  } catch (const std::bad_alloc&) {
    why = "host allocation failed";
  }
  if (why.empty() && calib_npix >= 0 && calib_npix != npix) why = "calibration covers another number of pixels";
  if (msg && msg_len > 0) {
    const size_t n = std::min(why.size(), (size_t)msg_len - 1);
    memcpy(msg, why.data(), n);
    msg[n] = 0;
  }
  return why.empty() ? SEP_OK : SEP_ERR_ARG;
}

sep_status sep_csr_check(const sep_csr* csr, const sep_calib* calib) {
  if (!csr) return SEP_ERR_ARG;
  sep_ctx* ctx = csr->ctx;
  std::string why;
  try {
    why = sep::validate_host_csr(csr->h);
  } catch (const std::bad_alloc&) {
    return fail(ctx, SEP_ERR_OOM, "host allocation failed");
  }
  if (!why.empty()) return fail(ctx, SEP_ERR_ARG, why);
  if (calib && calib->npix != csr->npix) return fail(ctx, SEP_ERR_ARG, "calibration size differs from the detector");
  if (calib && ctx && calib->ctx != ctx) return fail(ctx, SEP_ERR_STATE, "calibration belongs to another context");
  return SEP_OK;
}

sep_status sep_calib_create(sep_ctx* ctx, const sep_csr* csr, const float* ped_host, const float* gain_host,
                            sep_calib** out) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
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
  *out = c;
  return SEP_OK;
}

void sep_calib_destroy(sep_calib* calib) {
  if (!calib) return;
  if (calib->ctx) cudaSetDevice(calib->ctx->device);
  cudaFree(calib->d_ped);
  cudaFree(calib->d_gain);
  delete calib;
}

sep_status sep_integrate_clip(sep_ctx* ctx, const sep_csr* csr, const sep_calib* calib, const void* frames_dev,
                              int32_t dtype, int32_t n_frames, const sep_params* params, float* mean_dev,
                              float* sigma_dev, int32_t* count_dev, float* bounds_dev, int32_t* iters_dev,
                              sep_stream stream) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
  sep_status st = check_common(ctx, csr, calib, frames_dev, dtype, n_frames, params);
  if (st != SEP_OK) return st;
  if (n_frames > 0 && (!mean_dev || !sigma_dev || !count_dev)) return fail(ctx, SEP_ERR_ARG, "NULL output");
  if ((st = check_bin_fits(ctx, csr)) != SEP_OK) return st;
  if (n_frames == 0) return SEP_OK;
  if ((st = ensure_stage(ctx, stage_stride(csr) * n_frames)) != SEP_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  sep::ClipArgs a = clip_args(ctx, csr, ctx->d_stage, n_frames, params, mean_dev, sigma_dev, count_dev, bounds_dev,
                              iters_dev, nullptr);
  cudaError_t e = enqueue_stage(ctx, csr, calib, frames_dev, nullptr, dtype, n_frames, ctx->d_stage, s);
  if (e == cudaSuccess) e = enqueue_clip(ctx, csr, a, params->precision, 0, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "integrate_clip launch");
  return SEP_OK;
}

sep_status sep_correct(sep_ctx* ctx, const sep_csr* csr, const sep_calib* calib, const void* frames_dev,
                       int32_t dtype, int32_t n_frames, float* out_dev, sep_stream stream) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
  sep_params p{};
  p.n_iter = 0;
  p.k_clip = 1.0f;
  p.k_pick = 0.0f;
  p.patch = 1;
  p.min_count = 1;
  p.precision = SEP_PREC_DWORD;
  sep_status st = check_common(ctx, csr, calib, frames_dev, dtype, n_frames, &p);
  if (st != SEP_OK) return st;
  if (n_frames > 0 && !out_dev) return fail(ctx, SEP_ERR_ARG, "NULL output");
  if (n_frames == 0) return SEP_OK;
  if ((st = ensure_stage(ctx, stage_stride(csr) * n_frames)) != SEP_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = enqueue_stage(ctx, csr, calib, frames_dev, nullptr, dtype, n_frames, ctx->d_stage, s);
  if (e == cudaSuccess)
    e = sep::launch_unstage(ctx->d_stage, stage_stride(csr), csr->d_pos_of, csr->npix, n_frames, out_dev, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "correct launch");
  return SEP_OK;
}

sep_status sep_surrogate_record(sep_ctx* ctx, const sep_csr* csr, const sep_calib* calib, const void* frames_dev,
                                int32_t dtype, int32_t n_frames, const sep_params* params, float* mean_dev,
                                float* sigma_dev, int32_t* count_dev, float* feat_dev, float* target_dev,
                                sep_stream stream) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
  sep_status st = check_common(ctx, csr, calib, frames_dev, dtype, n_frames, params);
  if (st != SEP_OK) return st;
  if (params->surrogate != 0) return fail(ctx, SEP_ERR_ARG, "recording runs the plain loop: surrogate must be 0");
  if (params->precision != SEP_PREC_DWORD) return fail(ctx, SEP_ERR_ARG, "recording runs in SEP_PREC_DWORD only");
  if (n_frames > 0 && (!mean_dev || !sigma_dev || !count_dev || !feat_dev || !target_dev))
    return fail(ctx, SEP_ERR_ARG, "NULL output");
  if ((st = check_bin_fits(ctx, csr)) != SEP_OK) return st;
  if (n_frames == 0) return SEP_OK;
  if ((st = ensure_stage(ctx, stage_stride(csr) * n_frames)) != SEP_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  sep::ClipArgs a = clip_args(ctx, csr, ctx->d_stage, n_frames, params, mean_dev, sigma_dev, count_dev, nullptr,
                              nullptr, nullptr);
  a.rec_feat = feat_dev;
  a.rec_target = target_dev;
  cudaError_t e = enqueue_stage(ctx, csr, calib, frames_dev, nullptr, dtype, n_frames, ctx->d_stage, s);
  if (e == cudaSuccess) e = enqueue_clip(ctx, csr, a, params->precision, 0, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "surrogate_record launch");
  return SEP_OK;
}

sep_status sep_surrogate_stats(sep_ctx* ctx, uint64_t* accepted, uint64_t* fell_back, int32_t reset,
                               sep_stream stream) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
  if (!ctx) return SEP_ERR_ARG;
  SEP_CUDA(ctx, cudaSetDevice(ctx->device));
  unsigned long long v[2] = {0, 0};
  cudaStream_t s = (cudaStream_t)stream;
  SEP_CUDA(ctx, cudaMemcpyAsync(v, ctx->d_surr, sizeof v, cudaMemcpyDeviceToHost, s));
  if (reset) SEP_CUDA(ctx, cudaMemsetAsync(ctx->d_surr, 0, sizeof v, s));
  SEP_CUDA(ctx, cudaStreamSynchronize(s));
  if (accepted) *accepted = v[0];
  if (fell_back) *fell_back = v[1];
  return SEP_OK;
}

sep_status sep_clip_stats(sep_ctx* ctx, int32_t enable, uint64_t* counts, int32_t reset, sep_stream stream) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
  if (!ctx) return SEP_ERR_ARG;
  if (enable < -1 || enable > 1) return fail(ctx, SEP_ERR_ARG, "enable must be -1, 0 or 1");
  SEP_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (counts || reset) {
    unsigned long long v[SEP_CLIP_STATS] = {};
    if (counts) SEP_CUDA(ctx, cudaMemcpyAsync(v, ctx->d_clip_stats, sizeof v, cudaMemcpyDeviceToHost, s));
    if (reset) SEP_CUDA(ctx, cudaMemsetAsync(ctx->d_clip_stats, 0, sizeof v, s));
    SEP_CUDA(ctx, cudaStreamSynchronize(s));
    if (counts)
      for (int i = 0; i < SEP_CLIP_STATS; ++i) counts[i] = v[i];
  }
  if (enable >= 0) ctx->clip_stats_on = enable != 0;
  return SEP_OK;
}

sep_status sep_csr_attach_model(sep_csr* csr, const sep_model* model) {
  if (!csr) return SEP_ERR_ARG;
  if (model && model->ctx != csr->ctx) return fail(csr->ctx, SEP_ERR_STATE, "model belongs to another context");
  csr->model = model;
  return SEP_OK;
}

sep_status sep_sparsify(sep_ctx* ctx, const sep_csr* csr, const sep_calib* calib, const void* frames_dev,
                        int32_t dtype, int32_t n_frames, const sep_params* params, const float* mean_dev,
                        const float* sigma_dev, int32_t* idx_dev, float* val_dev, int64_t capacity,
                        int32_t* n_kept_dev, sep_stream stream) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
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
  cudaError_t e = cudaSuccess;
  if (params->interpolate) {
    set_interp(p, csr, params);
    e = sep::launch_mark_interp(p, n_frames, csr->h.nbins, mean_dev, sigma_dev, params->k_pick, ctx->d_bitmap, words,
                                s);
  } else {
    e = sep::launch_thresholds(mean_dev, sigma_dev, params->k_pick, (int64_t)n_frames * csr->h.nbins, ctx->d_thr, s);
    if (e == cudaSuccess) e = sep::launch_mark(p, n_frames, csr->h.nbins, ctx->d_thr, ctx->d_bitmap, words, s);
  }
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
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
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
  set_interp(p, csr, params);
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

sep_status sep_densify(sep_ctx* ctx, const sep_csr* csr, int32_t n_frames, const float* mean_dev,
                       const float* sigma_dev, const int32_t* idx_dev, const float* val_dev,
                       int64_t kept_capacity, const int32_t* n_kept_dev, const float* noise_dev, float fill,
                       int32_t interpolate, float* out_dev, sep_stream stream) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
  if (!ctx) return SEP_ERR_ARG;
  if (!csr) return fail(ctx, SEP_ERR_ARG, "NULL matrix");
  if (csr->ctx != ctx) return fail(ctx, SEP_ERR_STATE, "matrix belongs to another context");
  if (n_frames < 0 || kept_capacity < 0) return fail(ctx, SEP_ERR_ARG, "negative size");
  if (n_frames > SEP_MAX_FRAMES) return fail(ctx, SEP_ERR_ARG, "n_frames above SEP_MAX_FRAMES");
  if (n_frames == 0) return SEP_OK;
  if (!mean_dev || !out_dev || (noise_dev && !sigma_dev) ||
      (kept_capacity > 0 && (!idx_dev || !val_dev || !n_kept_dev)))
    return fail(ctx, SEP_ERR_ARG, "NULL argument");
  SEP_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaError_t e = sep::launch_densify(csr->d_bop, csr->npix, csr->h.nbins, n_frames, mean_dev, sigma_dev, idx_dev,
                                      val_dev, kept_capacity, n_kept_dev, noise_dev, fill,
                                      interpolate ? csr->d_interp_a : nullptr,
                                      interpolate ? csr->d_interp_t : nullptr, out_dev, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "densify launch");
  return SEP_OK;
}

sep_status sep_veto(sep_ctx* ctx, int32_t n_frames, const int32_t* n_peaks_dev, int32_t min_peaks,
                    int32_t* frame_list_dev, int32_t* n_pass_dev, sep_stream stream) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
  if (!ctx) return SEP_ERR_ARG;
  if (n_frames < 0 || n_frames > (1 << 24) || min_peaks < 0) return fail(ctx, SEP_ERR_ARG, "n_frames or min_peaks");
  if (!n_pass_dev || (n_frames > 0 && (!n_peaks_dev || !frame_list_dev))) return fail(ctx, SEP_ERR_ARG, "NULL argument");
  SEP_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaError_t e = sep::launch_veto(n_frames, n_peaks_dev, min_peaks, frame_list_dev, n_pass_dev, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "veto launch");
  return SEP_OK;
}

sep_status sep_compact_frames(sep_ctx* ctx, int32_t n_frames, const int32_t* frame_list_dev,
                              const int32_t* n_pass_dev, int64_t row_bytes, const void* src_dev, void* dst_dev,
                              sep_stream stream) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
  if (!ctx) return SEP_ERR_ARG;
  if (n_frames < 0 || n_frames > SEP_MAX_FRAMES || row_bytes < 0 || row_bytes % 4)
    return fail(ctx, SEP_ERR_ARG, "n_frames or row_bytes");
  if (n_frames == 0 || row_bytes == 0) return SEP_OK;
  if (!frame_list_dev || !n_pass_dev || !src_dev || !dst_dev) return fail(ctx, SEP_ERR_ARG, "NULL argument");
  const char *s0 = static_cast<const char*>(src_dev), *d0 = static_cast<const char*>(dst_dev);
  const int64_t span = row_bytes * n_frames;
  if (s0 < d0 + span && d0 < s0 + span) return fail(ctx, SEP_ERR_ARG, "src and dst overlap");
  SEP_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaError_t e = sep::launch_compact_rows(n_frames, frame_list_dev, n_pass_dev, row_bytes, src_dev, dst_dev,
                                           (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "compact launch");
  return SEP_OK;
}

sep_status sep_process_batch(sep_ctx* ctx, const sep_csr* csr, const sep_calib* calib, const void* frames_dev,
                             int32_t dtype, int32_t n_frames, const sep_params* params, float* mean_dev,
                             float* sigma_dev, int32_t* count_dev, int32_t* idx_dev, float* val_dev,
                             int64_t kept_capacity, int32_t* n_kept_dev, sep_peak* peaks_dev, int64_t peak_capacity,
                             int32_t* n_peaks_dev, int32_t use_graph, sep_stream stream) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
  sep_status st = check_common(ctx, csr, calib, frames_dev, dtype, n_frames, params);
  if (st != SEP_OK) return st;
  if (kept_capacity < 0 || peak_capacity < 0) return fail(ctx, SEP_ERR_ARG, "capacity < 0");
  if (n_frames > 0 && (!mean_dev || !sigma_dev || !count_dev || !n_kept_dev || !n_peaks_dev ||
                       (kept_capacity > 0 && (!idx_dev || !val_dev)) || (peak_capacity > 0 && !peaks_dev)))
    return fail(ctx, SEP_ERR_ARG, "NULL argument");
  if ((st = check_bin_fits(ctx, csr)) != SEP_OK) return st;
  if (n_frames == 0) return SEP_OK;
  const int64_t words = bitmap_words(csr->npix);
  if ((st = ensure_scratch(ctx, words * n_frames, (int64_t)n_frames * csr->h.nbins,
                           sep::consumer_scratch_words(n_frames, words, kept_capacity))) != SEP_OK)
    return st;
  if ((st = ensure_stage(ctx, stage_stride(csr) * n_frames)) != SEP_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;

  auto enqueue = [&](int mode) -> cudaError_t {
    // the clip kernel marks the kept pixels as each bin's threshold is known;
    // thresholds interpolated between bins wait for every bin of the frame
    sep::ClipArgs a = clip_args(ctx, csr, ctx->d_stage, n_frames, params, mean_dev, sigma_dev, count_dev, nullptr,
                                nullptr, nullptr);
    a.bitmap = params->interpolate ? nullptr : ctx->d_bitmap;
    a.words = words;
    sep::PixArgs p = pix_args(csr, calib, frames_dev, dtype);
    p.stage = ctx->d_stage;
    p.pos_of = csr->d_pos_of;
    p.npos = stage_stride(csr);
    set_interp(p, csr, params);
    cudaError_t e = cudaMemsetAsync(ctx->d_bitmap, 0, (size_t)(words * n_frames) * 4, s);
    if (e == cudaSuccess) e = enqueue_stage(ctx, csr, calib, frames_dev, nullptr, dtype, n_frames, ctx->d_stage, s);
    if (e == cudaSuccess)
      e = enqueue_clip(ctx, csr, a, params->precision, mode, s);
    if (e == cudaSuccess && params->interpolate)
      e = sep::launch_mark_interp(p, n_frames, csr->h.nbins, mean_dev, sigma_dev, params->k_pick, ctx->d_bitmap,
                                  words, s);
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
                               (uint64_t)(uintptr_t)s, csr->plan_version, (uint64_t)(uintptr_t)csr->model,
                               (uint64_t)(uintptr_t)ctx->d_stage, (uint64_t)(uintptr_t)ctx->d_thr,
                               (uint64_t)ctx->clip_stats_on};
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
    sep::ClipArgs a0 = clip_args(ctx, csr, ctx->d_stage, n_frames, params, mean_dev, sigma_dev, count_dev, nullptr,
                                 nullptr, ctx->d_thr);
    cudaError_t e = enqueue_clip(ctx, csr, a0, params->precision, 1, s);
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


sep_status sep_process_host(sep_ctx* ctx, const sep_csr* csr, const sep_calib* calib, const void* frames_host,
                            int32_t dtype, int32_t n_frames, const sep_params* params, float* mean_host,
                            float* sigma_host, int32_t* count_host, int32_t* idx_host, float* val_host,
                            int64_t kept_capacity, int32_t* n_kept_host, sep_peak* peaks_host,
                            int64_t peak_capacity, int32_t* n_peaks_host, int32_t chunk_frames, sep_stream stream) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
  sep_status st = check_common(ctx, csr, calib, frames_host, dtype, n_frames, params, true);
  if (st != SEP_OK) return st;
  if (kept_capacity < 0 || peak_capacity < 0) return fail(ctx, SEP_ERR_ARG, "capacity < 0");
  if (chunk_frames < 0 || chunk_frames > SEP_MAX_FRAMES)
    return fail(ctx, SEP_ERR_ARG, "chunk_frames outside [0, SEP_MAX_FRAMES]");
  if (n_frames > 0 && (!mean_host || !sigma_host || !count_host || !n_kept_host || !n_peaks_host ||
                       (kept_capacity > 0 && (!idx_host || !val_host)) || (peak_capacity > 0 && !peaks_host)))
    return fail(ctx, SEP_ERR_ARG, "NULL argument");
  if (n_frames == 0) return SEP_OK;
  const int32_t C = std::min(n_frames, chunk_frames > 0 ? chunk_frames : 64);
  const int64_t B = csr->h.nbins, N = csr->npix;
  const size_t px = dtype == SEP_DTYPE_U16_JF ? 2 : 4;
  // one slot: frames, mean, sigma, count, idx, val, n_kept, peaks, n_peaks (256-byte aligned pieces)
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t sz[9] = {al(px * N * C), al(4 * B * C), al(4 * B * C), al(4 * B * C), al(4 * kept_capacity * C),
                        al(4 * kept_capacity * C), al(4 * (size_t)C), al(sizeof(sep_peak) * peak_capacity * C),
                        al(4 * (size_t)C)};
  size_t slot = 0, off[9];
  for (int i = 0; i < 9; ++i) {
    off[i] = slot;
    slot += sz[i];
  }
  constexpr int NSL = sep_ctx::kSlots;
  if (NSL * slot > ctx->pipe_len) {
    if (ctx->d_pipe) cudaFree(ctx->d_pipe);
    ctx->d_pipe = nullptr;
    ctx->pipe_len = 0;
    if (cudaMalloc((void**)&ctx->d_pipe, NSL * slot) != cudaSuccess)
      return fail(ctx, SEP_ERR_OOM, "pipeline buffer allocation failed");
    ctx->pipe_len = NSL * slot;
  }
  constexpr int NS = sep_ctx::kCopyStreams;
  if (!ctx->s_out) {
    for (int j = 0; j < NS; ++j) SEP_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->s_in[j], cudaStreamNonBlocking));
    SEP_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->s_out, cudaStreamNonBlocking));
    for (int i = 0; i < sep_ctx::kSlots; ++i) {
      for (int j = 0; j < NS; ++j) SEP_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_in[i][j], cudaEventDisableTiming));
      SEP_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_done[i], cudaEventDisableTiming));
      SEP_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_out[i], cudaEventDisableTiming));
    }
    SEP_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_start, cudaEventDisableTiming));
  }
  cudaStream_t s = (cudaStream_t)stream;
  // Copy-in does not wait for earlier work on the caller's stream (the host
  // input is ready when the call is made), only for its slot to be free:
  // consecutive calls overlap their copies with each other's compute.
  const int32_t nch = (n_frames + C - 1) / C;
  for (int32_t c = 0; c < nch; ++c) {
    const int32_t f0 = c * C, m = std::min(C, n_frames - f0), k = c % NSL;
    unsigned char* base = ctx->d_pipe + (size_t)k * slot;
    void* d_fr = base + off[0];
    float* d_mean = reinterpret_cast<float*>(base + off[1]);
    float* d_sigma = reinterpret_cast<float*>(base + off[2]);
    int32_t* d_count = reinterpret_cast<int32_t*>(base + off[3]);
    int32_t* d_idx = reinterpret_cast<int32_t*>(base + off[4]);
    float* d_val = reinterpret_cast<float*>(base + off[5]);
    int32_t* d_nk = reinterpret_cast<int32_t*>(base + off[6]);
    sep_peak* d_pk = reinterpret_cast<sep_peak*>(base + off[7]);
    int32_t* d_np = reinterpret_cast<int32_t*>(base + off[8]);
    // slot k is free once its previous chunk's results have left it; the chunk's
    // frames are copied in NS pieces on as many streams (copy engines)
    const size_t bytes = px * N * m, piece = ((bytes + NS - 1) / NS + 255) & ~(size_t)255;
    for (int j = 0; j < NS; ++j) {
      const size_t o = (size_t)j * piece;
      // (an event never recorded yet is no dependency)
      SEP_CUDA(ctx, cudaStreamWaitEvent(ctx->s_in[j], ctx->ev_out[k], 0));
      if (o < bytes)
        SEP_CUDA(ctx, cudaMemcpyAsync(static_cast<unsigned char*>(d_fr) + o,
                                      static_cast<const unsigned char*>(frames_host) + px * N * f0 + o,
                                      std::min(piece, bytes - o), cudaMemcpyHostToDevice, ctx->s_in[j]));
      SEP_CUDA(ctx, cudaEventRecord(ctx->ev_in[k][j], ctx->s_in[j]));
      SEP_CUDA(ctx, cudaStreamWaitEvent(s, ctx->ev_in[k][j], 0));
    }
    st = sep_process_batch(ctx, csr, calib, d_fr, dtype, m, params, d_mean, d_sigma, d_count, d_idx, d_val,
                           kept_capacity, d_nk, d_pk, peak_capacity, d_np, 1, stream);
    if (st != SEP_OK) return st;
    SEP_CUDA(ctx, cudaEventRecord(ctx->ev_done[k], s));
    SEP_CUDA(ctx, cudaStreamWaitEvent(ctx->s_out, ctx->ev_done[k], 0));
    auto out = [&](void* h, const void* d, size_t bytes) -> cudaError_t {
      return bytes ? cudaMemcpyAsync(h, d, bytes, cudaMemcpyDeviceToHost, ctx->s_out) : cudaSuccess;
    };
    cudaError_t e = out(mean_host + B * f0, d_mean, 4 * B * m);
    if (e == cudaSuccess) e = out(sigma_host + B * f0, d_sigma, 4 * B * m);
    if (e == cudaSuccess) e = out(count_host + B * f0, d_count, 4 * B * m);
    if (e == cudaSuccess && kept_capacity > 0) e = out(idx_host + kept_capacity * f0, d_idx, 4 * kept_capacity * m);
    if (e == cudaSuccess && kept_capacity > 0) e = out(val_host + kept_capacity * f0, d_val, 4 * kept_capacity * m);
    if (e == cudaSuccess) e = out(n_kept_host + f0, d_nk, 4 * (size_t)m);
    if (e == cudaSuccess && peak_capacity > 0)
      e = out(peaks_host + peak_capacity * f0, d_pk, sizeof(sep_peak) * peak_capacity * m);
    if (e == cudaSuccess) e = out(n_peaks_host + f0, d_np, 4 * (size_t)m);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_out[k], ctx->s_out);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "process_host copy out");
  }
  // the caller's stream waits for the last copies
  SEP_CUDA(ctx, cudaStreamWaitEvent(s, ctx->ev_out[(nch - 1) % NSL], 0));
  return SEP_OK;
}

sep_status sep_csr_set_plan(sep_ctx* ctx, sep_csr* csr, int32_t n_classes, const int32_t* thresholds,
                            const int32_t* tpb) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
  if (!ctx) return SEP_ERR_ARG;
  if (!csr || csr->ctx != ctx) return fail(ctx, SEP_ERR_STATE, "csr missing or from another context");
  if (!tpb || (n_classes > 1 && !thresholds)) return fail(ctx, SEP_ERR_ARG, "NULL argument");
  SEP_CUDA(ctx, cudaSetDevice(ctx->device));
  return make_plan(ctx, csr, n_classes, thresholds, tpb);
}

sep_status sep_csr_get_plan(const sep_csr* csr, int32_t* n_classes, int32_t* thresholds, int32_t* tpb) {
  if (!csr || !n_classes) return SEP_ERR_ARG;
  if (csr->plan.empty()) {
    *n_classes = 1;
    if (tpb) tpb[0] = 256;
    return SEP_OK;
  }
  *n_classes = (int32_t)csr->plan.size();
  for (size_t i = 0; i < csr->plan.size(); ++i) {
    if (tpb) tpb[i] = csr->plan[i].tpb;
    if (thresholds && i + 1 < csr->plan.size()) thresholds[i] = csr->plan[i].threshold;
  }
  return SEP_OK;
}

sep_status sep_autotune(sep_ctx* ctx, sep_csr* csr, const sep_calib* calib, const void* frames_dev, int32_t dtype,
                        int32_t n_frames, const sep_params* params, const char* cache_path, float* best_ms,
                        sep_stream stream) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
  sep_status st = check_common(ctx, csr, calib, frames_dev, dtype, n_frames, params);
  if (st != SEP_OK) return st;
  if (n_frames < 1) return fail(ctx, SEP_ERR_ARG, "autotuning needs at least one sample frame");
  if ((st = check_bin_fits(ctx, csr)) != SEP_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaDeviceProp prop;
  SEP_CUDA(ctx, cudaGetDeviceProperties(&prop, ctx->device));
  char key[512];
  snprintf(key, sizeof key, "warp-tail|%dx%d|bins=%d|split=%d|nnz=%lld|max=%d|norm=%d|dtype=%d|prec=%d|%s", csr->h.rows,
           csr->h.cols, csr->h.nbins, csr->h.split, (long long)csr->nnz, csr->h.max_row, (int)csr->has_norm, dtype,
           params->precision, prop.name);
  // a plan already tuned for this detector and device
  if (cache_path) {
    FILE* fp = fopen(cache_path, "r");
    if (fp) {
      char line[1024];
      while (fgets(line, sizeof line, fp)) {
        char* tab = strchr(line, '\t');
        if (!tab) continue;
        *tab = 0;
        if (strcmp(line, key) != 0) continue;
        int nc = 0, t[4] = {0, 0, 0, 0}, b[4] = {256, 256, 256, 256};
        float ms = 0;
        if (sscanf(tab + 1, "%d %d %d %d %d %d %d %d %f", &nc, &t[0], &t[1], &t[2], &b[0], &b[1], &b[2], &b[3],
                   &ms) >= 8 &&
            nc >= 1 && nc <= 4) {
          fclose(fp);
          if (best_ms) *best_ms = ms;
          return make_plan(ctx, csr, nc, t, b);
        }
      }
      fclose(fp);
    }
  }
  // timed search over size-class splits and block sizes
  // (the clip kernel gives each warp its own frames: the block size sets how
  // many frames of one bin a CTA holds at once; size classes let short rows
  // take little shared memory, so more of them fit an SM)
  struct Cand { int nc; int t[3]; int b[4]; };
  std::vector<Cand> cands;
  for (int b0 : {32, 64, 128}) cands.push_back({1, {0, 0, 0}, {b0, 0, 0, 0}});
  for (int thr : {2048, 4096, 6144, 8192})
    for (const auto& bb : {std::pair<int, int>{32, 32}, {64, 32}, {128, 32}, {64, 64}})
      cands.push_back({2, {thr, 0, 0}, {bb.first, bb.second, 0, 0}});
  const int t3[3][2] = {{4096, 8192}, {6144, 10240}, {2048, 6144}};
  const int b3[3][3] = {{32, 32, 32}, {64, 32, 32}, {128, 64, 32}};
  for (const auto& tt : t3)
    for (const auto& bb : b3) cands.push_back({3, {tt[0], tt[1], 0}, {bb[0], bb[1], bb[2], 0}});
  float* d_out = nullptr;
  const size_t per = (size_t)n_frames * csr->h.nbins;
  SEP_CUDA(ctx, cudaMalloc((void**)&d_out, per * 12));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int best_i = -1;
  if ((st = ensure_stage(ctx, stage_stride(csr) * n_frames)) != SEP_OK) {
    cudaFree(d_out);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
  }
  // the staged sample is the same for every candidate schedule
  {
    cudaError_t e = enqueue_stage(ctx, csr, calib, frames_dev, nullptr, dtype, n_frames, ctx->d_stage, s);
    if (e != cudaSuccess) {
      cudaFree(d_out);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return cuda_fail(ctx, e, "autotune staging");
    }
  }
  sep::ClipArgs base = clip_args(ctx, csr, ctx->d_stage, n_frames, params, d_out, d_out + per,
                                 reinterpret_cast<int32_t*>(d_out + 2 * per), nullptr, nullptr, nullptr);
  // the trials mark kept pixels into the context's bitmap, as a batch does
  // (its contents are scratch here)
  const int64_t words = bitmap_words(csr->npix);
  if (!params->interpolate && ensure_scratch(ctx, words * n_frames, 0) == SEP_OK) {
    base.bitmap = ctx->d_bitmap;
    base.words = words;
  }
  for (size_t i = 0; i < cands.size(); ++i) {
    const Cand& c = cands[i];
    if ((st = make_plan(ctx, csr, c.nc, c.t, c.b)) != SEP_OK) break;
    cudaError_t e = enqueue_clip(ctx, csr, base, params->precision, 0, s);   // warm-up
    // the fastest of three timed runs
    float ms = 1e30f;
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
      e = cudaEventRecord(e0, s);
      if (e == cudaSuccess) e = enqueue_clip(ctx, csr, base, params->precision, 2, s);
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float t = 0;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
      if (e == cudaSuccess) ms = std::min(ms, t);
    }
    if (e != cudaSuccess) {
      st = cuda_fail(ctx, e, "autotune trial");
      break;
    }
    if (ms < best) {
      best = ms;
      best_i = (int)i;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d_out);
  if (st != SEP_OK) return st;
  const Cand& w = cands[best_i];
  if ((st = make_plan(ctx, csr, w.nc, w.t, w.b)) != SEP_OK) return st;
  if (best_ms) *best_ms = best;
  if (cache_path) {
    FILE* fp = fopen(cache_path, "a");
    if (fp) {
      fprintf(fp, "%s\t%d %d %d %d %d %d %d %d %.9g\n", key, w.nc, w.t[0], w.t[1], w.t[2], w.b[0], w.b[1], w.b[2],
              w.b[3], best);
      fclose(fp);
    }
  }
  return SEP_OK;
}


sep_status sep_process_mixed(sep_ctx* ctx, int32_t n_det, sep_csr* const* csrs, const sep_calib* const* calibs,
                             const sep_frame_desc* frames, int32_t n_frames, const sep_params* params,
                             float* mean_dev, float* sigma_dev, int32_t* count_dev, int64_t* row_off,
                             int32_t* idx_dev, float* val_dev, int64_t kept_capacity, int32_t* n_kept_dev,
                             sep_peak* peaks_dev, int64_t peak_capacity, int32_t* n_peaks_dev, int32_t use_graph,
                             sep_stream stream) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
  if (!ctx) return SEP_ERR_ARG;
  if (n_det < 1 || n_det > 4 || !csrs) return fail(ctx, SEP_ERR_ARG, "1 to 4 detectors");
  if (n_frames < 0 || n_frames > SEP_MAX_FRAMES || (n_frames > 0 && !frames))
    return fail(ctx, SEP_ERR_ARG, "bad frame list");
  if (kept_capacity < 0 || peak_capacity < 0) return fail(ctx, SEP_ERR_ARG, "capacity < 0");
  sep_status st = check_params(ctx, params);
  if (st != SEP_OK) return st;
  if (n_frames > 0 && (!mean_dev || !sigma_dev || !count_dev || !n_kept_dev || !n_peaks_dev ||
                       (kept_capacity > 0 && (!idx_dev || !val_dev)) || (peak_capacity > 0 && !peaks_dev)))
    return fail(ctx, SEP_ERR_ARG, "NULL argument");
  for (int d = 0; d < n_det; ++d) {
    if (!csrs[d] || csrs[d]->ctx != ctx) return fail(ctx, SEP_ERR_STATE, "csr missing or from another context");
    if ((st = check_bin_fits(ctx, csrs[d])) != SEP_OK) return st;
    if (params->error_model != SEP_ERROR_AZIMUTHAL && csrs[d]->has_norm)
      return fail(ctx, SEP_ERR_ARG, "the Poisson and hybrid models take frames without a norm");
    if (params->surrogate > 0 && (!csrs[d]->model || csrs[d]->model->ctx != ctx))
      return fail(ctx, SEP_ERR_STATE, "surrogate requested but a detector has no model of this context");
  }
  std::vector<std::vector<int32_t>> members(n_det);
  std::vector<int64_t> rows((size_t)n_frames + 1, 0);
  for (int32_t g = 0; g < n_frames; ++g) {
    const sep_frame_desc& fd = frames[g];
    if (fd.det < 0 || fd.det >= n_det || !fd.frame_dev) return fail(ctx, SEP_ERR_ARG, "bad frame descriptor");
    if (fd.dtype == SEP_DTYPE_U16_JF) {
      const sep_calib* c = calibs ? calibs[fd.det] : nullptr;
      if (!c || c->ctx != ctx || c->npix != csrs[fd.det]->npix)
        return fail(ctx, SEP_ERR_ARG, "raw frames need their detector's calibration");
    } else if (fd.dtype != SEP_DTYPE_F32) {
      return fail(ctx, SEP_ERR_ARG, "unknown dtype");
    }
    if (g > 0 && fd.det == frames[g - 1].det && fd.dtype != frames[g - 1].dtype) {
      // frames of one detector share a dtype (one kernel variant per detector)
    }
    members[fd.det].push_back(g);
    rows[g + 1] = rows[g] + csrs[fd.det]->h.nbins;
  }
  for (int d = 0; d < n_det; ++d)
    for (int32_t g : members[d])
      if (frames[g].dtype != frames[members[d][0]].dtype)
        return fail(ctx, SEP_ERR_ARG, "frames of one detector must share a dtype");
  if (row_off) memcpy(row_off, rows.data(), rows.size() * sizeof(int64_t));
  if (n_frames == 0) return SEP_OK;
  SEP_CUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;

  // descriptor table (device): per detector fptr[m], orow[m], fidx[m]
  std::vector<int64_t> desc;
  std::vector<size_t> off_fptr(n_det), off_orow(n_det), off_fidx(n_det);
  int64_t bm_total = 0, aux_total = 0, stage_total = 0, thr_total = rows[n_frames];
  std::vector<int64_t> bm_off(n_det), aux_off(n_det), words(n_det), soff(n_det);
  for (int d = 0; d < n_det; ++d) {
    const int64_t m = (int64_t)members[d].size();
    off_fptr[d] = desc.size();
    for (int32_t g : members[d]) desc.push_back((int64_t)(uintptr_t)frames[g].frame_dev);
    off_orow[d] = desc.size();
    for (int32_t g : members[d]) desc.push_back(rows[g]);
    off_fidx[d] = desc.size();
    for (size_t i = 0; i < members[d].size(); i += 2)
      desc.push_back((int64_t)(uint32_t)members[d][i] |
                     (i + 1 < members[d].size() ? (int64_t)members[d][i + 1] << 32 : 0));
    words[d] = bitmap_words(csrs[d]->npix);
    bm_off[d] = bm_total;
    bm_total += words[d] * m;
    aux_off[d] = aux_total;
    aux_total += sep::consumer_scratch_words((int32_t)m, words[d], kept_capacity);
    soff[d] = stage_total;
    stage_total += m * stage_stride(csrs[d]);
  }
  if ((st = ensure_scratch(ctx, bm_total, thr_total, aux_total)) != SEP_OK) return st;
  if ((st = ensure_stage(ctx, stage_total)) != SEP_OK) return st;
  if (desc.size() > ctx->desc_len) {
    if (ctx->d_desc) cudaFree(ctx->d_desc);
    if (ctx->h_desc) cudaFreeHost(ctx->h_desc);
    ctx->d_desc = nullptr;
    ctx->h_desc = nullptr;
    ctx->desc_len = 0;
    if (cudaMalloc((void**)&ctx->d_desc, desc.size() * 8) != cudaSuccess ||
        cudaMallocHost((void**)&ctx->h_desc, desc.size() * 8) != cudaSuccess)
      return fail(ctx, SEP_ERR_OOM, "descriptor table allocation failed");
    ctx->desc_len = desc.size();
  }
  // the previous call's copy may still be reading the staging buffer
  SEP_CUDA(ctx, cudaStreamSynchronize(s));
  memcpy(ctx->h_desc, desc.data(), desc.size() * 8);
  SEP_CUDA(ctx, cudaMemcpyAsync(ctx->d_desc, ctx->h_desc, desc.size() * 8, cudaMemcpyHostToDevice, s));

  auto enqueue = [&](int mode) -> cudaError_t {
    cudaError_t e = cudaSuccess;
    if (mode != 1) e = cudaEventRecord(ctx->ev_fork, s);
    for (int d = 0; d < n_det && e == cudaSuccess; ++d) {
      const int32_t m = (int32_t)members[d].size();
      if (m == 0) continue;
      const sep_csr* csr = csrs[d];
      const int32_t dtype = frames[members[d][0]].dtype;
      const sep_calib* calib = calibs ? calibs[d] : nullptr;
      cudaStream_t sd = d == 0 ? s : ctx->aux[d];
      if (d > 0 && mode != 1) e = cudaStreamWaitEvent(sd, ctx->ev_fork, 0);
      uint32_t* bm = ctx->d_bitmap + bm_off[d];
      int32_t* aux = ctx->d_aux + aux_off[d];
      const uint64_t* fptr = reinterpret_cast<const uint64_t*>(ctx->d_desc + off_fptr[d]);
      const int64_t* orow = ctx->d_desc + off_orow[d];
      const int32_t* fidx = reinterpret_cast<const int32_t*>(ctx->d_desc + off_fidx[d]);
      float* stage = ctx->d_stage + soff[d];
      sep::ClipArgs ca = clip_args(ctx, csr, stage, m, params, mean_dev, sigma_dev, count_dev, nullptr, nullptr,
                                   nullptr);
      ca.orow = orow;
      ca.bitmap = params->interpolate ? nullptr : bm;   // kept pixels are marked by the clip kernel
      ca.words = words[d];
      if (mode == 1) {
        e = enqueue_clip(ctx, csr, ca, params->precision, 1, sd, false);
        continue;
      }
      sep::PixArgs pa = pix_args(csr, calib, nullptr, dtype);
      pa.fptr = fptr;
      pa.fidx = fidx;
      pa.orow = orow;
      pa.stage = stage;
      pa.pos_of = csr->d_pos_of;
      pa.npos = stage_stride(csr);
      set_interp(pa, csr, params);
      if (e == cudaSuccess) e = cudaMemsetAsync(bm, 0, (size_t)(words[d] * m) * 4, sd);
      if (e == cudaSuccess) e = enqueue_stage(ctx, csr, calib, nullptr, fptr, dtype, m, stage, sd);
      if (e == cudaSuccess) e = enqueue_clip(ctx, csr, ca, params->precision, mode, sd, false);
      if (e == cudaSuccess && params->interpolate)
        e = sep::launch_mark_interp(pa, m, csr->h.nbins, mean_dev, sigma_dev, params->k_pick, bm, words[d], sd);
      if (e == cudaSuccess)
        e = sep::launch_compact(pa, m, bm, words[d], idx_dev, val_dev, kept_capacity, n_kept_dev, aux, ctx->d_status,
                                sd);
      if (e == cudaSuccess)
        e = sep::launch_peaks(pa, m, csr->h.nbins, mean_dev, sigma_dev, bm, words[d], idx_dev, n_kept_dev,
                              kept_capacity, params->patch, params->min_count, peaks_dev, peak_capacity, n_peaks_dev,
                              aux, ctx->d_status, sd);
      if (e == cudaSuccess && d > 0) e = cudaEventRecord(ctx->ev_join[d], sd);
    }
    for (int d = 1; d < n_det && e == cudaSuccess && mode != 1; ++d)
      if (!members[d].empty()) e = cudaStreamWaitEvent(s, ctx->ev_join[d], 0);
    return e;
  };

  if (!use_graph || s == nullptr) {
    cudaError_t e = enqueue(0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "process_mixed launch");
    return SEP_OK;
  }
  std::vector<uint64_t> key = {0x6d69786564ull, (uint64_t)n_frames, (uint64_t)(uintptr_t)mean_dev,
                               (uint64_t)(uintptr_t)sigma_dev, (uint64_t)(uintptr_t)count_dev,
                               (uint64_t)(uintptr_t)idx_dev, (uint64_t)(uintptr_t)val_dev, (uint64_t)kept_capacity,
                               (uint64_t)(uintptr_t)n_kept_dev, (uint64_t)(uintptr_t)peaks_dev, (uint64_t)peak_capacity,
                               (uint64_t)(uintptr_t)n_peaks_dev, (uint64_t)(uintptr_t)ctx->d_bitmap,
                               (uint64_t)(uintptr_t)ctx->d_aux, (uint64_t)(uintptr_t)ctx->d_desc,
                               (uint64_t)(uintptr_t)s, (uint64_t)(uintptr_t)ctx->d_stage,
                               (uint64_t)(uintptr_t)ctx->d_thr, (uint64_t)ctx->clip_stats_on};
  for (int d = 0; d < n_det; ++d) {
    key.push_back((uint64_t)(uintptr_t)csrs[d]);
    key.push_back(csrs[d]->plan_version);
    key.push_back((uint64_t)(uintptr_t)(calibs ? calibs[d] : nullptr));
  }
  for (int32_t g = 0; g < n_frames; ++g) key.push_back(((uint64_t)frames[g].det << 8) | (uint64_t)frames[g].dtype);
  for (int64_t v : desc) key.push_back((uint64_t)v);
  {
    uint32_t pw[sizeof(sep_params) / 4];
    memcpy(pw, params, sizeof(sep_params));
    for (uint32_t w : pw) key.push_back(w);
  }
  auto it = ctx->graphs.find(key);
  if (it == ctx->graphs.end()) {
    if (ctx->graphs.size() >= 16) {
      auto lru = ctx->graphs.begin();
      for (auto j = ctx->graphs.begin(); j != ctx->graphs.end(); ++j)
        if (j->second.last_use < lru->second.last_use) lru = j;
      cudaGraphExecDestroy(lru->second.exec);
      cudaGraphDestroy(lru->second.graph);
      ctx->graphs.erase(lru);
    }
    cudaError_t e = enqueue(1);   // kernel attributes, outside the capture
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel attribute");
    sep_graph_entry g;
    SEP_CUDA(ctx, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    e = enqueue(2);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail(ctx, e != cudaSuccess ? e : e2, "process_mixed capture");
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
