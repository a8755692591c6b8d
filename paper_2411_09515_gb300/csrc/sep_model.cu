// C ABI of the surrogate network: model handle, parameters, training loop,
// checkpoints.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "sep_internal.h"
#include "sep_mlp.cuh"

static_assert(sep::kNParams == SEP_MLP_PARAMS, "parameter count");
static_assert(sep::kNNorm == SEP_MLP_NORM, "normalisation block");

namespace {

sep_status mfail(sep_ctx* ctx, sep_status st, const std::string& m) {
  if (ctx) ctx->err = m;
  return st;
}

#define MCUDA(ctx, call)                                                               \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) return mfail((ctx), SEP_ERR_CUDA, std::string(#call ": ") + \
                                                                cudaGetErrorString(e_)); \
  } while (0)

uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

sep_status model_alloc(sep_ctx* ctx, sep_model* m) {
  const size_t P = sep::kNParams;
  if (cudaMalloc((void**)&m->d_params, P * 4) != cudaSuccess || cudaMalloc((void**)&m->d_wbf, P * 2) != cudaSuccess ||
      cudaMalloc((void**)&m->d_wbt, P * 2) != cudaSuccess ||
      cudaMalloc((void**)&m->d_m, P * 4) != cudaSuccess || cudaMalloc((void**)&m->d_v, P * 4) != cudaSuccess ||
      cudaMalloc((void**)&m->d_grad, P * 4) != cudaSuccess || cudaMalloc((void**)&m->d_loss, 8) != cudaSuccess ||
      cudaMalloc((void**)&m->d_norm, sep::kNNorm * 4) != cudaSuccess)
    return mfail(ctx, SEP_ERR_OOM, "model allocation failed");
  cudaMemset(m->d_m, 0, P * 4);
  cudaMemset(m->d_v, 0, P * 4);
  cudaMemset(m->d_grad, 0, P * 4);
  cudaMemset(m->d_loss, 0, 8);
  return SEP_OK;
}

sep_status upload_params(sep_model* m, const float* host) {
  std::vector<__nv_bfloat16> bf(sep::kNParams), bt(sep::kNParams);
  for (int i = 0; i < sep::kNParams; ++i) {
    bf[i] = __float2bfloat16_rn(host[i]);
    bt[sep::mlp_transposed_index(i)] = bf[i];
  }
  MCUDA(m->ctx, cudaMemcpy(m->d_params, host, sep::kNParams * 4, cudaMemcpyHostToDevice));
  MCUDA(m->ctx, cudaMemcpy(m->d_wbf, bf.data(), sep::kNParams * 2, cudaMemcpyHostToDevice));
  MCUDA(m->ctx, cudaMemcpy(m->d_wbt, bt.data(), sep::kNParams * 2, cudaMemcpyHostToDevice));
  return SEP_OK;
}

}  // namespace

extern "C" {

sep_status sep_model_create(sep_ctx* ctx, uint64_t seed, sep_model** out) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
  if (!ctx || !out) return SEP_ERR_ARG;
  *out = nullptr;
  MCUDA(ctx, cudaSetDevice(ctx->device));
  sep_model* m = new (std::nothrow) sep_model();
  if (!m) return mfail(ctx, SEP_ERR_OOM, "host allocation failed");
  m->ctx = ctx;
  sep_status st = model_alloc(ctx, m);
  if (st != SEP_OK) {
    sep_model_destroy(m);
    return st;
  }
  // He-style uniform weights (limit sqrt(6 / fan_in)), zero biases; identity normalisation
  std::vector<float> p(sep::kNParams, 0.0f);
  uint64_t s = seed;
  auto fill = [&](int off, int rows, int cols) {
    const double lim = sqrt(6.0 / cols);
    for (int i = 0; i < rows * cols; ++i)
      p[off + i] = (float)(lim * (2.0 * ((double)(splitmix(s) >> 11) * (1.0 / 9007199254740992.0)) - 1.0));
  };
  fill(sep::kW1, sep::kH, sep::kIn);
  fill(sep::kW2, sep::kH, sep::kH);
  fill(sep::kW3, sep::kOut, sep::kH);
  for (int i = 0; i < sep::kNNorm; ++i) m->norm[i] = (i >= sep::kIn && i < 2 * sep::kIn) || i >= 2 * sep::kIn + sep::kOut ? 1.0f : 0.0f;
  if ((st = upload_params(m, p.data())) != SEP_OK ||
      cudaMemcpy(m->d_norm, m->norm, sep::kNNorm * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
    sep_model_destroy(m);
    return st != SEP_OK ? st : mfail(ctx, SEP_ERR_CUDA, "cudaMemcpy");
  }
  *out = m;
  return SEP_OK;
}

void sep_model_destroy(sep_model* m) {
  if (!m) return;
  if (m->ctx) cudaSetDevice(m->ctx->device);
  cudaFree(m->d_params);
  cudaFree(m->d_wbf);
  cudaFree(m->d_wbt);
  cudaFree(m->d_m);
  cudaFree(m->d_v);
  cudaFree(m->d_grad);
  cudaFree(m->d_loss);
  cudaFree(m->d_norm);
  delete m;
}

sep_status sep_model_params(sep_model* m, float* get_host, const float* set_host) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
  if (!m) return SEP_ERR_ARG;
  MCUDA(m->ctx, cudaSetDevice(m->ctx->device));
  if (get_host) MCUDA(m->ctx, cudaMemcpy(get_host, m->d_params, sep::kNParams * 4, cudaMemcpyDeviceToHost));
  if (set_host) return upload_params(m, set_host);
  return SEP_OK;
}

sep_status sep_model_norm(sep_model* m, float* get_host, const float* set_host) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
  if (!m) return SEP_ERR_ARG;
  if (get_host) memcpy(get_host, m->norm, sizeof(m->norm));
  if (set_host) {
    for (int i = 0; i < sep::kIn; ++i)
      if (!(set_host[sep::kIn + i] > 0.0f)) return mfail(m->ctx, SEP_ERR_ARG, "feature deviations must be > 0");
    memcpy(m->norm, set_host, sizeof(m->norm));
    MCUDA(m->ctx, cudaSetDevice(m->ctx->device));
    MCUDA(m->ctx, cudaMemcpy(m->d_norm, m->norm, sizeof(m->norm), cudaMemcpyHostToDevice));
  }
  return SEP_OK;
}

sep_status sep_mlp_forward(sep_model* m, const float* x_dev, int64_t n, float* y_dev, sep_stream stream) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
  if (!m || n < 0 || (n > 0 && (!x_dev || !y_dev))) return SEP_ERR_ARG;
  MCUDA(m->ctx, cudaSetDevice(m->ctx->device));
  MCUDA(m->ctx, sep::launch_mlp_forward(m->d_wbf, x_dev, n, y_dev, (cudaStream_t)stream));
  return SEP_OK;
}

sep_status sep_mlp_loss_grad(sep_model* m, const float* x_dev, const float* t_dev, int64_t n, float* grad_dev,
                             float* loss_dev, sep_stream stream) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
  if (!m || n < 1 || !x_dev || !t_dev || !grad_dev || !loss_dev) return SEP_ERR_ARG;
  MCUDA(m->ctx, cudaSetDevice(m->ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  MCUDA(m->ctx, sep::launch_zero(grad_dev, sep::kNParams, s));
  MCUDA(m->ctx, sep::launch_zero(loss_dev, 1, s));
  MCUDA(m->ctx, sep::launch_mlp_grad(m->d_wbf, x_dev, t_dev, n, n, 0, 1, grad_dev, loss_dev, s));
  return SEP_OK;
}

sep_status sep_surrogate_train(sep_model* m, const float* x_dev, const float* t_dev, int64_t n,
                               const sep_train_cfg* cfg, float* final_loss, sep_stream stream) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
  if (!m || !cfg || n < 1 || !x_dev || !t_dev) return SEP_ERR_ARG;
  if (cfg->epochs < 1 || cfg->batch < 64 || !(cfg->lr > 0.0f)) return mfail(m->ctx, SEP_ERR_ARG, "bad training config");
  MCUDA(m->ctx, cudaSetDevice(m->ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  // a pseudo-random visiting order: row = (start + i * stride) mod n with
  // stride coprime to n, a fresh start per epoch
  uint64_t rs = cfg->seed ^ 0x5EEDull;
  int64_t stride = 1000003;
  auto gcd = [](int64_t a, int64_t b) { while (b) { int64_t t = a % b; a = b; b = t; } return a; };
  while (gcd(stride, n) != 1) stride += 2;
  const int64_t B = cfg->batch;
  const int64_t steps = (n + B - 1) / B;
  float last = 0.0f;
  for (int ep = 0; ep < cfg->epochs; ++ep) {
    const int64_t start0 = (int64_t)(splitmix(rs) % (uint64_t)n);
    MCUDA(m->ctx, sep::launch_zero(m->d_loss, 1, s));
    for (int64_t k = 0; k < steps; ++k) {
      const int64_t used = k + 1 < steps ? B : n - k * B;
      const int64_t start = (int64_t)(((__int128)start0 + (__int128)k * B % n * stride) % n);
      MCUDA(m->ctx, sep::launch_mlp_grad(m->d_wbf, x_dev, t_dev, n, used, start, stride, m->d_grad,
                                         m->d_loss, s));
      m->step += 1;
      MCUDA(m->ctx, sep::launch_adam(m->d_params, m->d_wbf, m->d_wbt, m->d_m, m->d_v, m->d_grad, cfg->lr, m->step, s));
    }
    float l = 0;
    MCUDA(m->ctx, cudaMemcpyAsync(&l, m->d_loss, 4, cudaMemcpyDeviceToHost, s));
    MCUDA(m->ctx, cudaStreamSynchronize(s));
    last = l / (float)steps;
  }
  if (final_loss) *final_loss = last;
  return SEP_OK;
}

sep_status sep_surrogate_prepare(sep_ctx* ctx, const float* feat_dev, const float* target_dev, int64_t n,
                                 float* x_dev, float* t_dev, float* norm_host, int64_t* n_valid, sep_stream stream) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
  if (!ctx || n < 0 || !norm_host || !n_valid || (n > 0 && (!feat_dev || !target_dev || !x_dev || !t_dev)))
    return mfail(ctx, SEP_ERR_ARG, "bad surrogate_prepare arguments");
  MCUDA(ctx, cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nb = sep::prep_blocks(n);
  const int C = sep::kIn + sep::kOut;
  *n_valid = 0;
  for (int i = 0; i < sep::kNNorm; ++i) norm_host[i] = i < sep::kIn || (i >= 2 * sep::kIn && i < 2 * sep::kIn + 2) ? 0.0f : 1.0f;
  if (n == 0) return SEP_OK;
  int32_t* d_cnt = nullptr;
  double* d_part = nullptr;
  int64_t* d_base = nullptr;
  float* d_norm = nullptr;
  auto cleanup = [&]() {
    cudaFree(d_cnt);
    cudaFree(d_part);
    cudaFree(d_base);
    cudaFree(d_norm);
  };
  if (cudaMalloc((void**)&d_cnt, nb * 4) != cudaSuccess || cudaMalloc((void**)&d_part, nb * 2 * C * 8) != cudaSuccess ||
      cudaMalloc((void**)&d_base, nb * 8) != cudaSuccess || cudaMalloc((void**)&d_norm, sep::kNNorm * 4) != cudaSuccess) {
    cleanup();
    return mfail(ctx, SEP_ERR_OOM, "surrogate_prepare scratch");
  }
  std::vector<int32_t> cnt(nb);
  std::vector<double> part((size_t)nb * 2 * C);
  cudaError_t e = sep::launch_prep_stats(feat_dev, target_dev, n, d_cnt, d_part, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cnt.data(), d_cnt, nb * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(part.data(), d_part, nb * 2 * C * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cleanup();
    return mfail(ctx, SEP_ERR_CUDA, std::string("surrogate_prepare: ") + cudaGetErrorString(e));
  }
  std::vector<int64_t> base(nb);
  int64_t tot = 0;
  std::vector<double> sum(C, 0.0), sq(C, 0.0);
  for (int64_t b = 0; b < nb; ++b) {
    base[b] = tot;
    tot += cnt[b];
    for (int c = 0; c < C; ++c) {
      sum[c] += part[(size_t)b * 2 * C + c];
      sq[c] += part[(size_t)b * 2 * C + C + c];
    }
  }
  if (tot > 0) {
    for (int c = 0; c < C; ++c) {
      const double mean = sum[c] / (double)tot;
      const double var = sq[c] / (double)tot - mean * mean;
      const double sd = var > 1e-12 ? sqrt(var) : 1.0;
      if (c < sep::kIn) {
        norm_host[c] = (float)mean;
        norm_host[sep::kIn + c] = (float)sd;
      } else {
        norm_host[2 * sep::kIn + (c - sep::kIn)] = (float)mean;
        norm_host[2 * sep::kIn + sep::kOut + (c - sep::kIn)] = (float)sd;
      }
    }
    e = cudaMemcpyAsync(d_base, base.data(), nb * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_norm, norm_host, sep::kNNorm * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = sep::launch_prep_scatter(feat_dev, target_dev, n, d_base, d_norm, x_dev, t_dev, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  cleanup();
  if (e != cudaSuccess) return mfail(ctx, SEP_ERR_CUDA, std::string("surrogate_prepare: ") + cudaGetErrorString(e));
  *n_valid = tot;
  return SEP_OK;
}

sep_status sep_model_save(const sep_model* m, const char* path) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
  if (!m || !path) return SEP_ERR_ARG;
  const size_t P = sep::kNParams;
  std::vector<float> buf(3 * P);
  cudaSetDevice(m->ctx->device);
  if (cudaMemcpy(buf.data(), m->d_params, P * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(buf.data() + P, m->d_m, P * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(buf.data() + 2 * P, m->d_v, P * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return SEP_ERR_CUDA;
  FILE* f = fopen(path, "wb");
  if (!f) return SEP_ERR_ARG;
  fprintf(f, "{\"format\": \"sep-surrogate-1\", \"n_in\": %d, \"n_hidden\": %d, \"n_out\": %d, \"n_params\": %d, "
             "\"n_norm\": %d, \"adam_step\": %lld, \"layout\": \"params, norm, adam m, adam v (float32 LE)\"}\n",
          sep::kIn, sep::kH, sep::kOut, sep::kNParams, sep::kNNorm, (long long)m->step);
  fwrite(buf.data(), 4, P, f);
  fwrite(m->norm, 4, sep::kNNorm, f);
  fwrite(buf.data() + P, 4, 2 * P, f);
  fclose(f);
  return SEP_OK;
}

sep_status sep_model_load(sep_ctx* ctx, const char* path, sep_model** out) {
  sep::DeviceGuard device_guard;
  sep::NvtxRange nvtx_range(__func__);
  if (!ctx || !path || !out) return SEP_ERR_ARG;
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) return mfail(ctx, SEP_ERR_ARG, std::string("cannot open ") + path);
  char line[1024];
  if (!fgets(line, sizeof line, f) || !strstr(line, "\"sep-surrogate-1\"")) {
    fclose(f);
    return mfail(ctx, SEP_ERR_ARG, "not a surrogate checkpoint");
  }
  long long step = 0;
  const char* ps = strstr(line, "\"adam_step\":");
  if (ps) sscanf(ps + 12, "%lld", &step);
  const size_t P = sep::kNParams;
  std::vector<float> prm(P), nrm(sep::kNNorm), mv(2 * P);
  const bool ok = fread(prm.data(), 4, P, f) == P && fread(nrm.data(), 4, sep::kNNorm, f) == (size_t)sep::kNNorm &&
                  fread(mv.data(), 4, 2 * P, f) == 2 * P;
  fclose(f);
  if (!ok) return mfail(ctx, SEP_ERR_ARG, "truncated checkpoint");
  sep_model* m = nullptr;
  sep_status st = sep_model_create(ctx, 0, &m);
  if (st != SEP_OK) return st;
  m->step = step;
  if ((st = sep_model_params(m, nullptr, prm.data())) != SEP_OK || (st = sep_model_norm(m, nullptr, nrm.data())) != SEP_OK) {
    sep_model_destroy(m);
    return st;
  }
  if (cudaMemcpy(m->d_m, mv.data(), P * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(m->d_v, mv.data() + P, P * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
    sep_model_destroy(m);
    return mfail(ctx, SEP_ERR_CUDA, "cudaMemcpy");
  }
  *out = m;
  return SEP_OK;
}

}  // extern "C"
