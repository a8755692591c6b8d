// The surrogate network: layout and device helpers shared by its training
// kernels and by the clip kernel's fused inference.
//   x (20 features) -> W1 [64][20] + b1 -> GELU -> W2 [64][64] + b2 -> GELU
//   -> W3 [2][64] + b3 -> (mean offset, log-deviation ratio), normalised.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sep {

constexpr int kIn = 20, kH = 64, kOut = 2;
constexpr int kW1 = 0;
constexpr int kB1 = kW1 + kH * kIn;
constexpr int kW2 = kB1 + kH;
constexpr int kB2 = kW2 + kH * kH;
constexpr int kW3 = kB2 + kH;
constexpr int kB3 = kW3 + kOut * kH;
constexpr int kNParams = kB3 + kOut;   // 5634
// The clip kernel's copy of the weights keeps W1 and W2 input-major (at
// kW1 + k kH + j and kW2 + k kH + j for unit j and input k), so that the
// lanes of a warp, one hidden unit each, read consecutive weights.
__host__ __device__ __forceinline__ int mlp_transposed_index(int i) {
  if (i >= kW1 && i < kB1) {
    const int j = (i - kW1) / kIn, k = (i - kW1) % kIn;
    return kW1 + k * kH + j;
  }
  if (i >= kW2 && i < kB2) {
    const int j = (i - kW2) / kH, k = (i - kW2) % kH;
    return kW2 + k * kH + j;
  }
  return i;
}

// normalisation block stored with a model: feature mean[20], feature std[20],
// target mean[2], target std[2]
constexpr int kNNorm = 2 * kIn + 2 * kOut;

// GELU(a) = a Phi(a) = a (1 + erf(a / sqrt 2)) / 2 and its derivative.
__device__ __forceinline__ float gelu_f(float a) { return 0.5f * a * (1.0f + erff(a * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float a) {
  return 0.5f * (1.0f + erff(a * 0.70710678118654752f)) + a * expf(-0.5f * a * a) * 0.39894228040143268f;
}

// One sample through the network (weights as FP32 in any memory space).
__device__ __forceinline__ void mlp_eval(const float* W, const float (&x)[kIn], float (&y)[kOut]) {
  float h1[kH];
#pragma unroll 4
  for (int j = 0; j < kH; ++j) {
    float a = W[kB1 + j];
#pragma unroll
    for (int k = 0; k < kIn; ++k) a = fmaf(W[kW1 + j * kIn + k], x[k], a);
    h1[j] = gelu_f(a);
  }
  float y0 = W[kB3], y1 = W[kB3 + 1];
  for (int j = 0; j < kH; ++j) {
    float a = W[kB2 + j];
#pragma unroll 16
    for (int k = 0; k < kH; ++k) a = fmaf(W[kW2 + j * kH + k], h1[k], a);
    const float h = gelu_f(a);
    y0 = fmaf(W[kW3 + j], h, y0);
    y1 = fmaf(W[kW3 + kH + j], h, y1);
  }
  y[0] = y0;
  y[1] = y1;
}

size_t mlp_grad_smem();
cudaError_t launch_mlp_grad(const __nv_bfloat16* wbf, const float* x, const float* t, int64_t n, int64_t n_used,
                            int64_t start, int64_t stride, float* grad, float* loss, cudaStream_t s);
cudaError_t launch_adam(float* theta, __nv_bfloat16* wbf, __nv_bfloat16* wbt, float* m, float* v, float* grad, float lr,
                        int64_t step, cudaStream_t s);
cudaError_t launch_mlp_forward(const __nv_bfloat16* wbf, const float* x, int64_t n, float* y, cudaStream_t s);
cudaError_t launch_zero(float* p, int64_t n, cudaStream_t s);
int64_t prep_blocks(int64_t n);
cudaError_t launch_prep_stats(const float* f, const float* t, int64_t n, int32_t* cnt, double* part, cudaStream_t s);
cudaError_t launch_prep_scatter(const float* f, const float* t, int64_t n, const int64_t* base, const float* norm,
                                float* x, float* y, cudaStream_t s);

}  // namespace sep
