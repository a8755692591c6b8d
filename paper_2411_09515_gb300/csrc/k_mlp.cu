// The surrogate network's own kernels: forward, loss + gradient by
// backpropagation over a batch, Adam, and the per-bin inference used inside
// the clip kernel. Network: 20 -> 64 -> GELU -> 64 -> GELU -> 2, GELU exact
// (x Phi(x)); weights are read as BF16, every product and sum is FP32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sep_mlp.cuh"

namespace sep {
namespace {

constexpr int kTile = 64;        // samples per CTA in the gradient kernel
constexpr int kGradThreads = 256;

// Weights (BF16 -> FP32) into shared memory.
__device__ __forceinline__ void load_weights(const __nv_bfloat16* wbf, float* w) {
  for (int i = threadIdx.x; i < kNParams; i += blockDim.x) w[i] = __bfloat162float(wbf[i]);
}

// Gradient of the mean squared error over n samples (x [n][20], t [n][2]),
// accumulated into grad [kNParams] and loss (sum over samples / n).
// Sample s of tile b is row idx(b * kTile + s) = (start + (b*kTile+s) * stride) mod n.
__global__ void __launch_bounds__(kGradThreads) k_mlp_grad(const __nv_bfloat16* wbf, const float* x, const float* t,
                                                           int64_t n, int64_t n_used, int64_t start, int64_t stride,
                                                           float* grad, float* loss) {
  extern __shared__ float sm[];
  float* W = sm;                                  // kNParams
  float* X = W + kNParams + 2;                    // [kTile][kIn]   (+2 keeps 8-byte alignment)
  float* A1 = X + kTile * kIn;                    // [kTile][kH]
  float* H1 = A1 + kTile * kH;
  float* A2 = H1 + kTile * kH;
  float* H2 = A2 + kTile * kH;
  float* Y = H2 + kTile * kH;                     // [kTile][kOut]
  __shared__ float lsum;
  const int tid = threadIdx.x;
  load_weights(wbf, W);
  if (tid == 0) lsum = 0.0f;
  const int64_t s0 = (int64_t)blockIdx.x * kTile;
  const int ns = (int)(n_used - s0 < kTile ? n_used - s0 : kTile);
  for (int i = tid; i < kTile * kIn; i += blockDim.x) {
    const int s = i / kIn, k = i - s * kIn;
    float v = 0.0f;
    if (s < ns) {
      const int64_t r = (start + (s0 + s) * stride) % n;
      v = x[r * kIn + k];
    }
    X[i] = v;
  }
  __syncthreads();
  const float* W1 = W + kW1; const float* b1 = W + kB1;
  const float* W2 = W + kW2; const float* b2 = W + kB2;
  const float* W3 = W + kW3; const float* b3 = W + kB3;
  // forward
  for (int i = tid; i < kTile * kH; i += blockDim.x) {
    const int s = i / kH, j = i - s * kH;
    float a = b1[j];
#pragma unroll
    for (int k = 0; k < kIn; ++k) a = fmaf(W1[j * kIn + k], X[s * kIn + k], a);
    A1[i] = a;
    H1[i] = gelu_f(a);
  }
  __syncthreads();
  for (int i = tid; i < kTile * kH; i += blockDim.x) {
    const int s = i / kH, j = i - s * kH;
    float a = b2[j];
#pragma unroll 16
    for (int k = 0; k < kH; ++k) a = fmaf(W2[j * kH + k], H1[s * kH + k], a);
    A2[i] = a;
    H2[i] = gelu_f(a);
  }
  __syncthreads();
  if (tid < kTile * kOut) {
    const int s = tid / kOut, o = tid - s * kOut;
    float y = b3[o];
#pragma unroll 16
    for (int k = 0; k < kH; ++k) y = fmaf(W3[o * kH + k], H2[s * kH + k], y);
    float d = 0.0f;
    if (s < ns) {
      const int64_t r = (start + (s0 + s) * stride) % n;
      const float e = y - t[r * kOut + o];
      atomicAdd(&lsum, e * e);
      d = 2.0f * e / (float)n_used;       // dL/dy
    }
    Y[tid] = d;
  }
  __syncthreads();
  // layer 3 gradients; then dL/da2 overwrites A2
  for (int p = tid; p < kOut * kH + kOut; p += blockDim.x) {
    float g = 0.0f;
    if (p < kOut * kH) {
      const int o = p / kH, k = p - o * kH;
      for (int s = 0; s < kTile; ++s) g = fmaf(Y[s * kOut + o], H2[s * kH + k], g);
      atomicAdd(grad + kW3 + p, g);
    } else {
      const int o = p - kOut * kH;
      for (int s = 0; s < kTile; ++s) g += Y[s * kOut + o];
      atomicAdd(grad + kB3 + o, g);
    }
  }
  __syncthreads();
  for (int i = tid; i < kTile * kH; i += blockDim.x) {
    const int s = i / kH, j = i - s * kH;
    float d = 0.0f;
#pragma unroll
    for (int o = 0; o < kOut; ++o) d = fmaf(Y[s * kOut + o], W3[o * kH + j], d);
    A2[i] = d * gelu_grad_f(A2[i]);
  }
  __syncthreads();
  // layer 2 gradients; then dL/da1 overwrites A1 (H2 is free: it holds dL/dh1)
  for (int p = tid; p < kH * kH + kH; p += blockDim.x) {
    float g = 0.0f;
    if (p < kH * kH) {
      const int j = p / kH, k = p - j * kH;
      for (int s = 0; s < kTile; ++s) g = fmaf(A2[s * kH + j], H1[s * kH + k], g);
      atomicAdd(grad + kW2 + p, g);
    } else {
      const int j = p - kH * kH;
      for (int s = 0; s < kTile; ++s) g += A2[s * kH + j];
      atomicAdd(grad + kB2 + j, g);
    }
  }
  for (int i = tid; i < kTile * kH; i += blockDim.x) {
    const int s = i / kH, k = i - s * kH;
    float d = 0.0f;
#pragma unroll 16
    for (int j = 0; j < kH; ++j) d = fmaf(A2[s * kH + j], W2[j * kH + k], d);
    H2[i] = d;
  }
  __syncthreads();
  for (int i = tid; i < kTile * kH; i += blockDim.x) A1[i] = H2[i] * gelu_grad_f(A1[i]);
  __syncthreads();
  // layer 1 gradients
  for (int p = tid; p < kH * kIn + kH; p += blockDim.x) {
    float g = 0.0f;
    if (p < kH * kIn) {
      const int j = p / kIn, k = p - j * kIn;
      for (int s = 0; s < kTile; ++s) g = fmaf(A1[s * kH + j], X[s * kIn + k], g);
      atomicAdd(grad + kW1 + p, g);
    } else {
      const int j = p - kH * kIn;
      for (int s = 0; s < kTile; ++s) g += A1[s * kH + j];
      atomicAdd(grad + kB1 + j, g);
    }
  }
  __syncthreads();
  if (tid == 0) atomicAdd(loss, lsum / (float)n_used);
}

// Adam step on the FP32 master parameters; refreshes the BF16 copies (the
// training layout and the clip kernel's input-major one) and clears the
// gradient for the next batch.
__global__ void k_adam(float* theta, __nv_bfloat16* wbf, __nv_bfloat16* wbt, float* m, float* v, float* grad, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNParams) return;
  const float g = grad[i];
  const float mi = b1 * m[i] + (1.0f - b1) * g;
  const float vi = b2 * v[i] + (1.0f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  const float th = theta[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  theta[i] = th;
  wbf[i] = __float2bfloat16_rn(th);
  wbt[mlp_transposed_index(i)] = __float2bfloat16_rn(th);
  grad[i] = 0.0f;
}

__global__ void k_mlp_forward(const __nv_bfloat16* wbf, const float* x, int64_t n, float* y) {
  __shared__ float W[kNParams];
  load_weights(wbf, W);
  __syncthreads();
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  float in[kIn], out[kOut];
#pragma unroll
  for (int k = 0; k < kIn; ++k) in[k] = x[s * kIn + k];
  mlp_eval(W, in, out);
  y[s * kOut] = out[0];
  y[s * kOut + 1] = out[1];
}

__global__ void k_zero(float* p, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = 0.0f;
}

// ---- training-set preparation: keep finite rows, normalise, compact ----
constexpr int kPrepThreads = 256;
constexpr int kPrepRows = 1024;   // rows per CTA

__device__ __forceinline__ bool row_valid(const float* f, const float* t, int64_t r) {
  bool ok = isfinite(t[2 * r]) && isfinite(t[2 * r + 1]);
#pragma unroll
  for (int k = 0; k < kIn; ++k) ok = ok && isfinite(f[r * kIn + k]);
  return ok;
}

// Per CTA: number of valid rows, and FP64 sums and sums of squares of the
// 22 columns over them (partials [blocks][2][22]).
__global__ void __launch_bounds__(kPrepThreads) k_prep_stats(const float* f, const float* t, int64_t n,
                                                             int32_t* cnt, double* part) {
  __shared__ double red[2 * (kIn + kOut)][kPrepThreads / 32];
  __shared__ int rc[kPrepThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * kPrepRows;
  double sum[kIn + kOut], sq[kIn + kOut];
#pragma unroll
  for (int c = 0; c < kIn + kOut; ++c) sum[c] = sq[c] = 0.0;
  int valid = 0;
  for (int i = tid; i < kPrepRows; i += kPrepThreads) {
    const int64_t r = r0 + i;
    if (r >= n || !row_valid(f, t, r)) continue;
    ++valid;
#pragma unroll
    for (int c = 0; c < kIn + kOut; ++c) {
      const double v = c < kIn ? (double)f[r * kIn + c] : (double)t[2 * r + c - kIn];
      sum[c] += v;
      sq[c] += v * v;
    }
  }
#pragma unroll
  for (int c = 0; c < kIn + kOut; ++c) {
    for (int o = 16; o > 0; o >>= 1) {
      sum[c] += __shfl_xor_sync(0xffffffffu, sum[c], o);
      sq[c] += __shfl_xor_sync(0xffffffffu, sq[c], o);
    }
  }
  valid = __reduce_add_sync(0xffffffffu, valid);
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < kIn + kOut; ++c) {
      red[c][warp] = sum[c];
      red[kIn + kOut + c][warp] = sq[c];
    }
    rc[warp] = valid;
  }
  __syncthreads();
  if (tid < 2 * (kIn + kOut)) {
    double x = 0.0;
    for (int w = 0; w < kPrepThreads / 32; ++w) x += red[tid][w];
    part[(int64_t)blockIdx.x * 2 * (kIn + kOut) + tid] = x;
  }
  if (tid == 0) {
    int x = 0;
    for (int w = 0; w < kPrepThreads / 32; ++w) x += rc[w];
    cnt[blockIdx.x] = x;
  }
}

// Valid rows of CTA b go, in order, to rows base[b] ... of (x, t), normalised.
__global__ void __launch_bounds__(kPrepThreads) k_prep_scatter(const float* f, const float* t, int64_t n,
                                                               const int64_t* base, const float* norm, float* x,
                                                               float* y) {
  __shared__ int wsum[kPrepThreads / 32];
  __shared__ int64_t off;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * kPrepRows;
  if (tid == 0) off = base[blockIdx.x];
  __syncthreads();
  for (int i0 = 0; i0 < kPrepRows; i0 += kPrepThreads) {
    const int64_t r = r0 + i0 + tid;
    const bool ok = r < n && row_valid(f, t, r);
    const unsigned m = __ballot_sync(0xffffffffu, ok);
    if (lane == 0) wsum[warp] = __popc(m);
    __syncthreads();
    int before = __popc(m & ((1u << lane) - 1u)), total = 0;
    for (int w = 0; w < kPrepThreads / 32; ++w) {
      if (w < warp) before += wsum[w];
      total += wsum[w];
    }
    if (ok) {
      const int64_t o = off + before;
#pragma unroll
      for (int k = 0; k < kIn; ++k) x[o * kIn + k] = (f[r * kIn + k] - norm[k]) / norm[kIn + k];
#pragma unroll
      for (int k = 0; k < kOut; ++k) y[o * kOut + k] = (t[r * kOut + k] - norm[2 * kIn + k]) / norm[2 * kIn + kOut + k];
    }
    __syncthreads();
    if (tid == 0) off += total;
    __syncthreads();
  }
}

}  // namespace

int64_t prep_blocks(int64_t n) { return (n + kPrepRows - 1) / kPrepRows; }

cudaError_t launch_prep_stats(const float* f, const float* t, int64_t n, int32_t* cnt, double* part, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_prep_stats<<<(unsigned)prep_blocks(n), kPrepThreads, 0, s>>>(f, t, n, cnt, part);
  return cudaGetLastError();
}

cudaError_t launch_prep_scatter(const float* f, const float* t, int64_t n, const int64_t* base, const float* norm,
                                float* x, float* y, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_prep_scatter<<<(unsigned)prep_blocks(n), kPrepThreads, 0, s>>>(f, t, n, base, norm, x, y);
  return cudaGetLastError();
}

size_t mlp_grad_smem() {
  return sizeof(float) * ((size_t)kNParams + 2 + kTile * kIn + 4 * kTile * kH + kTile * kOut);
}

cudaError_t launch_mlp_grad(const __nv_bfloat16* wbf, const float* x, const float* t, int64_t n, int64_t n_used,
                            int64_t start, int64_t stride, float* grad, float* loss, cudaStream_t s) {
  if (n_used <= 0) return cudaSuccess;
  const size_t smem = mlp_grad_smem();
  cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t blocks = (n_used + kTile - 1) / kTile;
  k_mlp_grad<<<(unsigned)blocks, kGradThreads, smem, s>>>(wbf, x, t, n, n_used, start, stride, grad, loss);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* theta, __nv_bfloat16* wbf, __nv_bfloat16* wbt, float* m, float* v, float* grad, float lr,
                        int64_t step, cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  k_adam<<<(kNParams + 255) / 256, 256, 0, s>>>(theta, wbf, wbt, m, v, grad, lr, b1, b2, 1e-8f, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const __nv_bfloat16* wbf, const float* x, int64_t n, float* y, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_mlp_forward<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(wbf, x, n, y);
  return cudaGetLastError();
}

cudaError_t launch_zero(float* p, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_zero<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, n);
  return cudaGetLastError();
}

}  // namespace sep
