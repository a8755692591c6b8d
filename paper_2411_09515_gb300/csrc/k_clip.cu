// Fused detector correction + CSR azimuthal integration + sigma-clipping.
//
// One CTA owns one radial bin (a row of the integration matrix) and walks
// frames_per_cta frames. Per frame it gathers the bin's pixels once from the
// frame (raw Jungfrau words are corrected on the fly, Section 1.2), keeps the
// values in shared memory, and runs every clipping pass (Eq. 19, Section 2.4)
// on chip: each moment evaluation is two passes (Eqs. 8-10 for the mean, then
// Eq. 6 / Eq. 11 for the deviation about it), each a block reduction. The
// set after t rejection steps is an interval of values [L_t, H_t] (rejection
// is cumulative and symmetric about the current mean), so no per-entry flag
// is stored. Finally the bin's centre pixels above mean + k_pick sigma are
// marked in the frame's kept-pixel bitmap (sparsification, Section 3).
//
// Precision (SEP_PREC_*): per-thread sums are FP32 (Kahan-compensated except
// in PLAIN); warp sums are FP32 pairs (value, compensation); the cross-warp
// merge and the finalisation (mean, deviation, bounds) are FP64 in
// FP64MERGE and FP32 otherwise.
#include <cuda_runtime.h>
#include <float.h>
#include <stdint.h>

#include "sep_device.cuh"
#include "sep_internal.h"

namespace sep {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// Compensated FP32 accumulator: value = s - c.
template <bool KAHAN>
struct Acc {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float x) {
    if (KAHAN) {
      float y = __fsub_rn(x, c);
      float t = __fadd_rn(s, y);
      c = __fsub_rn(__fsub_rn(t, s), y);
      s = t;
    } else {
      s = __fadd_rn(s, x);
    }
  }
};

// merge (s_a - c_a) + (s_b - c_b) with an error-free two-sum of s_a + s_b
__device__ __forceinline__ void pair_add(float& s, float& c, float so, float co) {
  float t = __fadd_rn(s, so);
  float bp = __fsub_rn(t, s);
  float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(so, bp));  // s + so = t + err exactly
  c = __fsub_rn(__fadd_rn(c, co), err);
  s = t;
}

// Block reduction of NV compensated sums; result (double) in out[] for every thread.
template <int NV, int PREC>
__device__ __forceinline__ void block_reduce(float (&s)[NV], float (&c)[NV], double (&out)[NV],
                                             double (*red)[kWarps], double* bc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float so = __shfl_xor_sync(0xffffffffu, s[v], o);
      if (PREC == SEP_PREC_PLAIN) {
        s[v] = __fadd_rn(s[v], so);
      } else {
        float co = __shfl_xor_sync(0xffffffffu, c[v], o);
        pair_add(s[v], c[v], so, co);
      }
    }
    if (lane == 0) {
      if (PREC == SEP_PREC_FP64MERGE)
        red[v][warp] = (double)s[v] - (double)c[v];
      else if (PREC == SEP_PREC_KAHAN)
        red[v][warp] = (double)__fsub_rn(s[v], c[v]);
      else
        red[v][warp] = (double)s[v];
    }
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      if (PREC == SEP_PREC_FP64MERGE) {
        double x = lane < kWarps ? red[v][lane] : 0.0;
#pragma unroll
        for (int o = kWarps / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) bc[v] = x;
      } else {
        // FP32 merge of the warp partials
        float x = lane < kWarps ? (float)red[v][lane] : 0.0f;
#pragma unroll
        for (int o = kWarps / 2; o > 0; o >>= 1) x = __fadd_rn(x, __shfl_xor_sync(0xffffffffu, x, o));
        if (lane == 0) bc[v] = (double)x;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int v = 0; v < NV; ++v) out[v] = bc[v];
  __syncthreads();
}

template <int PREC>
__device__ __forceinline__ double fin_div(double a, double b) {
  if (PREC == SEP_PREC_FP64MERGE) return a / b;
  return (double)__fdiv_rn((float)a, (float)b);
}
template <int PREC>
__device__ __forceinline__ double fin_sqrt(double a) {
  if (PREC == SEP_PREC_FP64MERGE) return sqrt(a);
  return (double)__fsqrt_rn((float)a);
}
// lower / upper clip bounds as floats such that (v >= lo) == (v >= L) for float v
template <int PREC>
__device__ __forceinline__ float bound_lo(double L) {
  if (PREC == SEP_PREC_FP64MERGE) return __double2float_ru(L);
  return (float)L;
}
template <int PREC>
__device__ __forceinline__ float bound_hi(double H) {
  if (PREC == SEP_PREC_FP64MERGE) return __double2float_rd(H);
  return (float)H;
}

template <int DT, bool SPLIT, bool NORM, int PREC>
__global__ void __launch_bounds__(kThreads) k_integrate_clip(ClipArgs a) {
  constexpr bool KAHAN = PREC != SEP_PREC_PLAIN;
  constexpr bool WEIGHTED = SPLIT || NORM;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* vals = reinterpret_cast<float*>(smem_raw);
  // per-entry weight (WEIGHTED only); its sign bit carries the centre flag
  // (weights are >= 0, and -0.0f still compares equal to 0). Without
  // splitting every entry is its pixel's only entry, hence a centre entry.
  float* wts = vals + a.cap;
  __shared__ double red[3][kWarps];
  __shared__ double bc[3];

  const int b = blockIdx.x;
  const int f0 = blockIdx.y * a.frames_per_cta;
  const int f1 = min(f0 + a.frames_per_cta, a.n_frames);
  const int r0 = a.rowptr[b];
  const int n = a.rowptr[b + 1] - r0;
  const uint32_t* ent = a.ent + r0;
  const int tid = threadIdx.x;

  if (WEIGHTED) {
    for (int e = tid; e < n; e += kThreads) {
      uint32_t u = __ldg(ent + e);
      float w;
      if (u & kZero) w = 0.0f;
      else if (NORM) w = __ldg(a.w + r0 + e);
      else w = (float)(((u >> kKShift) & 3u) + 1u) * 0.25f;
      wts[e] = (u & kCentre) ? -w : w;
    }
  }
  __syncthreads();

  for (int f = f0; f < f1; ++f) {
    const void* frame = DT == SEP_DTYPE_U16_JF
                            ? (const void*)(reinterpret_cast<const uint16_t*>(a.frames) + (int64_t)f * a.npix)
                            : (const void*)(reinterpret_cast<const float*>(a.frames) + (int64_t)f * a.npix);
    // ---- gather + correct; first-pass sums over all entries (Eqs. 8, 10)
    float s3[3] = {0, 0, 0}, c3[3] = {0, 0, 0};
    {
      Acc<KAHAN> om, vv;
      float cnt = 0.0f;
      for (int e = tid; e < n; e += kThreads) {
        uint32_t u = __ldg(ent + e);
        float v = pixel_value<DT, NORM>(frame, (int64_t)(u & kColMask), a.npix, a.ped, a.gain, a.norm);
        vals[e] = v;
        float w = WEIGHTED ? fabsf(wts[e]) : 1.0f;
        if (w != 0.0f) {
          cnt += 1.0f;
          om.add(w);
          vv.add(__fmul_rn(w, v));
        }
      }
      s3[0] = cnt; s3[1] = om.s; c3[1] = om.c; s3[2] = vv.s; c3[2] = vv.c;
    }
    double r3[3];
    block_reduce<3, PREC>(s3, c3, r3, red, bc);
    double n_cur = r3[0], Om = r3[1], V = r3[2];
    float L = -FLT_MAX, H = FLT_MAX;   // current set: L <= v <= H (and weight != 0)
    int steps = 0;
    double mu = 0.0, sd = 0.0;
    for (;;) {
      // ---- moments of the current set: mean (Eq. 12), deviation (Eqs. 11, 13)
      mu = Om != 0.0 ? fin_div<PREC>(V, Om) : 0.0;
      sd = 0.0;
      if (Om != 0.0) {
        const float muf = (float)mu;
        Acc<KAHAN> oo, q;
        for (int e = tid; e < n; e += kThreads) {
          float v = vals[e];
          float w = WEIGHTED ? fabsf(wts[e]) : 1.0f;
          if (v >= L && v <= H && w != 0.0f) {
            float d = __fsub_rn(v, muf);
            float wd = __fmul_rn(w, d);
            oo.add(__fmul_rn(w, w));
            q.add(__fmul_rn(wd, wd));
          }
        }
        float s2[2] = {oo.s, q.s}, c2[2] = {oo.c, q.c};
        double r2[2];
        block_reduce<2, PREC>(s2, c2, r2, red, bc);
        // VV is taken about the FP32-rounded mean; the shift of at most half
        // an ulp of the mean changes VV by a relative (ulp(mu) / sigma)^2
        const double VV = r2[1];
        sd = VV > 0.0 ? fin_sqrt<PREC>(fin_div<PREC>(VV, r2[0])) : 0.0;
      }
      if (steps >= a.n_iter) break;
      // ---- rejection step (Eq. 19): keep |v - mu| <= k sigma, cumulatively
      const double lim = (double)a.k_clip * sd;
      const float L2 = fmaxf(L, bound_lo<PREC>(mu - lim));
      const float H2 = fminf(H, bound_hi<PREC>(mu + lim));
      Acc<KAHAN> om, vv;
      float cnt = 0.0f;
      for (int e = tid; e < n; e += kThreads) {
        float v = vals[e];
        float w = WEIGHTED ? fabsf(wts[e]) : 1.0f;
        if (v >= L2 && v <= H2 && w != 0.0f) {
          cnt += 1.0f;
          om.add(w);
          vv.add(__fmul_rn(w, v));
        }
      }
      s3[0] = cnt; c3[0] = 0.0f; s3[1] = om.s; c3[1] = om.c; s3[2] = vv.s; c3[2] = vv.c;
      block_reduce<3, PREC>(s3, c3, r3, red, bc);
      if (r3[0] == n_cur) break;   // nothing discarded: the set is final
      n_cur = r3[0];
      Om = r3[1];
      V = r3[2];
      L = L2;
      H = H2;
      ++steps;
    }
    const int64_t o = (int64_t)f * a.nbins + b;
    if (tid == 0) {
      a.mean[o] = (float)mu;
      a.sigma[o] = (float)sd;
      a.count[o] = (int32_t)n_cur;
      if (a.bounds) {
        a.bounds[2 * o] = L;
        a.bounds[2 * o + 1] = H;
      }
      if (a.iters) a.iters[o] = steps;
    }
    // ---- sparsification mark (Section 3): centre entries above mu + k_pick sigma
    if (a.bitmap) {
      const float thr = PREC == SEP_PREC_FP64MERGE ? __double2float_rd(mu + (double)a.k_pick * sd)
                                                   : __fadd_rn((float)mu, __fmul_rn(a.k_pick, (float)sd));
      uint32_t* bm = a.bitmap + (int64_t)f * a.words;
      for (int e = tid; e < n; e += kThreads) {
        const bool centre = WEIGHTED ? signbit(wts[e]) : true;
        if (centre && vals[e] > thr) {
          uint32_t col = __ldg(ent + e) & kColMask;
          atomicOr(bm + (col >> 5), 1u << (col & 31u));
        }
      }
    }
    __syncthreads();   // vals are rewritten by the next frame
  }
}

// mode 0: set the shared-memory attribute and launch; 1: attribute only
// (done eagerly before a stream capture); 2: launch only.
template <int DT, bool SPLIT, bool NORM, int PREC>
cudaError_t launch_t(const ClipArgs& a, int mode, cudaStream_t s) {
  constexpr bool WEIGHTED = SPLIT || NORM;
  size_t smem = (size_t)a.cap * (WEIGHTED ? 8 : 4);
  smem = (smem + 15) & ~(size_t)15;
  auto k = k_integrate_clip<DT, SPLIT, NORM, PREC>;
  if (mode != 2) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess || mode == 1) return e;
  }
  dim3 grid(a.nbins, (a.n_frames + a.frames_per_cta - 1) / a.frames_per_cta);
  k<<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <int DT, bool SPLIT, bool NORM>
cudaError_t launch_p(const ClipArgs& a, int32_t prec, int mode, cudaStream_t s) {
  switch (prec) {
    case SEP_PREC_PLAIN: return launch_t<DT, SPLIT, NORM, SEP_PREC_PLAIN>(a, mode, s);
    case SEP_PREC_KAHAN: return launch_t<DT, SPLIT, NORM, SEP_PREC_KAHAN>(a, mode, s);
    default: return launch_t<DT, SPLIT, NORM, SEP_PREC_FP64MERGE>(a, mode, s);
  }
}

template <int DT>
cudaError_t launch_d(const ClipArgs& a, bool split, bool norm, int32_t prec, int mode, cudaStream_t s) {
  if (norm) return split ? launch_p<DT, true, true>(a, prec, mode, s) : launch_p<DT, false, true>(a, prec, mode, s);
  return split ? launch_p<DT, true, false>(a, prec, mode, s) : launch_p<DT, false, false>(a, prec, mode, s);
}

}  // namespace

size_t clip_smem_bytes(int32_t cap, bool weighted) {
  size_t smem = (size_t)cap * (weighted ? 8 : 4);
  return (smem + 15) & ~(size_t)15;
}

cudaError_t launch_integrate_clip(const ClipArgs& a, int32_t dtype, bool split, bool has_norm, int32_t precision,
                                  int mode, cudaStream_t s) {
  if (a.n_frames <= 0 || a.nbins <= 0) return cudaSuccess;
  if (dtype == SEP_DTYPE_U16_JF) return launch_d<SEP_DTYPE_U16_JF>(a, split, has_norm, precision, mode, s);
  return launch_d<SEP_DTYPE_F32>(a, split, has_norm, precision, mode, s);
}

}  // namespace sep
