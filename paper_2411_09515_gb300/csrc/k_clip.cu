// Fused detector correction + CSR azimuthal integration + sigma-clipping.
//
// One CTA (64, 128 or 256 threads: a tuning choice per size class of bins)
// owns one radial bin (a row of the integration matrix) and walks a group of
// frames. Per frame it gathers the bin's pixels
// once from the frame, corrects them (Section 1.2), and keeps the values in
// shared memory; every clipping pass (Eq. 19, Section 2.4) then runs on chip.
//
// Moments (Eqs. 8-13) are accumulated about a shift K (the previous mean):
// with d = v - K, per set S
//   Omega = sum w, A1 = sum w d, OO = sum w^2, B1 = sum w^2 d, B2 = sum w^2 d^2,
//   mu = K + A1 / Omega,  VV = B2 - 2 (mu - K) B1 + (mu - K)^2 OO  (Eq. 11),
//   sigma = sqrt(VV / OO)  (Eq. 13),
// which is exact algebra; with K close to mu the correction terms are small,
// so one pass per moment evaluation suffices (the gather pass supplies the
// first shift).
//
// Rejection is cumulative and symmetric about the current mean, so the set
// after t steps is every entry whose value lies in an interval [L_t, H_t]:
// no per-entry flag is kept. Row entries are grouped by coefficient class
// (a group shares one weight), so per-entry work is unweighted and the
// class weight is applied once per thread per pass.
//
// After the last evaluation, the bin's centre entries above mu + k_pick sigma
// set their pixel's bit in the frame's kept-pixel bitmap (Section 3).
//
// Precision (SEP_PREC_*): per-thread FP32 sums (Kahan-compensated in KAHAN)
// and FP32 warp shuffles (error-free pairs in KAHAN). The cross-warp merge,
// the variance finalisation and the clip bounds run on one warp only: FP64
// in FP64MERGE, FP32 pairs in KAHAN, FP32 in PLAIN. (FP64 runs at a small
// fraction of the FP32 rate on this GPU, so no FP64 instruction is issued by
// the other warps.)
#include <cuda_runtime.h>
#include <float.h>
#include <stdint.h>

#include "sep_device.cuh"
#include "sep_internal.h"

namespace sep {
namespace {


enum { MODE_UNIT = 0, MODE_CLASS = 1, MODE_ENTRY = 2 };

template <bool KAHAN>
struct Acc {
  float s = 0.0f, c = 0.0f;   // value = s - c
  __device__ __forceinline__ void add(float x) {
    if (KAHAN) {
      const float y = __fsub_rn(x, c);
      const float t = __fadd_rn(s, y);
      c = __fsub_rn(__fsub_rn(t, s), y);
      s = t;
    } else {
      s = __fadd_rn(s, x);
    }
  }
  __device__ __forceinline__ float val() const { return KAHAN ? __fsub_rn(s, c) : s; }
};

// (s - c) += (so - co): error-free two-sum of the leading parts
__device__ __forceinline__ void pair_add(float& s, float& c, float so, float co) {
  const float t = __fadd_rn(s, so);
  const float bp = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(so, bp));
  c = __fsub_rn(__fadd_rn(c, co), err);
  s = t;
}

// Shift of the next pass. With K = 0 the deviations d = v are exact, and
// the variance terms cancel by at most a factor 1 + mu^2 / sigma^2 <= 5 when
// |mu| <= 2 sigma; otherwise K = mu keeps the cancellation small and the
// rounding of d = v - K (relative 2^-24 of |d| ~ sigma) is far below the
// mean's own scale.
__device__ __forceinline__ float choose_shift(float mu, float sd) { return fabsf(mu) <= 2.0f * sd ? 0.0f : mu; }

// State shared by the CTA between passes (written by one thread).
struct Bcast {
  double mu, sd;       // moments of the current set
  float Ln, Hn, Kf;    // interval and shift of the next pass
  float L, H;          // interval of the current set
  float n_cur;         // entries (weight != 0) in the current set
  int steps, done;
};

// Moments of one set from its shifted sums (one thread).
template <int PREC>
__device__ __forceinline__ void finalise(double K, double Om, double A1, double OO, double B1, double B2, double& mu,
                                         double& sd) {
  if (Om == 0.0) {
    mu = 0.0;
    sd = 0.0;
    return;
  }
  if (PREC == SEP_PREC_PLAIN) {
    const float Kf = (float)K;
    const float muf = __fadd_rn(Kf, __fdiv_rn((float)A1, (float)Om));
    const float dl = __fsub_rn(muf, Kf);
    const float VV = __fadd_rn(__fsub_rn((float)B2, __fmul_rn(2.0f * dl, (float)B1)),
                               __fmul_rn(__fmul_rn(dl, dl), (float)OO));
    mu = (double)muf;
    sd = VV > 0.0f ? (double)__fsqrt_rn(__fdiv_rn(VV, (float)OO)) : 0.0;
  } else {
    // the two divisions act on a small correction and on a ratio: FP32 is exact enough
    mu = K + (double)__fdiv_rn((float)A1, (float)Om);
    const double dl = mu - K;
    const double VV = fma(dl * dl, OO, fma(-2.0 * dl, B1, B2));
    sd = VV > 0.0 ? (double)__fsqrt_rn(__fdiv_rn((float)VV, (float)OO)) : 0.0;
  }
}

// Next interval: keep |v - mu| <= k sd. With FP64 moments the float bounds
// use directed rounding, so for any float v (v >= L) == (v >= mu - k sd).
template <int PREC>
__device__ __forceinline__ void clip_bounds(double mu, double sd, float k, float& L, float& H) {
  if (PREC == SEP_PREC_PLAIN) {
    const float m = (float)mu, s = (float)sd;
    L = fmaxf(L, __fsub_rn(m, __fmul_rn(k, s)));
    H = fminf(H, __fadd_rn(m, __fmul_rn(k, s)));
  } else {
    L = fmaxf(L, __double2float_ru(fma(-(double)k, sd, mu)));
    H = fminf(H, __double2float_rd(fma((double)k, sd, mu)));
  }
}

// Sum NV per-thread values over the CTA; lanes v < NV of warp 0 hold total v
// on return (as double). Ends without a barrier: the caller's warp 0 works
// on the totals and then synchronises.
template <int NV, int PREC, int kWarps>
__device__ __forceinline__ double block_sum(float (&s)[NV], float (&c)[NV], float (*red_s)[kWarps],
                                            float (*red_c)[kWarps]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      if (PREC == SEP_PREC_KAHAN) {
        const float so = __shfl_xor_sync(0xffffffffu, s[v], o);
        const float co = __shfl_xor_sync(0xffffffffu, c[v], o);
        pair_add(s[v], c[v], so, co);
      } else {
        s[v] = __fadd_rn(s[v], __shfl_xor_sync(0xffffffffu, s[v], o));
      }
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      red_s[v][warp] = s[v];
      red_c[v][warp] = PREC == SEP_PREC_KAHAN ? c[v] : 0.0f;
    }
  }
  __syncthreads();
  double tot = 0.0;
  if (warp == 0 && lane < NV) {
    if (PREC == SEP_PREC_FP64MERGE) {
#pragma unroll
      for (int w = 0; w < kWarps; ++w) tot += (double)red_s[lane][w];
    } else if (PREC == SEP_PREC_KAHAN) {
      float hs = red_s[lane][0], hc = red_c[lane][0];
#pragma unroll
      for (int w = 1; w < kWarps; ++w) pair_add(hs, hc, red_s[lane][w], red_c[lane][w]);
      tot = (double)hs - (double)hc;
    } else {
      float x = red_s[lane][0];
#pragma unroll
      for (int w = 1; w < kWarps; ++w) x = __fadd_rn(x, red_s[lane][w]);
      tot = (double)x;
    }
  }
  return tot;
}

template <int DT, int MODE, int PREC, int kThreads>
__global__ void __launch_bounds__(kThreads) k_integrate_clip(ClipArgs a) {
  constexpr int kWarps = kThreads / 32;
  constexpr bool KAHAN = PREC == SEP_PREC_KAHAN;
  // MODE_UNIT: one class of weight 1; sums (count, S1, S2).
  // MODE_CLASS / MODE_ENTRY: sums (count, Omega, A1, OO, B1, B2).
  constexpr int NV = MODE == MODE_UNIT ? 3 : 6;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* vals = reinterpret_cast<float*>(smem_raw);
  float* wts = vals + a.cap;   // MODE_ENTRY only: per-entry weight
  __shared__ float red_s[NV][kWarps], red_c[NV][kWarps];
  __shared__ Bcast st;

  const int b = a.bin_list ? __ldg(a.bin_list + blockIdx.x) : (int)blockIdx.x;
  const int f0 = blockIdx.y * a.frames_per_cta;
  const int f1 = min(f0 + a.frames_per_cta, a.n_frames);
  const int r0 = __ldg(a.rowptr + b);
  const int n = __ldg(a.rowptr + b + 1) - r0;      // multiple of 4
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int ge[4];   // end of coefficient class 0..3 in the row; weight-0 carriers follow
#pragma unroll
  for (int c = 0; c < 4; ++c) ge[c] = __ldg(a.grp + 4 * b + c);
  const uint4* ent4 = reinterpret_cast<const uint4*>(a.ent + r0);
  float4* vals4 = reinterpret_cast<float4*>(vals);
  const int nq = n >> 2;

  if (MODE == MODE_ENTRY) {
    for (int e = tid; e < n; e += kThreads) {
      const uint32_t u = __ldg(a.ent + r0 + e);
      wts[e] = (u & (kZero | kPad)) ? 0.0f : __ldg(a.w + r0 + e);
    }
  }

  for (int f = f0; f < f1; ++f) {
    const void* frame = frame_ptr<DT>(a.frames, f, a.npix);
    // ------------- gather + correct; rough sums giving the first shift -------------
    float s0[NV], c0[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) s0[v] = c0[v] = 0.0f;
    {
      float om = 0.0f, vv = 0.0f, v2 = 0.0f;
      // two vectors of 4 entries per step, every load issued before any use
      for (int qa = tid; qa < nq; qa += 2 * kThreads) {
        const int qs[2] = {qa, qa + kThreads};
        uint32_t uu[2][4];
        float pp[2][4], gg[2][4];
        uint32_t rw[2][4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const bool ok = qs[h] < nq;
          const uint4 u = ok ? __ldg(ent4 + qs[h]) : make_uint4(kPad, kPad, kPad, kPad);
          uu[h][0] = u.x; uu[h][1] = u.y; uu[h][2] = u.z; uu[h][3] = u.w;
          if (DT == SEP_DTYPE_U16_JF && ok) {
            const float4* cal4 = reinterpret_cast<const float4*>(a.cal0 + r0);
            const float4 ca = __ldg(cal4 + 2 * qs[h]), cb = __ldg(cal4 + 2 * qs[h] + 1);
            pp[h][0] = ca.x; gg[h][0] = ca.y; pp[h][1] = ca.z; gg[h][1] = ca.w;
            pp[h][2] = cb.x; gg[h][2] = cb.y; pp[h][3] = cb.z; gg[h][3] = cb.w;
          } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) { pp[h][j] = 0.0f; gg[h][j] = 1.0f; }
          }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int64_t col = uu[h][j] & kColMask;
            if (uu[h][j] & kPad) rw[h][j] = 0u;
            else if (DT == SEP_DTYPE_U16_JF) rw[h][j] = __ldg(reinterpret_cast<const uint16_t*>(frame) + col);
            else rw[h][j] = __float_as_uint(__ldg(reinterpret_cast<const float*>(frame) + col));
          }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (qs[h] >= nq) continue;
          float x[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (uu[h][j] & kPad) {
              x[j] = __int_as_float(0x7fc00000);   // NaN: outside every interval
              continue;
            }
            const int64_t col = uu[h][j] & kColMask;
            if (DT == SEP_DTYPE_U16_JF) {
              const uint32_t raw = rw[h][j], code = raw >> 14;
              float ped = pp[h][j], gain = gg[h][j];
              if (code != 0) {   // gain levels 1 and 2 are rare: read the pixel-ordered planes
                const int64_t lvl = code == 1 ? 1 : 2;
                ped = __ldg(a.ped + lvl * a.npix + col);
                gain = __ldg(a.gain + lvl * a.npix + col);
              }
              x[j] = __fdiv_rn(__fsub_rn((float)(raw & 0x3FFFu), ped), gain);
            } else {
              x[j] = __uint_as_float(rw[h][j]);
            }
            if (MODE == MODE_ENTRY) x[j] = __fdiv_rn(x[j], __ldg(a.norm + col));
          }
          vals4[qs[h]] = make_float4(x[0], x[1], x[2], x[3]);
          // rough sums (plain FP32): they only choose the first shift
          const int e0 = qs[h] << 2;
          if (e0 < ge[3]) {
            float w = 1.0f;
            if (MODE == MODE_CLASS) w = e0 < ge[0] ? 1.0f : (e0 < ge[1] ? 0.75f : (e0 < ge[2] ? 0.5f : 0.25f));
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              if (MODE == MODE_ENTRY) w = wts[e0 + j];
              if (x[j] == x[j] && w != 0.0f) {
                om += w;
                const float wx = w * x[j];
                vv += wx;
                v2 = fmaf(wx, x[j], v2);
              }
            }
          }
        }
      }
      s0[0] = om;
      s0[1] = vv;
      s0[2] = v2;
    }
    {
      const double t = block_sum<NV, SEP_PREC_PLAIN, kWarps>(s0, c0, red_s, red_c);
      // lanes 0, 1, 2 of warp 0 hold Omega, V, sum w v^2
      const double Om = __shfl_sync(0xffffffffu, t, 0);
      const double V = __shfl_sync(0xffffffffu, t, 1);
      const double V2 = __shfl_sync(0xffffffffu, t, 2);
      if (tid == 0) {
        float K = 0.0f;
        if (Om > 0.0) {
          const float m = __fdiv_rn((float)V, (float)Om);
          const float var = __fsub_rn(__fdiv_rn((float)V2, (float)Om), m * m);
          K = choose_shift(m, var > 0.0f ? sqrtf(var) : 0.0f);
        }
        st.Kf = K;
        st.Ln = -FLT_MAX;
        st.Hn = FLT_MAX;
        st.L = -FLT_MAX;
        st.H = FLT_MAX;
        st.n_cur = -1.0f;
        st.steps = -1;
        st.done = 0;
        st.mu = 0.0;
        st.sd = 0.0;
      }
      __syncthreads();   // values and state visible to all
    }

    for (;;) {
      // ------------- one pass: shifted sums over entries in [Ln, Hn] -------------
      const float Ln = st.Ln, Hn = st.Hn, Kf = st.Kf;
      float ss[NV], cc[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) ss[v] = cc[v] = 0.0f;
      if (MODE == MODE_CLASS) {
        int lo = 0;
#pragma unroll
        for (int cls = 0; cls < 4; ++cls) {
          const int hi = ge[cls];
          const float w = 1.0f - 0.25f * (float)cls, w2 = w * w;
          float cnt = 0.0f;
          Acc<KAHAN> a1, a2;
          for (int q = (lo >> 2) + tid; q < (hi >> 2); q += kThreads) {
            const float4 v4 = vals4[q];
            const float xs[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              if (xs[j] >= Ln && xs[j] <= Hn) {
                const float d = __fsub_rn(xs[j], Kf);
                cnt += 1.0f;
                a1.add(d);
                a2.add(__fmul_rn(d, d));
              }
            }
          }
          // weights k/4 times counts below 2^22 are exact in FP32
          const float s1 = a1.val(), s2 = a2.val();
          ss[0] += cnt;
          ss[1] += w * cnt;
          ss[3] += w2 * cnt;
          if (KAHAN) {
            Acc<true> t2, t4, t5;
            t2.s = ss[2]; t2.c = cc[2]; t2.add(__fmul_rn(w, s1)); ss[2] = t2.s; cc[2] = t2.c;
            t4.s = ss[4]; t4.c = cc[4]; t4.add(__fmul_rn(w2, s1)); ss[4] = t4.s; cc[4] = t4.c;
            t5.s = ss[5]; t5.c = cc[5]; t5.add(__fmul_rn(w2, s2)); ss[5] = t5.s; cc[5] = t5.c;
          } else {
            ss[2] = fmaf(w, s1, ss[2]);
            ss[4] = fmaf(w2, s1, ss[4]);
            ss[5] = fmaf(w2, s2, ss[5]);
          }
          lo = hi;
        }
      } else if (MODE == MODE_UNIT) {
        float cnt = 0.0f;
        Acc<KAHAN> a1, a2;
        for (int q = tid; q < (ge[0] >> 2); q += kThreads) {
          const float4 v4 = vals4[q];
          const float xs[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (xs[j] >= Ln && xs[j] <= Hn) {
              const float d = __fsub_rn(xs[j], Kf);
              cnt += 1.0f;
              a1.add(d);
              a2.add(__fmul_rn(d, d));
            }
          }
        }
        ss[0] = cnt; ss[1] = a1.s; cc[1] = a1.c; ss[2] = a2.s; cc[2] = a2.c;
      } else {
        float cnt = 0.0f;
        Acc<KAHAN> om, a1, oo, b1, b2;
        for (int q = tid; q < (ge[3] >> 2); q += kThreads) {
          const float4 v4 = vals4[q];
          const float xs[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float w = wts[4 * q + j];
            if (w != 0.0f && xs[j] >= Ln && xs[j] <= Hn) {
              const float d = __fsub_rn(xs[j], Kf);
              const float w2 = __fmul_rn(w, w);
              const float w2d = __fmul_rn(w2, d);
              cnt += 1.0f;
              om.add(w);
              a1.add(__fmul_rn(w, d));
              oo.add(w2);
              b1.add(w2d);
              b2.add(__fmul_rn(w2d, d));
            }
          }
        }
        ss[0] = cnt;
        ss[1] = om.s; cc[1] = om.c; ss[2] = a1.s; cc[2] = a1.c; ss[3] = oo.s; cc[3] = oo.c;
        ss[4] = b1.s; cc[4] = b1.c; ss[5] = b2.s; cc[5] = b2.c;
      }
      const double tot = block_sum<NV, PREC, kWarps>(ss, cc, red_s, red_c);
      if (warp == 0) {
        double t[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) t[v] = __shfl_sync(0xffffffffu, tot, v);
        if (lane == 0) {
          // the pass measured S' = S ∩ [Ln, Hn]; S' == S means nothing was discarded
          if (st.steps >= 0 && (float)t[0] == st.n_cur) {
            st.done = 1;
          } else {
            st.n_cur = (float)t[0];
            st.L = Ln;
            st.H = Hn;
            double mu, sd;
            if (MODE == MODE_UNIT)
              finalise<PREC>((double)Kf, t[0], t[1], t[0], t[1], t[2], mu, sd);
            else
              finalise<PREC>((double)Kf, t[1], t[2], t[3], t[4], t[5], mu, sd);
            st.mu = mu;
            st.sd = sd;
            st.steps += 1;
            if (st.steps >= a.n_iter) {
              st.done = 1;
            } else {   // next set: reject |v - mu| > k sd (Eq. 19), cumulatively
              float L2 = Ln, H2 = Hn;
              clip_bounds<PREC>(mu, sd, a.k_clip, L2, H2);
              st.Ln = L2;
              st.Hn = H2;
              st.Kf = choose_shift((float)mu, (float)sd);
            }
          }
        }
      }
      __syncthreads();
      if (st.done) break;
    }
    const double mu = st.mu, sd = st.sd;
    const int64_t o = (int64_t)f * a.nbins + b;
    if (tid == 0) {
      a.mean[o] = (float)mu;
      a.sigma[o] = (float)sd;
      a.count[o] = (int32_t)st.n_cur;
      if (a.bounds) {
        a.bounds[2 * o] = st.L;
        a.bounds[2 * o + 1] = st.H;
      }
      if (a.iters) a.iters[o] = st.steps;
    }
    // ---------------- sparsification mark (Section 3) ----------------
    if (a.bitmap) {
      __shared__ float thr_s;
      if (tid == 0)
        thr_s = PREC == SEP_PREC_PLAIN ? __fadd_rn((float)mu, __fmul_rn(a.k_pick, (float)sd))
                                       : __double2float_rd(fma((double)a.k_pick, sd, mu));
      __syncthreads();
      const float thr = thr_s;
      uint32_t* bm = a.bitmap + (int64_t)f * a.words;
      for (int q = tid; q < nq; q += kThreads) {
        const float4 v4 = vals4[q];
        const float xs[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (xs[j] > thr) {   // NaN padding never passes
            const uint32_t u = __ldg(a.ent + r0 + 4 * q + j);
            if (MODE == MODE_UNIT || (u & kCentre)) {
              const uint32_t col = u & kColMask;
              atomicOr(bm + (col >> 5), 1u << (col & 31u));
            }
          }
        }
      }
    }
    __syncthreads();   // vals and state are rewritten by the next frame
  }
}

// mode 0: set the shared-memory attribute and launch; 1: attribute only
// (done eagerly before a stream capture); 2: launch only.
template <int DT, int MODE, int PREC, int TPB>
cudaError_t launch_t(const ClipArgs& a, int n_ctas, int mode, cudaStream_t s) {
  const size_t smem = clip_smem_bytes(a.cap, MODE == MODE_ENTRY);
  auto k = k_integrate_clip<DT, MODE, PREC, TPB>;
  if (mode != 2) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess || mode == 1) return e;
  }
  dim3 grid(n_ctas, (a.n_frames + a.frames_per_cta - 1) / a.frames_per_cta);
  k<<<grid, TPB, smem, s>>>(a);
  return cudaGetLastError();
}

template <int DT, int MODE, int PREC>
cudaError_t launch_b(const ClipArgs& a, int n_ctas, int tpb, int mode, cudaStream_t s) {
  switch (tpb) {
    case 64: return launch_t<DT, MODE, PREC, 64>(a, n_ctas, mode, s);
    case 128: return launch_t<DT, MODE, PREC, 128>(a, n_ctas, mode, s);
    default: return launch_t<DT, MODE, PREC, 256>(a, n_ctas, mode, s);
  }
}

template <int DT, int MODE>
cudaError_t launch_p(const ClipArgs& a, int n_ctas, int tpb, int32_t prec, int mode, cudaStream_t s) {
  switch (prec) {
    case SEP_PREC_PLAIN: return launch_b<DT, MODE, SEP_PREC_PLAIN>(a, n_ctas, tpb, mode, s);
    case SEP_PREC_KAHAN: return launch_b<DT, MODE, SEP_PREC_KAHAN>(a, n_ctas, tpb, mode, s);
    default: return launch_b<DT, MODE, SEP_PREC_FP64MERGE>(a, n_ctas, tpb, mode, s);
  }
}

template <int DT>
cudaError_t launch_d(const ClipArgs& a, int n_ctas, int tpb, bool split, bool norm, int32_t prec, int mode,
                     cudaStream_t s) {
  if (norm) return launch_p<DT, MODE_ENTRY>(a, n_ctas, tpb, prec, mode, s);
  return split ? launch_p<DT, MODE_CLASS>(a, n_ctas, tpb, prec, mode, s)
               : launch_p<DT, MODE_UNIT>(a, n_ctas, tpb, prec, mode, s);
}

}  // namespace

size_t clip_smem_bytes(int32_t cap, bool weighted) {
  size_t smem = (size_t)cap * (weighted ? 8 : 4);
  return (smem + 15) & ~(size_t)15;
}

cudaError_t launch_integrate_clip(const ClipArgs& a, int n_ctas, int tpb, int32_t dtype, bool split, bool has_norm,
                                  int32_t precision, int mode, cudaStream_t s) {
  if (a.n_frames <= 0 || n_ctas <= 0) return cudaSuccess;
  if (dtype == SEP_DTYPE_U16_JF) return launch_d<SEP_DTYPE_U16_JF>(a, n_ctas, tpb, split, has_norm, precision, mode, s);
  return launch_d<SEP_DTYPE_F32>(a, n_ctas, tpb, split, has_norm, precision, mode, s);
}

}  // namespace sep
