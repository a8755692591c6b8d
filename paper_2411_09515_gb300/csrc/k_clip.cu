// Integration + sigma-clipping over staged pixel values.
//
// One warp owns one radial bin (a row of the integration matrix) of one
// frame: it reads the bin's values from the frame's staged copy (k_stage.cu:
// corrected pixels, Section 1.2, one slot per matrix entry, so a bin's
// values are one contiguous run), accumulates the weighted moments
// (Eqs. 8-13) and runs the clip loop of Eq. 19 (Section 2.4) by tail replay
// (described with the kernel below). The warps of a CTA take other frames
// of the same bin and wait for one another only when the CTA takes its next
// unit of work (a persistent launch draws units from a work-queue counter).
//
// Moments are accumulated about a shift K: with d = v - K, per set S
//   Omega = sum w, A1 = sum w d, OO = sum w^2, B1 = sum w^2 d, B2 = sum w^2 d^2,
//   mu = K + A1 / Omega,  VV = B2 - 2 (mu - K) B1 + (mu - K)^2 OO  (Eq. 11),
//   sigma = sqrt(VV / OO)  (Eq. 13),
// which is exact algebra; with K close to mu (or 0 where |mu| <= 2 sigma)
// the correction terms are small.
//
// Rejection is cumulative and symmetric about the current mean, so the set
// after t steps is every entry whose value lies in an interval [L_t, H_t]:
// no per-entry flag is kept. Row entries are grouped by coefficient class (a
// group shares one weight), so per-entry work is unweighted and the class
// weight is applied once per lane and class.
//
// After the last evaluation the kernel writes mu + k_pick sigma, the bin's
// sparsification threshold (Section 3); with a bitmap it also marks the
// bin's kept pixels (its centre entries above the threshold).
//
// Precision (SEP_PREC_*): per-lane FP32 sums (Kahan-compensated in KAHAN);
// the merge over the lanes and the finalisation in plain FP32 (PLAIN),
// error-free FP32 pairs ("double-word": KAHAN and DWORD, the default) or
// FP64 (FP64MERGE). FP64 runs at a small fraction of the FP32 rate on this
// GPU, so DWORD issues no FP64 instruction.
#include <cuda_runtime.h>
#include <float.h>
#include <stdint.h>

#include <algorithm>

#include "sep_device.cuh"
#include "sep_internal.h"
#include "sep_mlp.cuh"

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
  // += x * y: compensated product in KAHAN, one fused multiply-add otherwise
  __device__ __forceinline__ void add_prod(float x, float y) {
    if (KAHAN) add(__fmul_rn(x, y));
    else s = __fmaf_rn(x, y, s);
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

// State of an item's clip loop (every lane of its warp holds the same
// copy, evaluated from bit-identical totals). The mean is kept as an
// unevaluated FP32 pair mu_hi + mu_lo (FP64MERGE keeps a double).
struct Bcast {
  double mu_d, sd_d;   // FP64MERGE
  float mu_hi, mu_lo, sd;
  float Ln, Hn, Kf;    // interval and shift of the next pass
  float L, H;          // interval of the current set
  float n_cur;         // entries (weight != 0) in the current set
  int steps, done;
  float sdP;           // Poisson deviation of the current set (error models 1, 2)
  double sdP_d;        // FP64MERGE
};

// Error-free sum: a + b = s + e exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// Smallest float >= hi + lo and largest float <= hi + lo for a normalised
// pair (hi = RN(hi + lo)).
__device__ __forceinline__ float round_up_pair(float hi, float lo) { return lo > 0.0f ? nextafterf(hi, INFINITY) : hi; }
__device__ __forceinline__ float round_dn_pair(float hi, float lo) { return lo < 0.0f ? nextafterf(hi, -INFINITY) : hi; }

// Mean and deviation of one set from its shifted sums (each lane of the
// item's warp, on the same totals):
//   mu = K + A1 / Omega,  VV = B2 - 2 (mu - K) B1 + (mu - K)^2 OO,  sd = sqrt(VV / OO)
// Sums arrive as FP32 pairs (value = hi + lo). The divisions act on a small
// correction and on a ratio, where FP32 is exact to ~1e-7 relative; the
// mean is kept as the exact pair K + corr. FP64MERGE does the same in FP64.
template <int PREC>
__device__ __forceinline__ void finalise(float Kf, const float (&hi)[6], const float (&lo)[6], Bcast& st) {
  // hi/lo layout: 0 Omega, 1 A1, 2 OO, 3 B1, 4 B2
  if (hi[0] == 0.0f) {
    st.mu_hi = st.mu_lo = st.sd = 0.0f;
    st.mu_d = st.sd_d = 0.0;
    return;
  }
  if (PREC == SEP_PREC_FP64MERGE) {
    const double Om = (double)hi[0] + lo[0], A1 = (double)hi[1] + lo[1], OO = (double)hi[2] + lo[2];
    const double B1 = (double)hi[3] + lo[3], B2 = (double)hi[4] + lo[4];
    const double mu = (double)Kf + (double)__fdiv_rn((float)A1, (float)Om);
    const double dl = mu - (double)Kf;
    const double VV = fma(dl * dl, OO, fma(-2.0 * dl, B1, B2));
    st.mu_d = mu;
    st.sd_d = VV > 0.0 ? (double)__fsqrt_rn(__fdiv_rn((float)VV, (float)OO)) : 0.0;
    st.mu_hi = (float)mu;
    st.mu_lo = (float)(mu - (double)st.mu_hi);
    st.sd = (float)st.sd_d;
    return;
  }
  const float Om = __fadd_rn(hi[0], lo[0]), OO = __fadd_rn(hi[2], lo[2]);
  const float corr = __fdiv_rn(__fadd_rn(hi[1], lo[1]), Om);
  if (PREC == SEP_PREC_PLAIN) {
    st.mu_hi = __fadd_rn(Kf, corr);
    st.mu_lo = 0.0f;
  } else {
    two_sum(Kf, corr, st.mu_hi, st.mu_lo);
  }
  // VV with the small correction terms in FP32 and the leading B2 as a pair
  float VV = __fsub_rn(hi[4], __fmul_rn(2.0f * corr, __fadd_rn(hi[3], lo[3])));
  VV = __fadd_rn(VV, __fmul_rn(__fmul_rn(corr, corr), OO));
  VV = __fadd_rn(VV, lo[4]);
  st.sd = VV > 0.0f ? __fsqrt_rn(__fdiv_rn(VV, OO)) : 0.0f;
}

// Next interval: keep |v - mu| <= k sd (Eq. 19). Except in PLAIN the float
// bounds are rounded outward-exact from the extended mean, so for any float
// v the test v >= L equals v >= mu - k sd up to the rounding of k sd.
template <int PREC>
__device__ __forceinline__ void clip_bounds(const Bcast& st, float k, float& L, float& H) {
  if (PREC == SEP_PREC_PLAIN) {
    const float ks = __fmul_rn(k, st.sd);
    L = fmaxf(L, __fsub_rn(st.mu_hi, ks));
    H = fminf(H, __fadd_rn(st.mu_hi, ks));
  } else if (PREC == SEP_PREC_FP64MERGE) {
    L = fmaxf(L, __double2float_ru(fma(-(double)k, st.sd_d, st.mu_d)));
    H = fminf(H, __double2float_rd(fma((double)k, st.sd_d, st.mu_d)));
  } else {
    const float ks = __fmul_rn(k, st.sd);
    float a, e;
    two_sum(st.mu_hi, -ks, a, e);
    e = __fadd_rn(e, st.mu_lo);
    float lh, ll;
    two_sum(a, e, lh, ll);
    L = fmaxf(L, round_up_pair(lh, ll));
    two_sum(st.mu_hi, ks, a, e);
    e = __fadd_rn(e, st.mu_lo);
    two_sum(a, e, lh, ll);
    H = fminf(H, round_dn_pair(lh, ll));
  }
}

// Threshold of sparsification, mu + k_pick sd, rounded down (v > thr is
// then the exact comparison for float v, up to the rounding of k sd).
template <int PREC>
__device__ __forceinline__ float pick_threshold(const Bcast& st, float k) {
  if (PREC == SEP_PREC_PLAIN) return __fadd_rn(st.mu_hi, __fmul_rn(k, st.sd));
  if (PREC == SEP_PREC_FP64MERGE) return __double2float_rd(fma((double)k, st.sd_d, st.mu_d));
  const float ks = __fmul_rn(k, st.sd);
  float a, e, th, tl;
  two_sum(st.mu_hi, ks, a, e);
  e = __fadd_rn(e, st.mu_lo);
  two_sum(a, e, th, tl);
  return round_dn_pair(th, tl);
}

template <int MODE>
struct Sums {
  // per pass, float sums and integer counts:
  //   MODE_UNIT:  (S1, S2) + count
  //   MODE_CLASS: (A1, B1, B2) + class counts packed 16 + 16 bits in two words
  //   MODE_ENTRY: (Omega, A1, OO, B1, B2) + count
  // (a row holds fewer than 2^16 entries: the host refuses longer rows; tail
  // slots keep an entry's index in 16 bits)
  static constexpr int NF = MODE == MODE_UNIT ? 2 : (MODE == MODE_CLASS ? 3 : 5);
  static constexpr int NI = MODE == MODE_CLASS ? 2 : 1;
};

// One step of the clip loop (every lane of the warp, on identical totals) after a pass measured the set
// S' = S ∩ [Ln, Hn] (count n_set, sums h/l about Kf). S' == S means nothing
// was discarded: the loop ends with the moments of S. Otherwise S' becomes
// the set, its moments are evaluated and the next interval is the
// intersection with [mu - k sd, mu + k sd] (Eq. 19, cumulative).
// (have_moments: st already holds the moments of S'.)
// Poisson deviation of a set (Eqs. 3-4, normalised as Eq. 13): each
// value's variance is the value plus the dark variance, weighted by the
// squared coefficients: sdP^2 = sum w^2 v / sum w^2 + dark = Kf + B1 / OO +
// dark from the pass's sums about Kf (0 when negative or the set is empty).
template <int PREC>
__device__ __forceinline__ void poisson_sd(float Kf, const float (&hi)[6], const float (&lo)[6], float dark,
                                           Bcast& st) {
  // hi/lo layout: 0 Omega, 1 A1, 2 OO, 3 B1, 4 B2
  if (hi[2] == 0.0f) {
    st.sdP = 0.0f;
    st.sdP_d = 0.0;
    return;
  }
  if (PREC == SEP_PREC_FP64MERGE) {
    const double OO = (double)hi[2] + lo[2], B1 = (double)hi[3] + lo[3];
    const double var = (double)Kf + B1 / OO + (double)dark;
    st.sdP_d = var > 0.0 ? sqrt(var) : 0.0;
    st.sdP = (float)st.sdP_d;
    return;
  }
  const float corr = __fdiv_rn(__fadd_rn(hi[3], lo[3]), __fadd_rn(hi[2], lo[2]));
  float s, e;
  two_sum(Kf, corr, s, e);
  const float var = __fadd_rn(s, __fadd_rn(e, dark));
  st.sdP = var > 0.0f ? __fsqrt_rn(var) : 0.0f;
  st.sdP_d = st.sdP;
}

// The reported (and, for the Poisson model, clipping) deviation becomes the
// Poisson one.
__device__ __forceinline__ void use_poisson(Bcast& st) {
  st.sd = st.sdP;
  st.sd_d = st.sdP_d;
}

// Chauvenet's cut-off for a set of n entries (Eq. 20): sqrt(2 ln(n / sqrt(2 pi))),
// n > 2 (FP32 library logarithm and square root).
__device__ __forceinline__ float chauvenet_k(float n) {
  return sqrtf(2.0f * logf(n * 0.3989422804014327f));
}

template <int PREC>
__device__ __forceinline__ void clip_step(Bcast& st, float n_set, const float (&h)[6], const float (&l)[6], float Kf,
                                          float Ln, float Hn, int n_iter, float k, bool have_moments = false,
                                          int cutoff = SEP_CUTOFF_FIXED, int model = SEP_ERROR_AZIMUTHAL,
                                          float dark = 0.0f) {
  if (st.steps >= 0 && n_set == st.n_cur) {
    if (model == SEP_ERROR_HYBRID) use_poisson(st);   // the final set's Poisson deviation
    st.done = 1;
    return;
  }
  st.n_cur = n_set;
  st.L = Ln;
  st.H = Hn;
  if (!have_moments) finalise<PREC>(Kf, h, l, st);
  if (model != SEP_ERROR_AZIMUTHAL) {
    poisson_sd<PREC>(Kf, h, l, dark, st);
    if (model == SEP_ERROR_POISSON) use_poisson(st);
  }
  st.steps += 1;
  // (Chauvenet: a set of two or fewer is not clipped, the loop ends here)
  if (st.steps >= n_iter || (cutoff == SEP_CUTOFF_CHAUVENET && n_set <= 2.0f)) {
    if (model == SEP_ERROR_HYBRID) use_poisson(st);
    st.done = 1;
    return;
  }
  if (cutoff == SEP_CUTOFF_CHAUVENET) k = chauvenet_k(n_set);
  float L2 = Ln, H2 = Hn;
  clip_bounds<PREC>(st, k, L2, H2);
  st.Ln = L2;
  st.Hn = H2;
  st.Kf = choose_shift(st.mu_hi, st.sd);
}

// A pass's totals as (count, Omega, A1, OO, B1, B2) pairs (every lane).
template <int MODE>
__device__ __forceinline__ void unpack_totals(const float* th, const float* tl, float& n_set, float (&h)[6],
                                              float (&l)[6]) {
#pragma unroll
  for (int v = 0; v < 6; ++v) h[v] = l[v] = 0.0f;
  if (MODE == MODE_CLASS) {
    // class counts are exact integers; their weighted sums are exact in FP32
    const uint32_t p01 = __float_as_uint(th[3]), p23 = __float_as_uint(th[4]);
    const float n0 = (float)(p01 & 0xffffu), n1 = (float)(p01 >> 16);
    const float n2 = (float)(p23 & 0xffffu), n3 = (float)(p23 >> 16);
    n_set = n0 + n1 + n2 + n3;
    h[0] = n0 + 0.75f * n1 + 0.5f * n2 + 0.25f * n3;
    h[2] = n0 + 0.5625f * n1 + 0.25f * n2 + 0.0625f * n3;
    h[1] = th[0]; l[1] = tl[0];
    h[3] = th[1]; l[3] = tl[1];
    h[4] = th[2]; l[4] = tl[2];
  } else if (MODE == MODE_UNIT) {
    n_set = (float)__float_as_uint(th[2]);
    h[0] = h[2] = n_set;
    h[1] = h[3] = th[0]; l[1] = l[3] = tl[0];
    h[4] = th[1]; l[4] = tl[1];
  } else {
    n_set = (float)__float_as_uint(th[5]);
#pragma unroll
    for (int v = 0; v < 5; ++v) { h[v] = th[v]; l[v] = tl[v]; }
  }
}

// ---------------------------------------------------------------------------
// Clip by tail replay, one warp per bin and frame (the plain path and the
// surrogate's record and inference variants).
//
// Every set of the clip loop is a value interval and the intervals are
// nested (Eq. 19 is cumulative). An interval C = [cLo, cHi] that lies inside
// every interval the loop has still to visit contributes the same entries,
// hence the same sums, to each remaining step; only the entries outside C
// (the tail) need to be tested again. Per bin and frame:
//   pass A  plain FP32 moments of the full set, used only to place C
//           kCoreMargin deviations inside the first clip interval;
//   pass B  one scan of the row: core entries are summed (in the call's
//           precision, about a shift K), every other valid entry is listed
//           in its lane's tail slots (value, entry index and class);
//   replay  the loop of Eq. 19 from the full set: the sums of a step are the
//           core sums plus a pass over the tail, finalised exactly as a full
//           pass would be (same set, sums in another order). When a new
//           interval no longer contains C, C is placed inside it and pass B
//           runs again; when a lane's tail slots overflow, the remaining
//           steps run as full passes.
// The kept-pixel marks come from the tail alone when the threshold lies at
// or above C (no core entry can exceed it), else from a scan of the row.
//
// A warp owns its item from the first load to the marks. The row is read
// straight from the staged frame (slot = entry, so a bin's values are one
// contiguous run: 16-byte loads, several in flight per lane); only the tail
// lives in shared memory, so many items fit an SM. Every total is a warp
// butterfly, which leaves bit-identical totals on all lanes (addition, and
// the error-free pair sum, are commutative), so every lane evaluates each
// clip step itself: no lane waits for another, and the warps of a CTA
// (other frames of the same bin) meet only between units of work.
constexpr float kCoreMargin = 1.0f;   // core margin inside the clip interval, in deviations
constexpr int kLoadsAhead = 4;        // 16-byte loads in flight per lane in a scan of the row
constexpr int kWarpsPerSM = 16;       // resident warps per SM the register budget is sized for

// One item's row: entry e's staged value at v4[e / 4] (padding slots NaN).
struct Row {
  const float4* v4;
};

// Scan of every step-th 16-byte group of [q0, q1) of a row by one lane of a
// warp: fn(v, q) for each of the lane's groups, kLoadsAhead loads issued
// before their use (groups past q1 are not loaded; fn is not called for
// them).
template <class F>
__device__ __forceinline__ void scan_row(const Row& row, int q0, int q1, int lane, F&& fn, int step = 1) {
  for (int q = q0 + lane * step; q < q1; q += 32 * step * kLoadsAhead) {
    float4 v[kLoadsAhead];
#pragma unroll
    for (int k = 0; k < kLoadsAhead; ++k)
      if (q + 32 * step * k < q1) v[k] = __ldg(row.v4 + q + 32 * step * k);
#pragma unroll
    for (int k = 0; k < kLoadsAhead; ++k)
      if (q + 32 * step * k < q1) fn(v[k], q + 32 * step * k);
  }
}

// Totals over the warp of NF per-lane sums (value s - c) as pairs
// hi + lo, identical on every lane: plain FP32 in PLAIN, doubles in
// FP64MERGE, error-free FP32 pairs otherwise.
template <int NF, int PREC>
__device__ __forceinline__ void warp_sum(const float (&s)[NF], const float (&c)[NF], float (&hi)[NF],
                                         float (&lo)[NF]) {
#pragma unroll
  for (int v = 0; v < NF; ++v) {
    if (PREC == SEP_PREC_PLAIN) {
      float x = s[v];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x = __fadd_rn(x, __shfl_xor_sync(0xffffffffu, x, o));
      hi[v] = x;
      lo[v] = 0.0f;
    } else if (PREC == SEP_PREC_FP64MERGE) {
      double t = (double)s[v] - (double)c[v];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      hi[v] = (float)t;
      lo[v] = (float)(t - (double)hi[v]);
    } else {
      float hs = s[v], hc = c[v];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float so = __shfl_xor_sync(0xffffffffu, hs, o);
        const float co = __shfl_xor_sync(0xffffffffu, hc, o);
        pair_add(hs, hc, so, co);
      }
      two_sum(hs, -hc, hi[v], lo[v]);
    }
  }
}

// Totals of a pass in the layout unpack_totals reads: NF float pairs, then
// the NI integer totals as raw bits.
template <int MODE, int PREC>
__device__ __forceinline__ void warp_totals(const float (&ss)[Sums<MODE>::NF], const float (&cc)[Sums<MODE>::NF],
                                            const uint32_t (&ci)[Sums<MODE>::NI], float& n_set, float (&h)[6],
                                            float (&l)[6]) {
  constexpr int NF = Sums<MODE>::NF, NI = Sums<MODE>::NI;
  float hi[NF], lo[NF];
  warp_sum<NF, PREC>(ss, cc, hi, lo);
  float th[NF + NI], tl[NF + NI];
#pragma unroll
  for (int v = 0; v < NF; ++v) {
    th[v] = hi[v];
    tl[v] = lo[v];
  }
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    th[NF + i] = __uint_as_float(__reduce_add_sync(0xffffffffu, ci[i]));
    tl[NF + i] = 0.0f;
  }
  unpack_totals<MODE>(th, tl, n_set, h, l);
}

// Pass A (one lane's share): plain FP32 sums about 0 of the finite entries
// of every `step`-th group of 4 (a sample of a long row: they only place
// the core), in the layout unpack_totals reads (per-lane values).
template <int MODE>
__device__ __forceinline__ void lane_full_sums(const Row& row, const float* wts, const int (&ge)[4],
                                               int lane, int step, float (&ss)[Sums<MODE>::NF],
                                               uint32_t (&ci)[Sums<MODE>::NI]) {
  constexpr int NF = Sums<MODE>::NF, NI = Sums<MODE>::NI;
#pragma unroll
  for (int v = 0; v < NF; ++v) ss[v] = 0.0f;
#pragma unroll
  for (int i = 0; i < NI; ++i) ci[i] = 0u;
  if (MODE == MODE_CLASS || MODE == MODE_UNIT) {
    constexpr int NCLS = MODE == MODE_CLASS ? 4 : 1;
    int lo = 0;
#pragma unroll 1
    for (int cls = 0; cls < NCLS; ++cls) {
      const int hi = ge[cls];
      uint32_t cnt = 0;
      float s1 = 0.0f, s2 = 0.0f;
      scan_row(row, lo >> 2, hi >> 2, lane, [&](const float4& v4, int) {
        const float xs[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (fabsf(xs[j]) <= FLT_MAX) {   // finite (padding slots hold NaN)
            ++cnt;
            s1 = __fadd_rn(s1, xs[j]);
            s2 = __fmaf_rn(xs[j], xs[j], s2);
          }
        }
      }, step);
      if (MODE == MODE_CLASS) {
        const float w = 1.0f - 0.25f * (float)cls, w2 = w * w;
        const uint32_t pk = cnt << (16 * (cls & 1));
        if (cls < 2) ci[0] += pk;
        else ci[NI - 1] += pk;
        ss[0] = fmaf(w, s1, ss[0]);
        ss[1] = fmaf(w2, s1, ss[1]);
        ss[2] = fmaf(w2, s2, ss[2]);
      } else {
        ci[0] = cnt;
        ss[0] = s1;
        ss[1] = s2;
      }
      lo = hi;
    }
  } else {
    uint32_t cnt = 0;
    float om = 0.0f, a1 = 0.0f, oo = 0.0f, b1 = 0.0f, b2 = 0.0f;
    scan_row(row, 0, ge[3] >> 2, lane, [&](const float4& v4, int q) {
      const float xs[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float w = wts[4 * q + j];
        if (w != 0.0f && fabsf(xs[j]) <= FLT_MAX) {
          const float w2 = __fmul_rn(w, w), w2d = __fmul_rn(w2, xs[j]);
          ++cnt;
          om = __fadd_rn(om, w);
          a1 = __fmaf_rn(w, xs[j], a1);
          oo = __fadd_rn(oo, w2);
          b1 = __fadd_rn(b1, w2d);
          b2 = __fmaf_rn(w2d, xs[j], b2);
        }
      }
    }, step);
    ci[0] = cnt;
    ss[0] = om; ss[1] = a1; ss[2] = oo; ss[3] = b1; ss[4] = b2;
  }
}

// Pass B (one lane's share): sums about Kf of the entries inside
// [cLo, cHi] (the layout unpack_totals reads); every other valid entry goes to the
// lane's tail: slot k at tl[32 k] = (value bits, entry index | class <<
// 16), written for every entry and kept only for the tail (m counts the
// slots kept, so the branch-free store of a core entry is overwritten).
// Returns false when a group of 4 entries found fewer than 4 of the tcap
// slots left (the sums are then incomplete).
template <int MODE, bool KAHAN>
__device__ __forceinline__ bool lane_core_sums(const Row& row, const float* wts, const int (&ge)[4], int lane,
                                               float cLo, float cHi, float Kf, uint2* tl, int tcap, int& m,
                                               float (&ss)[Sums<MODE>::NF], float (&cc)[Sums<MODE>::NF],
                                               uint32_t (&ci)[Sums<MODE>::NI]) {
  constexpr int NF = Sums<MODE>::NF, NI = Sums<MODE>::NI;
#pragma unroll
  for (int v = 0; v < NF; ++v) ss[v] = cc[v] = 0.0f;
#pragma unroll
  for (int i = 0; i < NI; ++i) ci[i] = 0u;
  m = 0;
  bool fit = true;
  if (MODE == MODE_CLASS || MODE == MODE_UNIT) {
    constexpr int NCLS = MODE == MODE_CLASS ? 4 : 1;
    int lo = 0;
#pragma unroll 1
    for (int cls = 0; cls < NCLS; ++cls) {
      const int hi = ge[cls];
      uint32_t cnt = 0;
      Acc<KAHAN> a1, a2;
      scan_row(row, lo >> 2, hi >> 2, lane, [&](const float4& v4, int q) {
        if (m + 4 > tcap) fit = false;
        if (!fit) return;
        const float xs[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const bool core = xs[j] >= cLo && xs[j] <= cHi;
          if (core) {
            const float d = __fsub_rn(xs[j], Kf);
            ++cnt;
            a1.add(d);
            a2.add_prod(d, d);
          }
          tl[32 * m] = make_uint2(__float_as_uint(xs[j]), (uint32_t)(4 * q + j) | ((uint32_t)cls << 16));
          m += (!core && xs[j] == xs[j]) ? 1 : 0;
        }
      });
      if (!fit) return false;
      const float s1 = a1.val(), s2 = a2.val();
      if (MODE == MODE_CLASS) {
        const float w = 1.0f - 0.25f * (float)cls, w2 = w * w;
        const uint32_t pk = cnt << (16 * (cls & 1));
        if (cls < 2) ci[0] += pk;
        else ci[NI - 1] += pk;
        if (KAHAN) {
          Acc<true> t0, t1, t2;
          t0.s = ss[0]; t0.c = cc[0]; t0.add(__fmul_rn(w, s1)); ss[0] = t0.s; cc[0] = t0.c;
          t1.s = ss[1]; t1.c = cc[1]; t1.add(__fmul_rn(w2, s1)); ss[1] = t1.s; cc[1] = t1.c;
          t2.s = ss[2]; t2.c = cc[2]; t2.add(__fmul_rn(w2, s2)); ss[2] = t2.s; cc[2] = t2.c;
        } else {
          ss[0] = fmaf(w, s1, ss[0]);
          ss[1] = fmaf(w2, s1, ss[1]);
          ss[2] = fmaf(w2, s2, ss[2]);
        }
      } else {
        ci[0] = cnt;
        ss[0] = a1.s; cc[0] = a1.c; ss[1] = a2.s; cc[1] = a2.c;
      }
      lo = hi;
    }
  } else {
    uint32_t cnt = 0;
    Acc<KAHAN> om, a1, oo, b1, b2;
    scan_row(row, 0, ge[3] >> 2, lane, [&](const float4& v4, int q) {
      if (m + 4 > tcap) fit = false;
      if (!fit) return;
      const float xs[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float w = wts[4 * q + j];
        if (w == 0.0f) continue;
        if (xs[j] >= cLo && xs[j] <= cHi) {
          const float d = __fsub_rn(xs[j], Kf);
          const float w2 = __fmul_rn(w, w);
          const float w2d = __fmul_rn(w2, d);
          ++cnt;
          om.add(w);
          a1.add(__fmul_rn(w, d));
          oo.add(w2);
          b1.add(w2d);
          b2.add_prod(w2d, d);
        } else if (xs[j] == xs[j]) {
          tl[32 * m] = make_uint2(__float_as_uint(xs[j]), (uint32_t)(4 * q + j));
          ++m;
        }
      }
    });
    if (!fit) return false;
    ci[0] = cnt;
    ss[0] = om.s; cc[0] = om.c; ss[1] = a1.s; cc[1] = a1.c; ss[2] = oo.s; cc[2] = oo.c;
    ss[3] = b1.s; cc[3] = b1.c; ss[4] = b2.s; cc[4] = b2.c;
  }
  return true;
}

// One lane's share of a full pass over [Ln, Hn] about Kf (the layout
// unpack_totals reads), read from the staged row.
template <int MODE, bool KAHAN>
__device__ __noinline__ void lane_range_sums(const Row& row, const float* wts, const int (&ge)[4],
                                                int lane, float Ln, float Hn, float Kf,
                                                float (&ss)[Sums<MODE>::NF], float (&cc)[Sums<MODE>::NF],
                                                uint32_t (&ci)[Sums<MODE>::NI]) {
  constexpr int NF = Sums<MODE>::NF, NI = Sums<MODE>::NI;
#pragma unroll
  for (int v = 0; v < NF; ++v) ss[v] = cc[v] = 0.0f;
#pragma unroll
  for (int i = 0; i < NI; ++i) ci[i] = 0u;
  if (MODE == MODE_CLASS || MODE == MODE_UNIT) {
    constexpr int NCLS = MODE == MODE_CLASS ? 4 : 1;
    int lo = 0;
#pragma unroll 1
    for (int cls = 0; cls < NCLS; ++cls) {
      const int hi = ge[cls];
      uint32_t cnt = 0;
      Acc<KAHAN> a1, a2;
      scan_row(row, lo >> 2, hi >> 2, lane, [&](const float4& v4, int) {
        const float xs[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (xs[j] >= Ln && xs[j] <= Hn) {
            const float d = __fsub_rn(xs[j], Kf);
            ++cnt;
            a1.add(d);
            a2.add_prod(d, d);
          }
        }
      });
      const float s1 = a1.val(), s2 = a2.val();
      if (MODE == MODE_CLASS) {
        const float w = 1.0f - 0.25f * (float)cls, w2 = w * w;
        const uint32_t pk = cnt << (16 * (cls & 1));
        if (cls < 2) ci[0] += pk;
        else ci[NI - 1] += pk;
        if (KAHAN) {
          Acc<true> t0, t1, t2;
          t0.s = ss[0]; t0.c = cc[0]; t0.add(__fmul_rn(w, s1)); ss[0] = t0.s; cc[0] = t0.c;
          t1.s = ss[1]; t1.c = cc[1]; t1.add(__fmul_rn(w2, s1)); ss[1] = t1.s; cc[1] = t1.c;
          t2.s = ss[2]; t2.c = cc[2]; t2.add(__fmul_rn(w2, s2)); ss[2] = t2.s; cc[2] = t2.c;
        } else {
          ss[0] = fmaf(w, s1, ss[0]);
          ss[1] = fmaf(w2, s1, ss[1]);
          ss[2] = fmaf(w2, s2, ss[2]);
        }
      } else {
        ci[0] = cnt;
        ss[0] = a1.s; cc[0] = a1.c; ss[1] = a2.s; cc[1] = a2.c;
      }
      lo = hi;
    }
  } else {
    uint32_t cnt = 0;
    Acc<KAHAN> om, a1, oo, b1, b2;
    scan_row(row, 0, ge[3] >> 2, lane, [&](const float4& v4, int q) {
      const float xs[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float w = wts[4 * q + j];
        if (w != 0.0f && xs[j] >= Ln && xs[j] <= Hn) {
          const float d = __fsub_rn(xs[j], Kf);
          const float w2 = __fmul_rn(w, w);
          const float w2d = __fmul_rn(w2, d);
          ++cnt;
          om.add(w);
          a1.add(__fmul_rn(w, d));
          oo.add(w2);
          b1.add(w2d);
          b2.add_prod(w2d, d);
        }
      }
    });
    ci[0] = cnt;
    ss[0] = om.s; cc[0] = om.c; ss[1] = a1.s; cc[1] = a1.c; ss[2] = oo.s; cc[2] = oo.c;
    ss[3] = b1.s; cc[3] = b1.c; ss[4] = b2.s; cc[4] = b2.c;
  }
}

// One lane's tail entries inside [Ln, Hn]: (Omega, A1, OO, B1, B2) about Kf
// and their count (m: the lane's slots).
template <int MODE, bool KAHAN>
__device__ __forceinline__ void lane_tail_sums(const uint2* tl, const float* wts, int m, float Ln, float Hn,
                                               float Kf, float (&ss)[5], float (&cc)[5], uint32_t& cnt) {
  Acc<KAHAN> acc[5];
  cnt = 0;
  for (int k = 0; k < m; ++k) {
    const uint2 t = tl[32 * k];
    const float v = __uint_as_float(t.x);
    if (v >= Ln && v <= Hn) {
      float w;
      if (MODE == MODE_CLASS) w = 1.0f - 0.25f * (float)(t.y >> 16);
      else if (MODE == MODE_UNIT) w = 1.0f;
      else w = wts[t.y & 0xffffu];
      const float d = __fsub_rn(v, Kf);
      const float w2 = __fmul_rn(w, w);
      const float w2d = __fmul_rn(w2, d);
      ++cnt;
      acc[0].add(w);
      acc[1].add(__fmul_rn(w, d));
      acc[2].add(w2);
      acc[3].add(w2d);
      acc[4].add_prod(w2d, d);
    }
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    ss[v] = acc[v].s;
    cc[v] = acc[v].c;
  }
}

// (h, l) += (a, b) for pairs, in the arithmetic of the precision mode.
template <int PREC>
__device__ __forceinline__ void add_pair(float& h, float& l, float a, float b) {
  if (PREC == SEP_PREC_PLAIN) {
    h = __fadd_rn(h, a);
  } else if (PREC == SEP_PREC_FP64MERGE) {
    const double t = ((double)h + (double)l) + ((double)a + (double)b);
    h = (float)t;
    l = (float)(t - (double)h);
  } else {
    float s, e;
    two_sum(h, a, s, e);
    e = __fadd_rn(e, __fadd_rn(l, b));
    two_sum(s, e, h, l);
  }
}

// ---- surrogate (no counterpart in the paper): features and inference ----
//
// Features of an item: 0 log(n) / 8 with n the valid entries of pass A's
// sample (every step-th group of 4 entries) times step, 1 Omega / n over
// that sample, 2 clamp(m1 / s1, -20, 20) / 4 with m1, s1 the sample's mean
// and Eq. 13 deviation; then, over a stratified subsample of at most 128 of
// the row's valid entries (sketch_element), 3 the share with z = (v - m1) /
// s1 >= 4 and 4 .. 19 the order statistics of z at ranks floor((j + 1/2)
// n' / 16) (n' the subsample's size; z clamped to [-4, 12]). The subsample
// is one 16-byte load per lane and four values a lane, sorted across the
// warp by a bitonic network.
constexpr float kSurrMargin = 0.5f;   // core margin inside the predicted final interval, in deviations

// Entry of the row behind sketch element s (0 .. 127) of a row whose first
// G groups of 4 hold its weighted entries: every entry when the row has at
// most 128 of them, else one entry of group floor(s G / 128) (-1: none).
__device__ __forceinline__ int sketch_element(int s, int G) {
  if (4 * G <= 128) return s < 4 * G ? s : -1;
  return 4 * (int)(((long long)s * G) >> 7) + (s & 3);
}

template <int MODE>
__device__ __forceinline__ void sample_features(const Row& row, const float* wts, const int (&ge)[4], int lane,
                                                int step, float n_s, float om_s, float m1, float s1,
                                                float (&feat)[kIn]) {
  const int G = ge[3] >> 2;
  // element s = 32 r + lane of the sketch in x[r] (+inf where none)
  float x[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int e = sketch_element(32 * r + lane, G);
    float v = INFINITY;
    if (e >= 0) {
      const float4 q = __ldg(row.v4 + (e >> 2));
      const float c = (e & 3) == 0 ? q.x : ((e & 3) == 1 ? q.y : ((e & 3) == 2 ? q.z : q.w));
      const bool ok = fabsf(c) <= FLT_MAX && (MODE != MODE_ENTRY || wts[e] != 0.0f);
      v = ok ? c : INFINITY;
    }
    x[r] = v;
  }
  // ascending bitonic sort of the 128 elements (index 32 r + lane)
#pragma unroll
  for (int k = 2; k <= 128; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      float y[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) y[r] = j >= 32 ? x[r ^ (j >> 5)] : __shfl_xor_sync(0xffffffffu, x[r], j);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int e = 32 * r + lane;
        const bool up = (e & k) == 0, low = (e & j) == 0;
        x[r] = (low == up) ? fminf(x[r], y[r]) : fmaxf(x[r], y[r]);
      }
    }
  }
  int nv = 0, hi4 = 0;
  const float z4 = fmaf(4.0f, s1, m1);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    nv += __popc(__ballot_sync(0xffffffffu, x[r] <= FLT_MAX));
    hi4 += __popc(__ballot_sync(0xffffffffu, x[r] <= FLT_MAX && x[r] >= z4));
  }
  const float inv = s1 > 0.0f ? 1.0f / s1 : 0.0f;
  const float n_est = n_s * (float)step;
  feat[0] = n_est > 0.0f ? logf(n_est) * 0.125f : 0.0f;
  feat[1] = n_s > 0.0f ? om_s / n_s : 0.0f;
  feat[2] = s1 > 0.0f ? fminf(fmaxf(m1 / s1, -20.0f), 20.0f) * 0.25f : 0.0f;
  feat[3] = nv > 0 ? (float)hi4 / (float)nv : 0.0f;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int p = ((2 * j + 1) * nv) >> 5;   // floor((j + 1/2) nv / 16)
    const int r = p >> 5;
    const float mine = r == 0 ? x[0] : (r == 1 ? x[1] : (r == 2 ? x[2] : x[3]));
    const float q = __shfl_sync(0xffffffffu, mine, p & 31);
    feat[4 + j] = nv > 0 ? fminf(fmaxf(__fmul_rn(__fsub_rn(q, m1), inv), -4.0f), 12.0f) : 0.0f;
  }
}

// The network on one warp (weights BF16 with W1 and W2 input-major, FP32
// arithmetic; W and nm in shared memory): lane l computes hidden units l and l + 32 of each layer, so
// the warp reads consecutive weights; every lane returns the de-normalised
// outputs (mean offset, log-deviation ratio).
__device__ __forceinline__ void warp_mlp(const __nv_bfloat16* W, const float* nm, const float (&feat)[kIn], int lane,
                                         float& u0, float& u1) {
  float a1[2] = {__bfloat162float(W[kB1 + lane]), __bfloat162float(W[kB1 + lane + 32])};
#pragma unroll
  for (int k = 0; k < kIn; ++k) {
    const float xk = (feat[k] - nm[k]) / nm[kIn + k];
    a1[0] = fmaf(__bfloat162float(W[kW1 + k * kH + lane]), xk, a1[0]);
    a1[1] = fmaf(__bfloat162float(W[kW1 + k * kH + lane + 32]), xk, a1[1]);
  }
  const float h1[2] = {gelu_f(a1[0]), gelu_f(a1[1])};
  // layer 2: every input unit comes from the lane that holds it
  float a2[2] = {__bfloat162float(W[kB2 + lane]), __bfloat162float(W[kB2 + lane + 32])};
#pragma unroll 4
  for (int k = 0; k < kH; ++k) {
    const float hk = __shfl_sync(0xffffffffu, h1[k >> 5], k & 31);
    a2[0] = fmaf(__bfloat162float(W[kW2 + k * kH + lane]), hk, a2[0]);
    a2[1] = fmaf(__bfloat162float(W[kW2 + k * kH + lane + 32]), hk, a2[1]);
  }
  const float h2a = gelu_f(a2[0]), h2b = gelu_f(a2[1]);
  // layer 3: two sums over the warp
  float y0 = __bfloat162float(W[kW3 + lane]) * h2a + __bfloat162float(W[kW3 + lane + 32]) * h2b;
  float y1 = __bfloat162float(W[kW3 + kH + lane]) * h2a + __bfloat162float(W[kW3 + kH + lane + 32]) * h2b;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    y0 += __shfl_xor_sync(0xffffffffu, y0, o);
    y1 += __shfl_xor_sync(0xffffffffu, y1, o);
  }
  u0 = (y0 + __bfloat162float(W[kB3])) * nm[2 * kIn + 2] + nm[2 * kIn];
  u1 = (y1 + __bfloat162float(W[kB3 + 1])) * nm[2 * kIn + 3] + nm[2 * kIn + 1];
}

__device__ __forceinline__ void mark_pixel(uint32_t* bm, const int32_t* cpix, int64_t e) {
  const int32_t i = __ldg(cpix + e);
  if (i >= 0) atomicOr(bm + (i >> 5), 1u << (i & 31));
}

// The first clip interval [lo, hi] from plain FP32 totals of the full set
// about 0 (h: Omega, A1, OO, B1, B2; the formulas of finalise, poisson_sd
// and clip_step in single rounding); only the core is placed with it.
__device__ __forceinline__ void approx_interval(float n_set, const float (&h)[6], float k, int cutoff, int model,
                                                float dark, float& lo, float& hi, float& mu, float& sd) {
  lo = -FLT_MAX;
  hi = FLT_MAX;
  mu = sd = 0.0f;
  if (h[0] == 0.0f || h[2] == 0.0f) return;
  mu = __fdiv_rn(h[1], h[0]);
  const float vv = __fadd_rn(__fsub_rn(h[4], __fmul_rn(2.0f * mu, h[3])), __fmul_rn(__fmul_rn(mu, mu), h[2]));
  sd = vv > 0.0f ? __fsqrt_rn(__fdiv_rn(vv, h[2])) : 0.0f;
  if (model == SEP_ERROR_POISSON) {
    const float var = __fadd_rn(__fdiv_rn(h[3], h[2]), dark);
    sd = var > 0.0f ? __fsqrt_rn(var) : 0.0f;
  }
  if (cutoff == SEP_CUTOFF_CHAUVENET) {
    if (n_set <= 2.0f) return;
    k = chauvenet_k(n_set);
  }
  lo = __fsub_rn(mu, __fmul_rn(k, sd));
  hi = __fadd_rn(mu, __fmul_rn(k, sd));
}

// SURR 0: the plain method; 1: also record the surrogate's features and
// training targets; 2: place the first core from the surrogate's prediction
// of the final interval (the replay is the same exact loop).
template <int MODE, int PREC, int kWarps, int SURR>
__global__ void __launch_bounds__(32 * kWarps, kWarpsPerSM / kWarps) k_clip_warp(ClipArgs a) {
  constexpr bool KAHAN = PREC == SEP_PREC_KAHAN;
  // the tail's share of a step is merged over the lanes in FP32 except
  // where the per-lane sums are compensated (KAHAN) or merged in FP64
  constexpr int TPREC = PREC == SEP_PREC_DWORD ? SEP_PREC_PLAIN : PREC;
  constexpr int NF = Sums<MODE>::NF, NI = Sums<MODE>::NI;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // [weights (MODE_ENTRY), shared by the warps] then per warp its tail
  // (8-byte slots, slot k of lane l at 32 k + l)
  const int capr = MODE == MODE_ENTRY ? (a.cap + 3) & ~3 : 0;
  float* wts = reinterpret_cast<float*>(smem_raw);
  uint2* tail = reinterpret_cast<uint2*>(wts + capr) + (size_t)warp * (32 * a.tcap) + lane;
  // with inference (SURR 2) the network's normalisation and BF16 weights
  // follow the tails, copied once per CTA (read by every item, they would
  // otherwise compete with the streamed rows for the L1 cache)
  float* nm_s = reinterpret_cast<float*>(reinterpret_cast<uint2*>(wts + capr) + (size_t)kWarps * 32 * a.tcap);
  __nv_bfloat16* w_s = reinterpret_cast<__nv_bfloat16*>(nm_s + kNNorm);
  (void)w_s;
  if (SURR == 2) {
    for (int i = threadIdx.x; i < kNParams; i += 32 * kWarps) w_s[i] = a.mlp_w[i];
    for (int i = threadIdx.x; i < kNNorm; i += 32 * kWarps) nm_s[i] = __ldg(a.mlp_norm + i);
    __syncthreads();
  }

  // optional counters (added by lane 0 as they occur): items, pass B
  // scans, overflows, replay steps, tail entries listed, items marked from
  // the tail, full passes
  auto stat = [&](int i, unsigned v) {
    if (a.clip_stats && lane == 0 && v) atomicAdd(a.clip_stats + i, (unsigned long long)v);
  };
  unsigned long long su[2] = {0, 0};   // surrogate: items whose predicted core held / that re-placed it

  // Units of work: a bin of this launch (in the launch's order, longest rows
  // first) and a group of frames_per_cta frames, x fastest. A persistent
  // launch (a.queue set) sizes its grid to the resident CTAs and every CTA
  // takes the next unit from the queue counter until none is left; else
  // CTA (x, y) runs unit y * gridDim.x + x alone.
  __shared__ int unit_s;
  for (int it = 0;; ++it) {
    int unit;
    if (a.queue) {
      if (threadIdx.x == 0) unit_s = atomicAdd(a.queue, 1);
      __syncthreads();
      unit = unit_s;
    } else {
      unit = it == 0 ? (int)(blockIdx.y * gridDim.x + blockIdx.x) : a.units;
    }
    if (unit >= a.units) break;
    const int ux = unit % a.units_x;
    const int b = a.bin_list ? __ldg(a.bin_list + ux) : ux;
    const int f0 = (unit / a.units_x) * a.frames_per_cta;
    const int f1 = min(f0 + a.frames_per_cta, a.n_frames);
    const int r0 = __ldg(a.rowptr + b);
    const int n = __ldg(a.rowptr + b + 1) - r0;      // multiple of 4
    const int nq = n >> 2;
    int ge[4];   // end of coefficient class 0..3 in the row; weight-0 carriers follow
#pragma unroll
    for (int c = 0; c < 4; ++c) ge[c] = __ldg(a.grp + 4 * b + c);

    if (MODE == MODE_ENTRY) {
      for (int e = threadIdx.x; e < n; e += 32 * kWarps) {
        const uint32_t u = __ldg(a.ent + r0 + e);
        wts[e] = (u & (kZero | kPad)) ? 0.0f : __ldg(a.w + r0 + e);
      }
      __syncthreads();
    }

    for (int f = f0 + warp; f < f1; f += kWarps) {
      // this item's values: entry e of the row at slot r0 + e of the staged frame
      const Row row{reinterpret_cast<const float4*>(a.stage + (int64_t)f * a.npos + r0)};
      const int64_t o = (a.orow ? a.orow[f] : (int64_t)f * a.nbins) + b;
      stat(0, 1);
      // ------------- pass A: where to place the core -------------
      float cLo, cHi, K;
      float pLo = 0.0f, pHi = 0.0f, pK = 0.0f;   // SURR 2: the plain placement, for a retry
      float feat[kIn], m1 = 0.0f, s1 = 0.0f;
      (void)feat;
      {
        float ss[NF], cz[NF];
        uint32_t ci[NI];
        // (rows of 2048 entries and more: every 4th group of 4, 512 and more:
        // every 2nd)
        const int step = nq >= 512 ? 4 : (nq >= 128 ? 2 : 1);
        lane_full_sums<MODE>(row, wts, ge, lane, step, ss, ci);
#pragma unroll
        for (int v = 0; v < NF; ++v) cz[v] = 0.0f;
        float n_set, h[6], l[6], lo, hi, mu, sd;
        warp_totals<MODE, SEP_PREC_PLAIN>(ss, cz, ci, n_set, h, l);
        approx_interval(n_set * (float)step, h, a.k_clip, a.cutoff, a.error_model, a.dark_var, lo, hi, mu, sd);
        const float mg = __fmul_rn(kCoreMargin, sd);
        cLo = __fadd_rn(lo, mg);
        cHi = __fsub_rn(hi, mg);
        K = choose_shift(mu, sd);
        if (SURR != 0) {
          m1 = mu;
          s1 = sd;
          sample_features<MODE>(row, wts, ge, lane, step, n_set, h[0], m1, s1, feat);
        }
        if (SURR == 2) {
          // the predicted final interval, and the core half a deviation inside it
          pLo = cLo;
          pHi = cHi;
          pK = K;
          float u0, u1;
          warp_mlp(w_s, nm_s, feat, lane, u0, u1);
          const float mh = fmaf(s1, u0, m1), sh = s1 * expf(fminf(u1, 20.0f));
          if (s1 > 0.0f && sh > 0.0f && fabsf(mh) <= FLT_MAX && sh <= FLT_MAX) {
            const float half = __fmul_rn(a.k_clip, sh), mgs = __fmul_rn(kSurrMargin, sh);
            cLo = __fadd_rn(__fsub_rn(mh, half), mgs);
            cHi = __fsub_rn(__fadd_rn(mh, half), mgs);
          }
        }
      }
      // ------------- the loop of Eq. 19: replay on core + tail, or full passes -------------
      Bcast st;
      st.Ln = -FLT_MAX;
      st.Hn = FLT_MAX;
      st.L = -FLT_MAX;
      st.H = FLT_MAX;
      st.n_cur = -1.0f;
      st.steps = -1;
      st.done = 0;
      st.Kf = K;
      bool ovf = false, scan = true, retried = SURR != 2;
      int m = 0, scans = 0;
      float cn = 0.0f, ch[6], cl[6];
      for (;;) {
        const float Ln = st.Ln, Hn = st.Hn;
        if (scan) {
          // pass B: the core's sums and the tail, for the core placed last
          float ss[NF], cc[NF];
          uint32_t ci[NI];
          const bool fit =
              lane_core_sums<MODE, KAHAN>(row, wts, ge, lane, cLo, cHi, K, tail, a.tcap, m, ss, cc, ci);
          ovf = __any_sync(0xffffffffu, !fit);
          ++scans;
          if (a.clip_stats) {
            const unsigned listed = __reduce_add_sync(0xffffffffu, (unsigned)m);
            stat(1, 1);
            stat(2, ovf ? 1 : 0);
            stat(4, listed);
          }
          if (!retried) {
            // first pass B only (the plain placement is inside the first
            // interval, not necessarily inside a later one): when the
            // predicted core left more entries outside it than the tail holds
            // (a heavy-tailed bin), the plain placement instead
            retried = true;
            if (ovf) {
              cLo = pLo;
              cHi = pHi;
              K = pK;
              continue;
            }
          }
          if (!ovf) warp_totals<MODE, PREC>(ss, cc, ci, cn, ch, cl);
          scan = false;
        }
        float n_set, h[6], l[6], Kf;
        if (!ovf) {
          // a step of the replay: the core sums plus the tail inside [Ln, Hn]
          float ts[5], tc[5], th[5], tl[5];
          uint32_t tn;
          lane_tail_sums<MODE, KAHAN>(tail, wts, m, Ln, Hn, K, ts, tc, tn);
          warp_sum<5, TPREC>(ts, tc, th, tl);
          tn = __reduce_add_sync(0xffffffffu, tn);
          stat(3, 1);
#pragma unroll
          for (int v = 0; v < 5; ++v) {
            h[v] = ch[v];
            l[v] = cl[v];
            add_pair<PREC>(h[v], l[v], th[v], tl[v]);
          }
          h[5] = l[5] = 0.0f;
          n_set = cn + (float)tn;
          Kf = K;
        } else {
          // a tail overflowed: a full pass over [Ln, Hn]
          float ss[NF], cc[NF];
          uint32_t ci[NI];
          Kf = st.Kf;
          lane_range_sums<MODE, KAHAN>(row, wts, ge, lane, Ln, Hn, Kf, ss, cc, ci);
          stat(6, 1);
          warp_totals<MODE, PREC>(ss, cc, ci, n_set, h, l);
        }
        clip_step<PREC>(st, n_set, h, l, Kf, Ln, Hn, a.n_iter, a.k_clip, false, a.cutoff, a.error_model, a.dark_var);
        if (st.done) break;
        if (!ovf && (cLo < st.Ln || cHi > st.Hn)) {
          // the next interval cuts into the core: place it inside and scan again
          const float mg = __fmul_rn(kCoreMargin, st.sd);
          cLo = __fadd_rn(st.Ln, mg);
          cHi = __fsub_rn(st.Hn, mg);
          K = st.Kf;
          scan = true;
        }
      }
      if (lane == 0) {
        a.mean[o] = st.mu_hi;
        a.sigma[o] = st.sd;
        a.count[o] = (int32_t)st.n_cur;
        if (a.bounds) {
          a.bounds[2 * o] = st.L;
          a.bounds[2 * o + 1] = st.H;
        }
        if (a.iters) a.iters[o] = st.steps;
        if (SURR == 1) {
          // training record: the features and the result as normalised targets
          for (int k = 0; k < kIn; ++k) a.rec_feat[o * kIn + k] = feat[k];
          const bool ok = s1 > 0.0f && st.sd > 0.0f && st.n_cur >= 2.0f;
          a.rec_target[o * 2] = ok ? (st.mu_hi - m1) / s1 : __int_as_float(0x7fc00000);
          a.rec_target[o * 2 + 1] = ok ? logf(st.sd / s1) : __int_as_float(0x7fc00000);
        }
      }
      if (SURR == 2) su[(scans == 1 && !ovf) ? 0 : 1] += 1;
      // threshold of sparsification (Section 3) from the final state
      const float thr = pick_threshold<PREC>(st, a.k_pick);
      if (a.thr_out && lane == 0) a.thr_out[o] = thr;
      if (a.bitmap) {
        // kept pixels of this bin: its centre entries whose value exceeds the
        // threshold (only kept pixels touch the pixel table and the bitmap)
        uint32_t* bm = a.bitmap + (int64_t)f * a.words;
        const int32_t* cp = a.cpix + r0;
        // without an overflow and with thr at or above the core, no core entry
        // exceeds thr: the lane's tail, then the weight-0 carriers of the row;
        // else every entry (padding slots hold NaN, never above a threshold)
        const bool from_tail = MODE != MODE_ENTRY && !ovf && thr >= cHi;
        if (from_tail) {
          stat(5, 1);
          for (int k = 0; k < m; ++k)
            if (__uint_as_float(tail[32 * k].x) > thr) mark_pixel(bm, cp, (int64_t)(tail[32 * k].y & 0xffffu));
        }
        scan_row(row, from_tail ? ge[3] >> 2 : 0, nq, lane, [&](const float4& v4, int q) {
          const float xs[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (xs[j] > thr) mark_pixel(bm, cp, 4 * q + j);
        });
      }
      __syncwarp();   // the tail is rewritten by the warp's next frame
    }
    // the next unit rewrites unit_s and the shared row weights
    __syncthreads();
  }
  if (SURR == 2 && a.surr_stats && lane == 0) {
    if (su[0]) atomicAdd(a.surr_stats, su[0]);
    if (su[1]) atomicAdd(a.surr_stats + 1, su[1]);
  }
}

// Opt-in shared memory per block of the current device (cached).
int smem_optin() {
  static int cached[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  if (cached[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0)
      v = 48 * 1024;
    cached[dev] = v;
  }
  return cached[dev];
}

// Multiprocessors of the current device (cached).
int sm_count() {
  static int cached[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  if (cached[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
    cached[dev] = v;
  }
  return cached[dev];
}

template <int MODE, int PREC, int kWarps, int SURR>
cudaError_t launch_warp_t(ClipArgs a, int n_ctas, int mode, cudaStream_t s) {
  // shared memory: the weights of a row (per-entry weights only), then
  // each warp's tail (8 bytes a slot, 32 lanes)
  const long capr = ((long)a.cap + 3) & ~3L;
  const long wbytes = MODE == MODE_ENTRY ? 4 * capr : 0;
  const long budget = (long)smem_optin() - kClipStaticSmem - wbytes -
                     (SURR == 2 ? kNNorm * 4 + ((kNParams * 2 + 15) & ~15) : 0);
  long tcap = clip_tail_slots(a.cap, 32 * kWarps);
  if (kWarps * 256 * tcap > budget) tcap = std::max(0L, budget / (256L * kWarps));
  if (tcap < 5) tcap = 0;   // no room for a tail: every step runs as a full pass
  a.tcap = (int32_t)tcap;
  const size_t smem = (size_t)(wbytes + kWarps * 256 * tcap + (SURR == 2 ? kNNorm * 4 + ((kNParams * 2 + 15) & ~15) : 0));
  auto k = k_clip_warp<MODE, PREC, kWarps, SURR>;
  // resident CTAs per multiprocessor of this instance at this shared-memory
  // size, cached per device (the first query comes before any capture: the
  // attribute pass below asks it). A stale or missing value changes only the
  // grid of a persistent launch, never its results (0: not persistent).
  auto resident = [&]() -> int {
    static int occ_smem[64][8], occ_val[64][8] = {}, occ_next[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    for (int i = 0; i < 8; ++i)
      if (occ_val[dev][i] > 0 && occ_smem[dev][i] == (int)smem) return occ_val[dev][i];
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k, 32 * kWarps, smem) != cudaSuccess) v = 0;
    const int i = occ_next[dev]++ & 7;
    occ_smem[dev][i] = (int)smem;
    occ_val[dev][i] = v;
    return v;
  };
  if (mode != 2) {
    // the attribute only grows: size classes sharing this instance may set
    // it in any order before a capture
    static int attr[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    if ((int)smem > attr[dev]) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      attr[dev] = (int)smem;
    }
    if (mode == 1) {
      (void)resident();
      return cudaSuccess;
    }
  }
  const int gy = (a.n_frames + a.frames_per_cta - 1) / a.frames_per_cta;
  a.units_x = n_ctas;
  a.units = n_ctas * gy;
  dim3 grid(n_ctas, gy);
  if (a.queue) {
    // persistent: as many CTAs as stay resident, while the units outnumber them
    const int per_sm = resident();
    const int64_t slots = (int64_t)sm_count() * per_sm;
    if (per_sm > 0 && slots < a.units) {
      grid = dim3((unsigned)slots, 1);
      cudaError_t e = cudaMemsetAsync(a.queue, 0, sizeof(int32_t), s);
      if (e != cudaSuccess) return e;
    } else {
      a.queue = nullptr;
    }
  }
  k<<<grid, 32 * kWarps, smem, s>>>(a);
  return cudaGetLastError();
}

template <int MODE, int PREC, int SURR = 0>
cudaError_t launch_tail_b(const ClipArgs& a, int n_ctas, int tpb, int mode, cudaStream_t s) {
  switch (tpb) {
    case 32: return launch_warp_t<MODE, PREC, 1, SURR>(a, n_ctas, mode, s);
    case 64: return launch_warp_t<MODE, PREC, 2, SURR>(a, n_ctas, mode, s);
    case 128: return launch_warp_t<MODE, PREC, 4, SURR>(a, n_ctas, mode, s);
    default: return launch_warp_t<MODE, PREC, 8, SURR>(a, n_ctas, mode, s);
  }
}

template <int MODE>
cudaError_t launch_p(const ClipArgs& a, int n_ctas, int tpb, int32_t prec, int mode, cudaStream_t s) {
  // the surrogate modes exist for the default precision only
  if (a.rec_feat) return launch_tail_b<MODE, SEP_PREC_DWORD, 1>(a, n_ctas, tpb, mode, s);
  // (inference: at least 4 warps a CTA share one copy of the weights)
  if (a.mlp_w) return launch_tail_b<MODE, SEP_PREC_DWORD, 2>(a, n_ctas, std::max(tpb, 128), mode, s);
  switch (prec) {
    case SEP_PREC_PLAIN: return launch_tail_b<MODE, SEP_PREC_PLAIN>(a, n_ctas, tpb, mode, s);
    case SEP_PREC_KAHAN: return launch_tail_b<MODE, SEP_PREC_KAHAN>(a, n_ctas, tpb, mode, s);
    case SEP_PREC_FP64MERGE: return launch_tail_b<MODE, SEP_PREC_FP64MERGE>(a, n_ctas, tpb, mode, s);
    default: return launch_tail_b<MODE, SEP_PREC_DWORD>(a, n_ctas, tpb, mode, s);
  }
}

}  // namespace

size_t clip_smem_bytes(int32_t cap, bool weighted) {
  // the shared memory a clip launch cannot do without: the per-entry weights
  // of the longest row (a tail can shrink to nothing)
  size_t smem = weighted ? (size_t)cap * 4 : 0;
  return (smem + 15) & ~(size_t)15;
}

int32_t clip_tail_slots(int32_t cap, int32_t tpb) {
  // per lane of a warp: 1/12 of the row over 32 lanes (a tail holds about
  // 1/20 of a row's entries), plus the 4 slots a pass B keeps free and some
  // room for uneven lanes; a lane that runs out switches its item to full
  // passes (tpb: the block size, one warp per item whatever it is)
  (void)tpb;
  return (int32_t)((cap + 383) / 384) + 6;
}

cudaError_t launch_integrate_clip(const ClipArgs& a, int n_ctas, int tpb, bool split, bool has_norm,
                                  int32_t precision, int mode, cudaStream_t s) {
  if (a.n_frames <= 0 || n_ctas <= 0) return cudaSuccess;
  if (has_norm) return launch_p<MODE_ENTRY>(a, n_ctas, tpb, precision, mode, s);
  return split ? launch_p<MODE_CLASS>(a, n_ctas, tpb, precision, mode, s)
               : launch_p<MODE_UNIT>(a, n_ctas, tpb, precision, mode, s);
}

}  // namespace sep
