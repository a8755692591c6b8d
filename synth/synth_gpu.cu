/*
 * Seeded synthetic frames generated on the GPU: the frame model of synth.c
 * (isotropic background profile + Gaussian Bragg spots + Poisson counting
 * noise, optionally encoded as raw Jungfrau words), with the same
 * Philox4x32-10 streams (Salmon, Moraes, Dror & Shaw, SC 2011) keyed by
 * (seed, frame, pixel/spot, stream), so that large training sets need no
 * host generation. Like synth.c it makes inputs only and holds none of the
 * method's arithmetic. The arithmetic is binary64 as in synth.c; the device
 * math library may round exp / log / pow / cos differently from the host's
 * in the last place, and spot footprints are summed in another order, so a
 * rare pixel may differ by one count from the host generator's.
 *
 * C ABI (device pointers, the caller's stream):
 *   synth_gpu_frames(spec, frame0, n_frames, ped, gain, mask, out, scratch,
 *                    scratch_bytes, stream)
 *   synth_gpu_scratch_bytes(spec, n_frames): scratch a call needs.
 */
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

extern "C" {
typedef struct {
  int32_t rows, cols;
  double cx, cy;
  int32_t bg_kind;
  double bg_scale_lo, bg_scale_hi;
  double bg_clip_lo, bg_clip_hi;
  double hit_rate;
  int32_t spots_min, spots_max;
  double amp_lo, amp_hi;
  int32_t amp_log;
  double sig_lo, sig_hi;
  int32_t out_raw;
  double read_noise_adu;
  uint64_t seed;
} synth_spec;
}

namespace {

constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u, kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;
enum { ST_PIXEL = 0, ST_FRAME = 1, ST_SPOT = 2 };

struct P4 {
  uint32_t x[4];
};

__device__ __forceinline__ P4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(kM0, c0), lo0 = kM0 * c0;
    const uint32_t hi1 = __umulhi(kM1, c2), lo1 = kM1 * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += kW0;
    k1 += kW1;
  }
  P4 o;
  o.x[0] = c0;
  o.x[1] = c1;
  o.x[2] = c2;
  o.x[3] = c3;
  return o;
}

__device__ __forceinline__ P4 draw(const synth_spec& s, uint64_t index, uint32_t frame, uint32_t stream) {
  return philox10((uint32_t)index, (uint32_t)(index >> 32), frame, stream, (uint32_t)s.seed,
                  (uint32_t)(s.seed >> 32));
}

__device__ __forceinline__ double u01(uint32_t x) { return ((double)(x >> 8) + 0.5) * (1.0 / 16777216.0); }

__device__ __forceinline__ double normal2(uint32_t a, uint32_t b) {
  return sqrt(-2.0 * log(u01(a))) * cos(6.283185307179586 * u01(b));
}

struct FramePar {
  double scale, A, r0, rr[3], ra[3], rw[3];
  int hit, nspots;
};

__device__ void frame_params(const synth_spec& s, uint32_t f, double rmax, FramePar& fp) {
  const P4 a = draw(s, 0, f, ST_FRAME), b = draw(s, 1, f, ST_FRAME), c = draw(s, 2, f, ST_FRAME),
           d = draw(s, 3, f, ST_FRAME);
  fp.scale = s.bg_scale_lo * pow(s.bg_scale_hi / s.bg_scale_lo, u01(a.x[0]));
  fp.A = 0.5 + u01(a.x[1]);
  fp.r0 = rmax * (0.2 + 0.4 * u01(a.x[2]));
  for (int m = 0; m < 3; ++m) {
    fp.rr[m] = rmax * (0.15 + 0.7 * u01(b.x[m]));
    fp.ra[m] = 0.2 + 0.8 * u01(c.x[m]);
    fp.rw[m] = rmax * (0.01 + 0.03 * u01(d.x[m]));
  }
  fp.hit = u01(a.x[3]) < s.hit_rate;
  const int span = s.spots_max - s.spots_min + 1;
  fp.nspots = fp.hit ? s.spots_min + (int)(u01(b.x[3]) * span) : 0;
  if (fp.nspots > s.spots_max) fp.nspots = s.spots_max;
}

__device__ double bg_profile(const synth_spec& s, const FramePar& fp, double r) {
  if (s.bg_kind == 0) return 50.0 * exp(-r / 80.0) + 30.0 * exp(-(r - 90.0) * (r - 90.0) / (2.0 * 36.0));
  double v = fp.A * exp(-r / fp.r0);
  for (int m = 0; m < 3; ++m) {
    const double t = (r - fp.rr[m]) / fp.rw[m];
    v += fp.ra[m] * exp(-0.5 * t * t);
  }
  v *= fp.scale;
  if (v < s.bg_clip_lo) v = s.bg_clip_lo;
  if (v > s.bg_clip_hi) v = s.bg_clip_hi;
  return v;
}

// One CTA per frame: the background table on the 1/8-pixel radial grid
// (value and e^-value), then every spot's footprint added into extra.
__global__ void k_frame_setup(synth_spec s, int64_t frame0, double rmax, int64_t ntab, double* tab, float* extra,
                              int32_t* nspots) {
  const int fi = blockIdx.x;
  const uint32_t f = (uint32_t)(frame0 + fi);
  FramePar fp;
  frame_params(s, f, rmax, fp);
  double* tb = tab + (int64_t)fi * 2 * ntab;
  for (int64_t t = threadIdx.x; t < ntab; t += blockDim.x) {
    const double v = bg_profile(s, fp, (double)t / 8.0);
    tb[t] = v;
    tb[ntab + t] = exp(-v);
  }
  if (threadIdx.x == 0) nspots[fi] = fp.nspots;
  const int64_t rows = s.rows, cols = s.cols;
  float* ex = extra + (int64_t)fi * rows * cols;
  for (int j = 0; j < fp.nspots; ++j) {
    const P4 r = draw(s, (uint64_t)j, f, ST_SPOT);
    const float x = (float)(u01(r.x[0]) * (double)cols), y = (float)(u01(r.x[1]) * (double)rows);
    const double u = u01(r.x[2]);
    const double amp = s.amp_log ? s.amp_lo * pow(s.amp_hi / s.amp_lo, u) : s.amp_lo + (s.amp_hi - s.amp_lo) * u;
    const float sg = (float)(s.sig_lo + (s.sig_hi - s.sig_lo) * u01(r.x[3]));
    const double sx = x, sy = y, sgd = sg;
    const int w = (int)ceil(4.0 * sgd) + 1;
    const int64_t r_lo = (int64_t)floor(sy) - w, c_lo = (int64_t)floor(sx) - w;
    const int side = 2 * w + 1;
    for (int k = threadIdx.x; k < side * side; k += blockDim.x) {
      const int64_t rr = r_lo + k / side, cc = c_lo + k % side;
      if (rr < 0 || rr >= rows || cc < 0 || cc >= cols) continue;
      const double dx = (double)cc + 0.5 - sx, dy = (double)rr + 0.5 - sy;
      atomicAdd(ex + rr * cols + cc, (float)(amp * exp(-(dx * dx + dy * dy) / (2.0 * sgd * sgd))));
    }
  }
}

// Poisson count with mean lam (e^-lam = p0) from one uniform u: inversion by
// sequential search below 40, a rounded normal (z) above.
__device__ __forceinline__ double poisson_draw(double lam, double p0, double u, double z) {
  if (lam <= 0.0) return 0.0;
  if (lam < 40.0) {
    double k = 0.0, p = p0, F = p0;
    while (u > F && k < 400.0) {
      k += 1.0;
      p *= lam / k;
      F += p;
    }
    return k;
  }
  const double n = floor(lam + sqrt(lam) * z + 0.5);
  return n < 0.0 ? 0.0 : n;
}

// One thread per pixel and frame.
__global__ void k_pixels(synth_spec s, int64_t frame0, int32_t n_frames, int64_t ntab, const double* tab,
                         const float* extra, const float* ped, const float* gain, const uint8_t* mask, void* out) {
  const int64_t npix = (int64_t)s.rows * s.cols;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int fi = blockIdx.y;
  if (i >= npix || fi >= n_frames) return;
  const uint32_t f = (uint32_t)(frame0 + fi);
  float* outf = s.out_raw ? nullptr : reinterpret_cast<float*>(out) + (int64_t)fi * npix;
  uint16_t* outr = s.out_raw ? reinterpret_cast<uint16_t*>(out) + (int64_t)fi * npix : nullptr;
  if (mask && mask[i]) {
    if (outf) outf[i] = 0.0f;
    else outr[i] = 0;
    return;
  }
  const int64_t rr = i / s.cols, cc = i % s.cols;
  const double dy = (double)rr + 0.5 - s.cy, dx = (double)cc + 0.5 - s.cx;
  int64_t t = (int64_t)(sqrt(dx * dx + dy * dy) * 8.0 + 0.5);
  if (t >= ntab) t = ntab - 1;
  const double* tb = tab + (int64_t)fi * 2 * ntab;
  double lam = tb[t], p0 = tb[ntab + t];
  const float e = extra[(int64_t)fi * npix + i];
  if (e != 0.0f) {
    lam += (double)e;
    p0 = exp(-lam);
  }
  const P4 r = draw(s, (uint64_t)i, f, ST_PIXEL);
  double zp = 0.0;
  if (lam >= 40.0) {
    const P4 r2 = draw(s, (uint64_t)i, f, ST_PIXEL + 8);
    zp = normal2(r2.x[0], r2.x[1]);
  }
  const double n = poisson_draw(lam, p0, u01(r.x[0]), zp);
  if (outf) {
    outf[i] = (float)n;
    return;
  }
  const double p0d = ped[i], g0 = gain[i];
  double adc;
  uint32_t code;
  if (p0d + g0 * n <= 16000.0) {
    adc = p0d + g0 * n + s.read_noise_adu * normal2(r.x[1], r.x[2]);
    code = 0;
  } else if (n <= 9000.0) {
    adc = (double)ped[npix + i] + (double)gain[npix + i] * n;
    code = 1;
  } else {
    adc = (double)ped[2 * npix + i] + (double)gain[2 * npix + i] * n;
    code = 3;
  }
  adc = floor(adc + 0.5);
  if (adc < 0.0) adc = 0.0;
  if (adc > 16383.0) adc = 16383.0;
  outr[i] = (uint16_t)((code << 14) | (uint32_t)adc);
}

double radius_max(const synth_spec* s) {
  double rmax = 0.0;
  const double xs[2] = {0.0, (double)s->cols}, ys[2] = {0.0, (double)s->rows};
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      const double r = hypot(xs[a] - s->cx, ys[b] - s->cy);
      if (r > rmax) rmax = r;
    }
  return rmax;
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" size_t synth_gpu_scratch_bytes(const synth_spec* s, int32_t n_frames) {
  if (!s || n_frames <= 0 || s->rows <= 0 || s->cols <= 0) return 0;
  const int64_t ntab = (int64_t)(radius_max(s) * 8.0) + 2;
  const int64_t npix = (int64_t)s->rows * s->cols;
  return al256((size_t)n_frames * 2 * ntab * 8) + al256((size_t)n_frames * npix * 4) + al256((size_t)n_frames * 4);
}

// Returns 0 on success, 1 bad arguments, 2 scratch too small, 3 a CUDA error.
extern "C" int synth_gpu_frames(const synth_spec* s, int64_t frame0, int32_t n_frames, const float* ped,
                                const float* gain, const uint8_t* mask, void* out, void* scratch, size_t scratch_bytes,
                                void* stream) {
  if (!s || n_frames < 0 || s->rows <= 0 || s->cols <= 0 || frame0 < 0 || !out) return 1;
  if (n_frames == 0) return 0;
  if (s->out_raw && (!ped || !gain)) return 1;
  if (s->spots_max < s->spots_min || s->spots_min < 0) return 1;
  if (!scratch || scratch_bytes < synth_gpu_scratch_bytes(s, n_frames)) return 2;
  cudaStream_t st = (cudaStream_t)stream;
  const double rmax = radius_max(s);
  const int64_t ntab = (int64_t)(rmax * 8.0) + 2;
  const int64_t npix = (int64_t)s->rows * s->cols;
  unsigned char* b = static_cast<unsigned char*>(scratch);
  double* tab = reinterpret_cast<double*>(b);
  float* extra = reinterpret_cast<float*>(b + al256((size_t)n_frames * 2 * ntab * 8));
  int32_t* nsp = reinterpret_cast<int32_t*>(b + al256((size_t)n_frames * 2 * ntab * 8) +
                                            al256((size_t)n_frames * npix * 4));
  if (cudaMemsetAsync(extra, 0, (size_t)n_frames * npix * 4, st) != cudaSuccess) return 3;
  k_frame_setup<<<n_frames, 256, 0, st>>>(*s, frame0, rmax, ntab, tab, extra, nsp);
  dim3 grid((unsigned)((npix + 255) / 256), (unsigned)n_frames);
  k_pixels<<<grid, 256, 0, st>>>(*s, frame0, n_frames, ntab, tab, extra, ped, gain, mask, out);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}
