/*
 * Seeded synthetic inputs for the signal-separation path.
 *
 * This module only *makes inputs*: detector masks, Jungfrau-like calibration
 * planes and diffraction-like frames (isotropic background + Gaussian Bragg
 * spots + Poisson counting noise, optionally encoded as raw Jungfrau words).
 * It holds none of the method's arithmetic (no correction, no binning, no
 * moments, no clipping) and is used by both the CPU oracle tests and the GPU
 * path, which therefore see identical frames.
 *
 * Randomness: Philox4x32-10, the counter-based generator of Salmon, Moraes,
 * Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC 2011),
 * keyed by the 64-bit seed, with counter (index_lo, index_hi, frame, stream).
 * Every draw is a pure function of (seed, frame, pixel/spot, stream), so the
 * output does not depend on thread count or scheduling.
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC -ffp-contract=off synth.c -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Philox4x32-10                                                        */
/* ------------------------------------------------------------------ */
#define PH_M0 0xD2511F53u
#define PH_M1 0xCD9E8D57u
#define PH_W0 0x9E3779B9u
#define PH_W1 0xBB67AE85u

typedef struct { uint32_t x[4]; } ph4;

static inline ph4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                           uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)PH_M0 * c0;
    uint64_t p1 = (uint64_t)PH_M1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += PH_W0; k1 += PH_W1;
  }
  ph4 o; o.x[0] = c0; o.x[1] = c1; o.x[2] = c2; o.x[3] = c3;
  return o;
}

enum { ST_PIXEL = 0, ST_FRAME = 1, ST_SPOT = 2, ST_CALIB = 3 };

typedef struct { uint32_t k0, k1; } key_t2;

static inline ph4 draw(key_t2 k, uint64_t index, uint32_t frame, uint32_t stream) {
  return philox10((uint32_t)index, (uint32_t)(index >> 32), frame, stream, k.k0, k.k1);
}

/* uniform in the open interval (0, 1) from 24 random bits */
static inline double u01(uint32_t x) { return ((double)(x >> 8) + 0.5) * (1.0 / 16777216.0); }

/* one standard normal from two uniforms (Box-Muller) */
static inline double normal2(uint32_t a, uint32_t b) {
  return sqrt(-2.0 * log(u01(a))) * cos(6.283185307179586 * u01(b));
}

/* ------------------------------------------------------------------ */
/* Detector masks                                                       */
/* ------------------------------------------------------------------ */
/*
 * Jungfrau-style layout: n_mr x n_mc modules of 514 x 1030 pixels, each made
 * of 2 x 4 chips of 256 x 256 separated by 2-pixel chip gaps; modules are
 * separated by inter-module gaps that share out the remaining rows/columns
 * (floor), any remainder goes to the bottom/right edge. Chip gaps,
 * inter-module gaps and the remainder are masked (mask = 1).
 * A 4 x 2 grid in 2164 x 2068 gives 36-row and 8-column gaps.
 */
int synth_jf_mask(int32_t rows, int32_t cols, int32_t n_mr, int32_t n_mc, uint8_t* mask) {
  const int MR = 514, MC = 1030;
  if (rows < n_mr * MR || cols < n_mc * MC || n_mr < 1 || n_mc < 1) return 1;
  int gap_r = n_mr > 1 ? (rows - n_mr * MR) / (n_mr - 1) : 0;
  int gap_c = n_mc > 1 ? (cols - n_mc * MC) / (n_mc - 1) : 0;
  memset(mask, 1, (size_t)rows * cols);
  for (int mr = 0; mr < n_mr; ++mr) {
    int r0 = mr * (MR + gap_r);
    for (int mc = 0; mc < n_mc; ++mc) {
      int c0 = mc * (MC + gap_c);
      for (int r = 0; r < MR; ++r) {
        if (r == 256 || r == 257) continue;               /* chip gap rows */
        uint8_t* row = mask + (size_t)(r0 + r) * cols + c0;
        for (int c = 0; c < MC; ++c) {
          /* chips of 256 columns separated by 2-column gaps */
          if (c == 256 || c == 257 || c == 514 || c == 515 || c == 772 || c == 773) continue;
          row[c] = 0;
        }
      }
    }
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Jungfrau calibration planes                                          */
/* ------------------------------------------------------------------ */
/*
 * ped[p][i] ~ N(ped_mean[p], ped_std[p]); gain[p][i] = gain_nom[p] * (1 + U[-tol, tol]).
 * Layout: plane-major, ped[p * npix + i].
 */
void synth_calib(uint64_t seed, int64_t npix, const double* ped_mean, const double* ped_std,
                 const double* gain_nom, double gain_tol, float* ped, float* gain) {
  key_t2 k = {(uint32_t)seed, (uint32_t)(seed >> 32)};
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < npix; ++i) {
    for (int p = 0; p < 3; ++p) {
      ph4 r = draw(k, (uint64_t)i, (uint32_t)p, ST_CALIB);
      double z = normal2(r.x[0], r.x[1]);
      double u = u01(r.x[2]);
      ped[(int64_t)p * npix + i] = (float)(ped_mean[p] + ped_std[p] * z);
      gain[(int64_t)p * npix + i] = (float)(gain_nom[p] * (1.0 + gain_tol * (2.0 * u - 1.0)));
    }
  }
}

/* ------------------------------------------------------------------ */
/* Frames                                                               */
/* ------------------------------------------------------------------ */
typedef struct {
  int32_t rows, cols;
  double cx, cy;            /* beam centre in px: x = column, y = row; pixel centres at idx + 0.5 */
  int32_t bg_kind;          /* 0: fixed profile 50 exp(-r/80) + 30 exp(-(r-90)^2/72); 1: random solvent profile */
  double bg_scale_lo, bg_scale_hi; /* kind 1: log-uniform overall scale of the profile */
  double bg_clip_lo, bg_clip_hi;   /* kind 1: background photons/px clipped into this range */
  double hit_rate;          /* probability that a frame carries spots */
  int32_t spots_min, spots_max;
  double amp_lo, amp_hi;    /* spot peak amplitude (photons) */
  int32_t amp_log;          /* 1: log-uniform amplitude, 0: uniform */
  double sig_lo, sig_hi;    /* spot Gaussian width (px) */
  int32_t out_raw;          /* 0: float32 photon counts, 1: raw Jungfrau uint16 words */
  double read_noise_adu;    /* Gaussian read noise in gain level 0 (ADU) */
  uint64_t seed;
} synth_spec;

typedef struct { float x, y, amp, sigma; } synth_spot;

/* Draw a Poisson count with mean lam, given e^-lam (p0) and one uniform u.
 * Inversion by sequential search for lam < 40, a rounded normal above. */
static inline double poisson_draw(double lam, double p0, double u, double z) {
  if (lam <= 0.0) return 0.0;
  if (lam < 40.0) {
    double k = 0.0, p = p0, F = p0;
    while (u > F && k < 400.0) { k += 1.0; p *= lam / k; F += p; }
    return k;
  }
  double n = floor(lam + sqrt(lam) * z + 0.5);
  return n < 0.0 ? 0.0 : n;
}

typedef struct {
  double scale, A, r0, rr[3], ra[3], rw[3];
  int hit, nspots;
} frame_par;

static void frame_params(const synth_spec* s, key_t2 k, uint32_t f, double rmax, frame_par* fp) {
  ph4 a = draw(k, 0, f, ST_FRAME);
  ph4 b = draw(k, 1, f, ST_FRAME);
  ph4 c = draw(k, 2, f, ST_FRAME);
  ph4 d = draw(k, 3, f, ST_FRAME);
  fp->scale = s->bg_scale_lo * pow(s->bg_scale_hi / s->bg_scale_lo, u01(a.x[0]));
  fp->A = 0.5 + u01(a.x[1]);
  fp->r0 = rmax * (0.2 + 0.4 * u01(a.x[2]));
  for (int m = 0; m < 3; ++m) {
    fp->rr[m] = rmax * (0.15 + 0.7 * u01(b.x[m]));
    fp->ra[m] = 0.2 + 0.8 * u01(c.x[m]);
    fp->rw[m] = rmax * (0.01 + 0.03 * u01(d.x[m]));
  }
  fp->hit = u01(a.x[3]) < s->hit_rate;
  int span = s->spots_max - s->spots_min + 1;
  fp->nspots = fp->hit ? s->spots_min + (int)(u01(b.x[3]) * span) : 0;
  if (fp->nspots > s->spots_max) fp->nspots = s->spots_max;
}

static double bg_profile(const synth_spec* s, const frame_par* fp, double r) {
  if (s->bg_kind == 0)
    return 50.0 * exp(-r / 80.0) + 30.0 * exp(-(r - 90.0) * (r - 90.0) / (2.0 * 36.0));
  double v = fp->A * exp(-r / fp->r0);
  for (int m = 0; m < 3; ++m) {
    double t = (r - fp->rr[m]) / fp->rw[m];
    v += fp->ra[m] * exp(-0.5 * t * t);
  }
  v *= fp->scale;
  if (v < s->bg_clip_lo) v = s->bg_clip_lo;
  if (v > s->bg_clip_hi) v = s->bg_clip_hi;
  return v;
}

/*
 * Generate frames [frame0, frame0 + n_frames).
 *   out: float32 [n_frames][npix] (out_raw = 0) or uint16 [n_frames][npix] (out_raw = 1)
 *   ped/gain: calibration planes [3][npix] (needed for out_raw = 1)
 *   mask: nonzero = masked (written as 0); may be NULL
 *   spots_out: optional [n_frames][max_spots] truth list, n_spots_out: [n_frames]
 * The background is tabulated on a 1/8-px radial grid (nearest node), which
 * defines the generator's background exactly.
 * Returns 0 on success.
 */
int synth_frames(const synth_spec* s, int64_t frame0, int32_t n_frames, const float* ped,
                 const float* gain, const uint8_t* mask, void* out, synth_spot* spots_out,
                 int32_t max_spots, int32_t* n_spots_out) {
  const int64_t rows = s->rows, cols = s->cols, npix = rows * cols;
  if (rows <= 0 || cols <= 0) return 1;
  if (s->out_raw && (!ped || !gain)) return 2;
  key_t2 k = {(uint32_t)s->seed, (uint32_t)(s->seed >> 32)};
  double rmax = 0.0;
  {
    double xs[2] = {0.0, (double)cols}, ys[2] = {0.0, (double)rows};
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        double r = hypot(xs[a] - s->cx, ys[b] - s->cy);
        if (r > rmax) rmax = r;
      }
  }
  const int64_t ntab = (int64_t)(rmax * 8.0) + 2;
  int err = 0;

#pragma omp parallel
  {
    float* extra = (float*)calloc((size_t)npix, sizeof(float));
    double* tab = (double*)malloc((size_t)ntab * sizeof(double));
    double* tabe = (double*)malloc((size_t)ntab * sizeof(double));
    synth_spot* sp = (synth_spot*)malloc(sizeof(synth_spot) * (size_t)(s->spots_max > 0 ? s->spots_max : 1));
    if (!extra || !tab || !tabe || !sp) {
#pragma omp atomic write
      err = 3;
    }
#pragma omp for schedule(dynamic, 1)
    for (int32_t fi = 0; fi < n_frames; ++fi) {
      if (err) continue;
      uint32_t f = (uint32_t)(frame0 + fi);
      frame_par fp;
      frame_params(s, k, f, rmax, &fp);
      for (int64_t t = 0; t < ntab; ++t) {
        tab[t] = bg_profile(s, &fp, (double)t / 8.0);
        tabe[t] = exp(-tab[t]);
      }
      /* spots */
      for (int j = 0; j < fp.nspots; ++j) {
        ph4 r = draw(k, (uint64_t)j, f, ST_SPOT);
        sp[j].x = (float)(u01(r.x[0]) * (double)cols);
        sp[j].y = (float)(u01(r.x[1]) * (double)rows);
        double u = u01(r.x[2]);
        double amp = s->amp_log ? s->amp_lo * pow(s->amp_hi / s->amp_lo, u)
                                : s->amp_lo + (s->amp_hi - s->amp_lo) * u;
        sp[j].amp = (float)amp;
        sp[j].sigma = (float)(s->sig_lo + (s->sig_hi - s->sig_lo) * u01(r.x[3]));
        double sx = sp[j].x, sy = sp[j].y, sg = sp[j].sigma;
        int w = (int)ceil(4.0 * sg) + 1;
        int64_t r_lo = (int64_t)floor(sy) - w, r_hi = (int64_t)floor(sy) + w;
        int64_t c_lo = (int64_t)floor(sx) - w, c_hi = (int64_t)floor(sx) + w;
        for (int64_t rr = r_lo < 0 ? 0 : r_lo; rr <= r_hi && rr < rows; ++rr)
          for (int64_t cc = c_lo < 0 ? 0 : c_lo; cc <= c_hi && cc < cols; ++cc) {
            double dx = (double)cc + 0.5 - sx, dy = (double)rr + 0.5 - sy;
            extra[rr * cols + cc] += (float)(amp * exp(-(dx * dx + dy * dy) / (2.0 * sg * sg)));
          }
      }
      if (spots_out && n_spots_out) {
        int nn = fp.nspots < max_spots ? fp.nspots : max_spots;
        memcpy(spots_out + (int64_t)fi * max_spots, sp, sizeof(synth_spot) * (size_t)nn);
        n_spots_out[fi] = fp.nspots;
      }
      /* pixels */
      float* outf = s->out_raw ? NULL : (float*)out + (int64_t)fi * npix;
      uint16_t* outr = s->out_raw ? (uint16_t*)out + (int64_t)fi * npix : NULL;
      for (int64_t rr = 0; rr < rows; ++rr) {
        double dy = (double)rr + 0.5 - s->cy;
        for (int64_t cc = 0; cc < cols; ++cc) {
          int64_t i = rr * cols + cc;
          if (mask && mask[i]) {
            if (outf) outf[i] = 0.0f; else outr[i] = 0;
            continue;
          }
          double dx = (double)cc + 0.5 - s->cx;
          int64_t t = (int64_t)(sqrt(dx * dx + dy * dy) * 8.0 + 0.5);
          if (t >= ntab) t = ntab - 1;
          double lam = tab[t], p0 = tabe[t];
          if (extra[i] != 0.0f) { lam += (double)extra[i]; p0 = exp(-lam); }
          ph4 r = draw(k, (uint64_t)i, f, ST_PIXEL);
          double zp = 0.0;
          if (lam >= 40.0) { ph4 r2 = draw(k, (uint64_t)i, f, ST_PIXEL + 8); zp = normal2(r2.x[0], r2.x[1]); }
          double n = poisson_draw(lam, p0, u01(r.x[0]), zp);
          if (outf) { outf[i] = (float)n; continue; }
          /* Jungfrau encoding: gain level chosen by the charge, ADC falls with
           * charge in levels 1 and 2 (negative gains), read noise in level 0 */
          double p0d = ped[i], g0 = gain[i];
          double adc; uint16_t code;
          if (p0d + g0 * n <= 16000.0) {
            adc = p0d + g0 * n + s->read_noise_adu * normal2(r.x[1], r.x[2]);
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
          outr[i] = (uint16_t)((code << 14) | (uint16_t)adc);
        }
      }
      /* clear the spot windows for the next frame */
      for (int j = 0; j < fp.nspots; ++j) {
        double sx = sp[j].x, sy = sp[j].y, sg = sp[j].sigma;
        int w = (int)ceil(4.0 * sg) + 1;
        int64_t r_lo = (int64_t)floor(sy) - w, r_hi = (int64_t)floor(sy) + w;
        int64_t c_lo = (int64_t)floor(sx) - w, c_hi = (int64_t)floor(sx) + w;
        for (int64_t rr = r_lo < 0 ? 0 : r_lo; rr <= r_hi && rr < rows; ++rr)
          for (int64_t cc = c_lo < 0 ? 0 : c_lo; cc <= c_hi && cc < cols; ++cc) extra[rr * cols + cc] = 0.0f;
      }
    }
    free(extra); free(tab); free(tabe); free(sp);
  }
  return err;
}

/* Raw Philox block, exposed for the generator's own statistical tests. */
void synth_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  ph4 r = philox10(ctr[0], ctr[1], ctr[2], ctr[3], key[0], key[1]);
  memcpy(out, r.x, sizeof(r.x));
}

int synth_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
