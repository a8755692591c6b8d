/*
 * CPU oracle for the signal-separation path (Kieffer et al., "Application of
 * signal separation to diffraction image compression and serial
 * crystallography", arXiv 2411.09515).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct
 * statement of what the GPU path computes. Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark call it. It shares no code,
 * header, table or helper with the CUDA library; both sides only consume the
 * same seeded inputs.
 *
 * Precision: everything is IEEE binary64 with direct loops, except the
 * detector correction, which is defined as two binary32 operations (see
 * oracle_jf_photons). Compile with -ffp-contract=off and without -ffast-math.
 *
 * Parity status of each function is stated in its comment; the pins live in
 * tests/test_oracle_*.py.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* 1. Detector correction (Section 1.2; Eq. 1 numerator)                      */
/* ------------------------------------------------------------------------ */
/*
 * A raw Jungfrau word carries the gain level in its two top bits and a 14-bit
 * ADC value below (three gain levels, each with its own pedestal and gain,
 * Section 1.2). Code 0 is level 0, code 1 level 1, codes 2 and 3 level 2.
 * The corrected pixel value (photons) is the dark-subtracted signal of Eq. 1
 * divided by the gain of the selected level:
 *     p = RN32( RN32(adc - ped[g]) / gain[g] )
 * i.e. one binary32 subtraction and one binary32 division, both rounded to
 * nearest-even. This is the only binary32 arithmetic in the oracle.
 * Parity: pinned by closed-form cases and by the decode table (tests).
 */
static inline int jf_level(uint16_t raw) {
  int code = raw >> 14;
  return code == 0 ? 0 : (code == 1 ? 1 : 2);
}

void oracle_jf_photons(int64_t n, const uint16_t* raw, const float* ped, const float* gain,
                       int64_t plane_stride, float* out) {
  for (int64_t i = 0; i < n; ++i) {
    int g = jf_level(raw[i]);
    float adc = (float)(raw[i] & 0x3FFF);
    float x = adc - ped[(int64_t)g * plane_stride + i];
    out[i] = x / gain[(int64_t)g * plane_stride + i];
  }
}

/* ------------------------------------------------------------------------ */
/* 2. Pixel-to-bin coefficients c_{i,r} (Section 2.2, azimuthal averaging)    */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t rows, cols;
  double pixel_y, pixel_x;   /* m */
  double dist;               /* m, flat detector normal to the beam */
  double cx, cy;             /* beam centre in px (x = column, y = row) */
  double wavelength;         /* m */
  int32_t unit;              /* 0: 2theta in degrees, 1: q in nm^-1, 2: r in mm */
  int32_t nbins;
  int32_t split;             /* s: s x s sub-pixel centres per pixel */
  double lo, hi;             /* radial range; NaN = automatic */
} oracle_geom;

/*
 * Radial unit of the point at (row + fy, col + fx) in pixel coordinates
 * (pixel (row, col) spans [row, row+1) x [col, col+1)):
 *   dy = (row + fy - cy) * pixel_y,  dx = (col + fx - cx) * pixel_x,
 *   r = sqrt(dx*dx + dy*dy),  2theta = atan2(r, dist),
 *   unit 0: 2theta * 180 / pi;  unit 1: 4 pi sin(2theta / 2) / (wavelength * 1e9);
 *   unit 2: r * 1e3.
 */
static double unit_value(const oracle_geom* g, int64_t row, int64_t col, double fy, double fx) {
  double dy = ((double)row + fy - g->cy) * g->pixel_y;
  double dx = ((double)col + fx - g->cx) * g->pixel_x;
  double r = sqrt(dx * dx + dy * dy);
  if (g->unit == 2) return r * 1.0e3;
  double tth = atan2(r, g->dist);
  if (g->unit == 0) return tth * (180.0 / M_PI);
  return 4.0 * M_PI * sin(0.5 * tth) / (g->wavelength * 1.0e9);
}

/* sub-pixel centre offset: (a + 0.5) / s */
static double sub_off(int a, int s) { return ((double)a + 0.5) / (double)s; }

/* Bin index of unit value x on [lo, hi] with B equal bins; -1 if outside. */
static int32_t bin_of(double x, double lo, double hi, int32_t B) {
  if (!(x >= lo && x <= hi)) return -1;
  double t = (x - lo) / (hi - lo) * (double)B;
  int64_t b = (int64_t)floor(t);
  if (b >= B) b = B - 1;
  if (b < 0) b = 0;
  return (int32_t)b;
}

/* Automatic range: minimum and maximum unit value over all sub-pixel centres
 * of all valid pixels. */
void oracle_unit_range(const oracle_geom* g, const uint8_t* mask, double* lo, double* hi) {
  double mn = INFINITY, mx = -INFINITY;
  int s = g->split;
  for (int64_t row = 0; row < g->rows; ++row)
    for (int64_t col = 0; col < g->cols; ++col) {
      if (mask && mask[row * g->cols + col]) continue;
      for (int a = 0; a < s; ++a)
        for (int b = 0; b < s; ++b) {
          double x = unit_value(g, row, col, sub_off(a, s), sub_off(b, s));
          if (x < mn) mn = x;
          if (x > mx) mx = x;
        }
    }
  *lo = mn;
  *hi = mx;
}

/* Radial value of every pixel centre (unit_value at offset 0.5, 0.5), masked
 * ones included. */
void oracle_pixel_unit(const oracle_geom* g, double* out) {
  for (int64_t row = 0; row < g->rows; ++row)
    for (int64_t col = 0; col < g->cols; ++col) out[row * g->cols + col] = unit_value(g, row, col, 0.5, 0.5);
}

/*
 * Coefficients c_{i,r}: the fraction of pixel i falling in radial bin r
 * (Section 2.2), measured by s x s sub-pixel centres: c = (#centres in r)/s^2.
 * With s = 1 every coefficient is 1 (no pixel splitting).
 * Output (pixel-major, bins ascending within a pixel): e_pix, e_bin, e_c.
 * bin_of_pixel[i] = bin of the pixel centre (clamped into [0, B-1]), -1 for a
 * masked pixel. Returns the number of entries (entries beyond cap are not
 * written). lo/hi are taken from g unless NaN, then from oracle_unit_range.
 * Parity: pinned by sum_r c = 1, by symmetric pixels, and by an inverse-unit
 * recomputation of every bin edge (tests).
 */
int64_t oracle_weights(const oracle_geom* g_in, const uint8_t* mask, int64_t cap, int32_t* e_pix,
                       int32_t* e_bin, double* e_c, int32_t* bin_of_pixel, double* range_out) {
  oracle_geom g = *g_in;
  if (isnan(g.lo) || isnan(g.hi)) {
    double lo, hi;
    oracle_unit_range(&g, mask, &lo, &hi);
    if (isnan(g.lo)) g.lo = lo;
    if (isnan(g.hi)) g.hi = hi;
  }
  if (range_out) { range_out[0] = g.lo; range_out[1] = g.hi; }
  int s = g.split;
  int32_t* sb = (int32_t*)malloc(sizeof(int32_t) * (size_t)(s * s));
  int64_t n = 0;
  for (int64_t row = 0; row < g.rows; ++row)
    for (int64_t col = 0; col < g.cols; ++col) {
      int64_t i = row * g.cols + col;
      if (mask && mask[i]) {
        if (bin_of_pixel) bin_of_pixel[i] = -1;
        continue;
      }
      if (bin_of_pixel) {
        double xc = unit_value(&g, row, col, 0.5, 0.5);
        int32_t bc;
        if (xc < g.lo) bc = 0;
        else if (xc > g.hi) bc = g.nbins - 1;
        else bc = bin_of(xc, g.lo, g.hi, g.nbins);
        bin_of_pixel[i] = bc;
      }
      int m = 0;
      for (int a = 0; a < s; ++a)
        for (int b = 0; b < s; ++b) sb[m++] = bin_of(unit_value(&g, row, col, sub_off(a, s), sub_off(b, s)), g.lo, g.hi, g.nbins);
      /* one entry per distinct bin, ascending */
      int32_t last = -1;
      for (;;) {
        int32_t nxt = INT32_MAX;
        for (int t = 0; t < m; ++t)
          if (sb[t] > last && sb[t] < nxt) nxt = sb[t];
        if (nxt == INT32_MAX) break;
        int cnt = 0;
        for (int t = 0; t < m; ++t) cnt += (sb[t] == nxt);
        if (n < cap) {
          e_pix[n] = (int32_t)i;
          e_bin[n] = nxt;
          e_c[n] = (double)cnt / (double)(s * s);
        }
        ++n;
        last = nxt;
      }
    }
  free(sb);
  return n;
}

/* ------------------------------------------------------------------------ */
/* 3. Moments and sigma-clipping (Eqs. 2, 6, 8-13, 19; Section 2.4)           */
/* ------------------------------------------------------------------------ */
/*
 * For a set S of entries e = (pixel i, coefficient c) of one bin, with
 * signal_i, norm_i, v_i = signal_i / norm_i and weight w_e = c * norm_i:
 *   Omega   = sum w                         (Eq. 8)
 *   OmegaOm = sum w^2                       (Eq. 9)
 *   V       = sum c * signal = sum w v      (Eq. 10)
 *   mu      = V / Omega                     (Eqs. 2 and 12)
 *   VV      = sum w^2 (v - mu)^2            (Eq. 11, second pass as Eq. 6)
 *   sigma   = sqrt(VV / OmegaOm)            (Eq. 13; the deviation of one pixel, "std")
 * An empty set (Omega = 0) has mu = 0, sigma = 0.
 */
/*
 * sigma_p: the deviation of one pixel under the Poisson model (Eqs. 3 and 4
 * of Section 2.2): every pixel's variance is its signal plus the dark
 * variance, var_i = signal_i + dark (Eq. 3), propagated with squared
 * coefficients (Eq. 4) and normalised like sigma (the deviation of one
 * pixel, so that Eq. 5 turns it into the error of the mean):
 * sigma_p^2 = sum c^2 var_i / sum c^2 norm^2.
 */
typedef struct { double mu, sigma, omega, sigma_p; int64_t count; } moments_t;

static moments_t moments(int64_t m, const int64_t* ent, const uint8_t* keep, const double* ec,
                         const int32_t* epix, const double* v, const double* nrm, double dark) {
  moments_t r = {0.0, 0.0, 0.0, 0.0, 0};
  double Om = 0.0, V = 0.0, OO = 0.0, VV = 0.0, VP = 0.0;
  for (int64_t t = 0; t < m; ++t) {
    if (!keep[t]) continue;
    int64_t e = ent[t];
    double w = ec[e] * nrm[epix[e]];
    if (w == 0.0) continue;
    Om += w;
    V += w * v[epix[e]];
    r.count += 1;
  }
  if (Om == 0.0) { r.count = 0; return r; }
  double mu = V / Om;
  for (int64_t t = 0; t < m; ++t) {
    if (!keep[t]) continue;
    int64_t e = ent[t];
    double w = ec[e] * nrm[epix[e]];
    if (w == 0.0) continue;
    double d = v[epix[e]] - mu;
    OO += w * w;
    VV += w * w * d * d;
    VP += ec[e] * ec[e] * (v[epix[e]] * nrm[epix[e]] + dark);
  }
  r.mu = mu;
  r.sigma = sqrt(VV / OO);
  r.sigma_p = VP > 0.0 ? sqrt(VP / OO) : 0.0;
  r.omega = Om;
  return r;
}

/*
 * Integrate one frame and sigma-clip every bin (Eq. 19 applied repeatedly,
 * Section 2.4):
 *   S_0 = all entries of the bin;
 *   for t = 0 .. n_iter-1:
 *       (mu_t, sigma_t) = moments(S_t)
 *       S_{t+1} = { e in S_t : |v_e - mu_t| <= k_t sigma_t }   (reject iff >, Eq. 19)
 *       stop as soon as S_{t+1} == S_t (nothing discarded)
 * with k_t = k, or with chauvenet != 0 the cut-off of Eq. 20 for the current
 * set's size n_t = |S_t|: k_t = sqrt(2 ln(n_t / sqrt(2 pi))); a set of two
 * entries or fewer (ln <= 0) is not clipped (the loop stops).
 * Error model (Section 2.4.1): 0 azimuthal (sigma_t, Eq. 13, clips and is
 * reported), 1 Poisson (sigma_p clips and is reported), 2 hybrid (sigma
 * clips, sigma_p of the final set is reported); dark: the dark variance.
 *   report moments(S_final) for the last set computed, and |S_final|.
 * Discarded entries never come back. Entries with weight 0 take part in no
 * sum and are not counted.
 *
 * band[b] (optional) = min over every rejection decision taken in bin b of
 *   | |v - mu_t| - k sigma_t | / max(|mu_t| + k sigma_t, DBL_MIN)
 * i.e. how close the closest entry came to a clip boundary, relative.
 * keep_out (optional, per entry, in input order): 1 if in S_final.
 * iters[b] = number of rejection steps taken (0 .. n_iter).
 * Parity: pinned by the two-pixel example of Section 2.4.1, closed-form sets,
 * the truncated-Gaussian fixed point and brute force (tests).
 */
int oracle_integrate_clip(int64_t npix, int64_t n_ent, const int32_t* e_pix, const int32_t* e_bin,
                          const double* e_c, int32_t nbins, const float* signal, const float* norm,
                          int32_t n_iter, double k, int32_t chauvenet, int32_t model, double dark,
                          double* mean, double* sigma, int32_t* count, int32_t* iters, double* band,
                          uint8_t* keep_out) {
  double* v = (double*)malloc(sizeof(double) * (size_t)npix);
  double* nrm = (double*)malloc(sizeof(double) * (size_t)npix);
  int64_t* start = (int64_t*)calloc((size_t)nbins + 1, sizeof(int64_t));
  int64_t* ent = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n_ent > 0 ? n_ent : 1));
  uint8_t* keep = (uint8_t*)malloc((size_t)(n_ent > 0 ? n_ent : 1));
  uint8_t* nk = (uint8_t*)malloc((size_t)(n_ent > 0 ? n_ent : 1));
  if (!v || !nrm || !start || !ent || !keep || !nk) return 1;
  for (int64_t i = 0; i < npix; ++i) {
    nrm[i] = norm ? (double)norm[i] : 1.0;
    v[i] = (double)signal[i] / nrm[i];
  }
  /* group entries by bin (counting sort, input order kept within a bin) */
  for (int64_t e = 0; e < n_ent; ++e) start[e_bin[e] + 1] += 1;
  for (int32_t b = 0; b < nbins; ++b) start[b + 1] += start[b];
  {
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)nbins);
    memcpy(fill, start, sizeof(int64_t) * (size_t)nbins);
    for (int64_t e = 0; e < n_ent; ++e) ent[fill[e_bin[e]]++] = e;
    free(fill);
  }
  for (int32_t b = 0; b < nbins; ++b) {
    int64_t m = start[b + 1] - start[b];
    const int64_t* eb = ent + start[b];
    uint8_t* kb = keep + start[b];
    uint8_t* nb = nk + start[b];
    for (int64_t t = 0; t < m; ++t) kb[t] = 1;
    double bmin = INFINITY;
    int32_t steps = 0;
    for (int32_t it = 0; it < n_iter; ++it) {
      moments_t mo = moments(m, eb, kb, e_c, e_pix, v, nrm, dark);
      double kt = k;
      if (chauvenet) {
        if (mo.count <= 2) break;
        kt = sqrt(2.0 * log((double)mo.count / sqrt(2.0 * M_PI)));
      }
      double lim = kt * (model == 1 ? mo.sigma_p : mo.sigma);
      double scale = fabs(mo.mu) + lim;
      if (scale < DBL_MIN) scale = DBL_MIN;
      int changed = 0;
      for (int64_t t = 0; t < m; ++t) {
        nb[t] = kb[t];
        if (!kb[t]) continue;
        int64_t e = eb[t];
        if (e_c[e] * nrm[e_pix[e]] == 0.0) continue;
        double dev = fabs(v[e_pix[e]] - mo.mu);
        double rel = fabs(dev - lim) / scale;
        if (rel < bmin) bmin = rel;
        if (dev > lim) { nb[t] = 0; changed = 1; }
      }
      if (!changed) break;
      memcpy(kb, nb, (size_t)m);
      steps += 1;
    }
    moments_t fin = moments(m, eb, kb, e_c, e_pix, v, nrm, dark);
    mean[b] = fin.mu;
    sigma[b] = model == 0 ? fin.sigma : fin.sigma_p;
    if (count) count[b] = (int32_t)fin.count;
    if (iters) iters[b] = steps;
    if (band) band[b] = bmin;
    if (keep_out)
      for (int64_t t = 0; t < m; ++t) keep_out[eb[t]] = kb[t];
  }
  free(v); free(nrm); free(start); free(ent); free(keep); free(nk);
  return 0;
}

/*
 * Moments of an explicit subset, used by the tests to re-evaluate a bin on a
 * set chosen elsewhere (same definitions as above).
 */
void oracle_moments_subset(int64_t m, const int32_t* pix, const double* c, const uint8_t* sel,
                           const float* signal, const float* norm, int32_t model, double dark, double* out3) {
  double Om = 0, V = 0, OO = 0, VV = 0, VP = 0;
  int64_t cnt = 0;
  for (int64_t t = 0; t < m; ++t) {
    if (!sel[t]) continue;
    double nr = norm ? (double)norm[pix[t]] : 1.0;
    double w = c[t] * nr;
    if (w == 0.0) continue;
    Om += w;
    V += w * ((double)signal[pix[t]] / nr);
    cnt++;
  }
  double mu = Om == 0.0 ? 0.0 : V / Om;
  for (int64_t t = 0; t < m && Om != 0.0; ++t) {
    if (!sel[t]) continue;
    double nr = norm ? (double)norm[pix[t]] : 1.0;
    double w = c[t] * nr;
    if (w == 0.0) continue;
    double d = (double)signal[pix[t]] / nr - mu;
    OO += w * w;
    VV += w * w * d * d;
    VP += c[t] * c[t] * ((double)signal[pix[t]] + dark);
  }
  out3[0] = mu;
  out3[1] = Om == 0.0 ? 0.0 : (model == 0 ? sqrt(VV / OO) : (VP > 0.0 ? sqrt(VP / OO) : 0.0));
  out3[2] = (double)(Om == 0.0 ? 0 : cnt);
}

/* ------------------------------------------------------------------------ */
/* 4. Sparsification (Section 3)                                              */
/* ------------------------------------------------------------------------ */
/*
 * A pixel is kept when its intensity is above the background of its radial
 * position by more than k_pick deviations: v_i > mu_b + k_pick sigma_b with
 * b = bin_of_pixel(i) (the bin of the pixel centre). Masked pixels are never
 * kept. Output: ascending pixel index, value v_i. Returns the number of kept
 * pixels (only the first cap are written).
 * Parity: pinned by the normal tail fractions of Section 3 and closed forms.
 */
int64_t oracle_sparsify(int64_t npix, const int32_t* bin_of_pixel, const float* signal,
                        const float* norm, const double* mean, const double* sigma, double k_pick,
                        int64_t cap, int32_t* idx, double* val) {
  int64_t n = 0;
  for (int64_t i = 0; i < npix; ++i) {
    int32_t b = bin_of_pixel[i];
    if (b < 0) continue;
    double vi = (double)signal[i] / (norm ? (double)norm[i] : 1.0);
    if (vi > mean[b] + k_pick * sigma[b]) {
      if (n < cap) { idx[n] = (int32_t)i; val[n] = vi; }
      ++n;
    }
  }
  return n;
}

/* ------------------------------------------------------------------------ */
/* 5. Peak picking (Section 4)                                                */
/* ------------------------------------------------------------------------ */
/*
 * Over the kept pixels i of a frame (Section 3 criterion), with P the
 * patch x patch square centred on i, clipped to the image, masked pixels
 * excluded:
 *   (a) i is the maximum of P: for every other j in P, v_i > v_j, or
 *       v_i == v_j and i < j (one winner on a plateau);
 *   (b) at least min_count pixels of P (i included) are kept.
 * For a peak: w_j = v_j - mu_{b(j)} over the kept j in P,
 *   I = sum w_j,  centroid = sum w_j (row_j + 0.5, col_j + 0.5) / I,
 *   sigma_I = sqrt(sum sigma_{b(j)}^2)  (propagated deviation),
 *   npix = number of kept pixels in P.
 * Peaks are reported in ascending pixel index. Returns the number of peaks.
 * Parity: pinned by recovery of injected spots at known centres and by
 * hand-built patches (tests).
 */
typedef struct { int32_t idx; double y, x, I, sigma; int32_t npix; } oracle_peak;

int64_t oracle_peaks(int32_t rows, int32_t cols, const int32_t* bin_of_pixel, const float* signal,
                     const float* norm, const double* mean, const double* sigma, double k_pick,
                     int32_t patch, int32_t min_count, int64_t cap, oracle_peak* out) {
  int64_t npix = (int64_t)rows * cols;
  int h = patch / 2;
  int64_t n = 0;
  for (int64_t i = 0; i < npix; ++i) {
    int32_t bi = bin_of_pixel[i];
    if (bi < 0) continue;
    double vi = (double)signal[i] / (norm ? (double)norm[i] : 1.0);
    if (!(vi > mean[bi] + k_pick * sigma[bi])) continue;
    int64_t r0 = i / cols, c0 = i % cols;
    int is_max = 1, nk = 0;
    double I = 0, sy = 0, sx = 0, s2 = 0;
    for (int64_t r = r0 - h; r <= r0 + h; ++r)
      for (int64_t c = c0 - h; c <= c0 + h; ++c) {
        if (r < 0 || r >= rows || c < 0 || c >= cols) continue;
        int64_t j = r * cols + c;
        int32_t bj = bin_of_pixel[j];
        if (bj < 0) continue;
        double vj = (double)signal[j] / (norm ? (double)norm[j] : 1.0);
        if (j != i && !(vi > vj || (vi == vj && i < j))) is_max = 0;
        if (vj > mean[bj] + k_pick * sigma[bj]) {
          double w = vj - mean[bj];
          nk += 1;
          I += w;
          sy += w * ((double)r + 0.5);
          sx += w * ((double)c + 0.5);
          s2 += sigma[bj] * sigma[bj];
        }
      }
    if (!is_max || nk < min_count) continue;
    if (n < cap) {
      out[n].idx = (int32_t)i;
      out[n].I = I;
      out[n].y = sy / I;
      out[n].x = sx / I;
      out[n].sigma = sqrt(s2);
      out[n].npix = nk;
    }
    ++n;
  }
  return n;
}

/* ------------------------------------------------------------------------ */
/* 6. Whole frames (the baseline timing drives this)                          */
/* ------------------------------------------------------------------------ */
/*
 * Process n_frames frames end to end: correction (raw input) or float input,
 * integration + clipping, sparsification count and peak count per frame.
 * Frames are independent; with OpenMP they run in parallel, one frame per
 * thread. Outputs: mean/sigma [n_frames][nbins], n_kept and n_peaks
 * [n_frames]. Returns 0 on success.
 */
int oracle_process_frames(int32_t rows, int32_t cols, int64_t n_ent, const int32_t* e_pix,
                          const int32_t* e_bin, const double* e_c, const int32_t* bin_of_pixel,
                          int32_t nbins, int32_t n_frames, int32_t is_raw, const void* frames,
                          const float* ped, const float* gain, const float* norm, int32_t n_iter,
                          double k_clip, double k_pick, int32_t patch, int32_t min_count,
                          double* mean, double* sigma, int32_t* n_kept, int32_t* n_peaks,
                          int32_t n_threads) {
  int64_t npix = (int64_t)rows * cols;
  int err = 0;
#ifdef _OPENMP
  if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
  for (int32_t f = 0; f < n_frames; ++f) {
    float* sig = (float*)malloc(sizeof(float) * (size_t)npix);
    if (!sig) { err = 1; continue; }
    if (is_raw)
      oracle_jf_photons(npix, (const uint16_t*)frames + (int64_t)f * npix, ped, gain, npix, sig);
    else
      memcpy(sig, (const float*)frames + (int64_t)f * npix, sizeof(float) * (size_t)npix);
    double* mu = mean + (int64_t)f * nbins;
    double* sd = sigma + (int64_t)f * nbins;
    if (oracle_integrate_clip(npix, n_ent, e_pix, e_bin, e_c, nbins, sig, norm, n_iter, k_clip, 0, 0, 0.0,
                              mu, sd, NULL, NULL, NULL, NULL))
      err = 1;
    n_kept[f] = (int32_t)oracle_sparsify(npix, bin_of_pixel, sig, norm, mu, sd, k_pick, 0, NULL, NULL);
    n_peaks[f] = (int32_t)oracle_peaks(rows, cols, bin_of_pixel, sig, norm, mu, sd, k_pick, patch,
                                       min_count, 0, NULL);
    free(sig);
  }
  return err;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
