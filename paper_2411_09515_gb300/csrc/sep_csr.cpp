// Host construction of the integration matrix (Section 2.2).
//
// The coefficient c_{i,r} is the fraction of pixel i falling into radial bin
// r; it is measured with split x split sub-pixel centres, so c = k / split^2
// with k the number of centres of pixel i inside bin r, or (split 0) as the
// exact area fraction: the bin's edges map to detector radii and c is the
// area of the pixel between the two circles over the pixel's area
// (rectangle-disc intersections in closed form, binary64). The radial value of a
// point and its bin follow one fixed sequence of binary64 operations (the
// definition the tests compare against):
//   dy = (row + fy - cy) * pixel_y,  dx = (col + fx - cx) * pixel_x,
//   r = sqrt(dx*dx + dy*dy),  2theta = atan2(r, dist)
//   2theta unit: 2theta * (180 / pi);  q unit: 4 pi sin(2theta / 2) / (lambda * 1e9);
//   r unit: r * 1e3
//   bin = floor((x - lo) / (hi - lo) * nbins), the top edge going to nbins - 1,
//   values outside [lo, hi] dropped; sub-pixel offsets f = (a + 0.5) / split.
// Compiled with -ffp-contract=off so no multiply-add is fused.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <limits>

#include "sep_internal.h"

namespace sep {
namespace {

struct Geo {
  double py, px, dist, cx, cy, lam;
  int unit;
};

inline double radial(const Geo& g, int64_t row, int64_t col, double fy, double fx) {
  double dy = ((double)row + fy - g.cy) * g.py;
  double dx = ((double)col + fx - g.cx) * g.px;
  double r = sqrt(dx * dx + dy * dy);
  if (g.unit == SEP_UNIT_R_MM) return r * 1.0e3;
  double tth = atan2(r, g.dist);
  if (g.unit == SEP_UNIT_2TH_DEG) return tth * (180.0 / M_PI);
  return 4.0 * M_PI * sin(0.5 * tth) / (g.lam * 1.0e9);
}

// Detector-plane radius (metres) of a radial value and back (the unit's
// function of r in radial(), inverted); radii below 0 clamp to 0.
inline double radius_of(const Geo& g, double x) {
  double R;
  if (g.unit == SEP_UNIT_R_MM) {
    R = x * 1.0e-3;
  } else {
    double tth;
    if (g.unit == SEP_UNIT_2TH_DEG) {
      tth = x * (M_PI / 180.0);
    } else {
      const double sarg = x * g.lam * 1.0e9 / (4.0 * M_PI);
      tth = sarg >= 1.0 ? M_PI : 2.0 * asin(sarg);
    }
    R = tth >= 0.5 * M_PI ? std::numeric_limits<double>::infinity() : g.dist * tan(tth);
  }
  return R > 0.0 ? R : 0.0;
}
inline double unit_of(const Geo& g, double R) {
  if (g.unit == SEP_UNIT_R_MM) return R * 1.0e3;
  const double tth = atan2(R, g.dist);
  if (g.unit == SEP_UNIT_2TH_DEG) return tth * (180.0 / M_PI);
  return 4.0 * M_PI * sin(0.5 * tth) / (g.lam * 1.0e9);
}

// Area of the disc of radius R about the origin inside the quadrant
// rectangle [0, x] x [0, y] (x, y >= 0): the column under the circle,
// G(t) = integral_0^t sqrt(R^2 - u^2) du = (t sqrt(R^2 - t^2) + R^2 asin(t / R)) / 2.
inline double quadrant_area(double x, double y, double R) {
  if (R <= 0.0 || x <= 0.0 || y <= 0.0) return 0.0;
  auto G = [R](double t) { return 0.5 * (t * sqrt(std::max(R * R - t * t, 0.0)) + R * R * asin(std::min(t / R, 1.0))); };
  const double xc = std::min(x, R);
  if (y >= R) return G(xc);
  const double us = sqrt(R * R - y * y);   // where the circle leaves the top edge y
  if (xc <= us) return xc * y;
  return us * y + G(xc) - G(us);
}
// signed: the area in [0, x] x [0, y] with orientation sign(x) sign(y)
inline double corner_area(double x, double y, double R) {
  const double a = quadrant_area(fabs(x), fabs(y), R);
  return (x < 0) != (y < 0) ? -a : a;
}
// Area of the rectangle [x0, x1] x [y0, y1] inside the disc of radius R.
inline double rect_disc_area(double x0, double x1, double y0, double y1, double R) {
  if (!(R > 0.0)) return 0.0;
  if (isinf(R)) return (x1 - x0) * (y1 - y0);
  return corner_area(x1, y1, R) - corner_area(x0, y1, R) - corner_area(x1, y0, R) + corner_area(x0, y0, R);
}

inline int32_t bin_index(double x, double lo, double hi, int32_t B) {
  if (!(x >= lo && x <= hi)) return -1;
  double t = (x - lo) / (hi - lo) * (double)B;
  double fl = floor(t);
  int64_t b = (int64_t)fl;
  if (b >= B) b = B - 1;
  if (b < 0) b = 0;
  return (int32_t)b;
}

}  // namespace

std::string build_csr_host(const sep_geometry& gm, const uint8_t* mask, const float* norm, HostCsr* out) {
  const int64_t rows = gm.rows, cols = gm.cols;
  if (rows <= 0 || cols <= 0) return "rows and cols must be positive";
  if (rows * cols > (int64_t)SEP_MAX_PIXELS) return "rows * cols exceeds SEP_MAX_PIXELS";
  if (gm.nbins < 1 || gm.nbins > SEP_MAX_BINS) return "nbins out of range";
  if (gm.split != 0 && gm.split != 1 && gm.split != 2) return "split must be 0 (exact area), 1 or 2";
  if (gm.unit < 0 || gm.unit > 2) return "unknown unit";
  if (!(gm.dist_m > 0) || !(gm.pixel_m[0] > 0) || !(gm.pixel_m[1] > 0)) return "distance and pixel size must be > 0";
  if (gm.unit == SEP_UNIT_Q_NM && !(gm.wavelength_m > 0)) return "wavelength must be > 0 for q";
  const int64_t npix = rows * cols;
  // exact: area fractions (one weighted class); else s x s sub-pixel centres
  const bool exact = gm.split == 0;
  const int s = exact ? 1 : gm.split;
  Geo g{gm.pixel_m[0], gm.pixel_m[1], gm.dist_m, gm.center_px[0], gm.center_px[1], gm.wavelength_m, gm.unit};
  double off[2];
  for (int a = 0; a < s; ++a) off[a] = ((double)a + 0.5) / (double)s;

  if (norm) {
    for (int64_t i = 0; i < npix; ++i)
      if ((!mask || !mask[i]) && !(norm[i] > 0.0f)) return "norm must be > 0 on valid pixels";
  }

  // range: automatic = min / max over valid sub-pixel centres
  double lo = gm.range[0], hi = gm.range[1];
  if (isnan(lo) || isnan(hi)) {
    double mn = std::numeric_limits<double>::infinity(), mx = -mn;
#pragma omp parallel for reduction(min : mn) reduction(max : mx) schedule(static)
    for (int64_t row = 0; row < rows; ++row)
      for (int64_t col = 0; col < cols; ++col) {
        if (mask && mask[row * cols + col]) continue;
        if (exact) {   // the whole pixel: its nearest and farthest points
          const double x0 = ((double)col - g.cx) * g.px, x1 = x0 + g.px;
          const double y0 = ((double)row - g.cy) * g.py, y1 = y0 + g.py;
          const double nx = x0 > 0 ? x0 : (x1 < 0 ? x1 : 0.0), ny = y0 > 0 ? y0 : (y1 < 0 ? y1 : 0.0);
          const double fx = std::max(fabs(x0), fabs(x1)), fy = std::max(fabs(y0), fabs(y1));
          const double a = unit_of(g, sqrt(nx * nx + ny * ny)), b = unit_of(g, sqrt(fx * fx + fy * fy));
          mn = a < mn ? a : mn;
          mx = b > mx ? b : mx;
          continue;
        }
        for (int a = 0; a < s; ++a)
          for (int b = 0; b < s; ++b) {
            double x = radial(g, row, col, off[a], off[b]);
            mn = x < mn ? x : mn;
            mx = x > mx ? x : mx;
          }
      }
    if (isnan(lo)) lo = mn;
    if (isnan(hi)) hi = mx;
  }
  if (!(hi > lo)) return "empty radial range (no valid pixel, or lo >= hi)";
  const int32_t B = gm.nbins;

  // per pixel: up to s*s (bin, k) pairs + centre bin (exact: up to kMaxExact
  // bins with their area fractions in pc, k = 1; a carrier has k = 0)
  constexpr int kMaxExact = 15;
  const int maxe = exact ? kMaxExact + 1 : s * s + 1;
  std::vector<int32_t> pb((size_t)npix * maxe, -1);
  std::vector<uint8_t> pk((size_t)npix * maxe, 0);
  std::vector<double> pc(exact ? (size_t)npix * maxe : 0, 0.0);
  int too_many = 0;
  std::vector<uint8_t> pn((size_t)npix, 0);
  std::vector<int32_t> bop((size_t)npix, -1);
  std::vector<float> xcen((size_t)npix, 0.0f);   // radial value of the pixel centre (staging order)
  out->interp_a.assign((size_t)npix, 0);
  out->interp_t.assign((size_t)npix, 0.0f);
#pragma omp parallel for schedule(static)
  for (int64_t row = 0; row < rows; ++row) {
    for (int64_t col = 0; col < cols; ++col) {
      const int64_t i = row * cols + col;
      if (mask && mask[i]) continue;
      // centre bin: the bin of the pixel centre, clamped into [0, B-1]
      double xc = radial(g, row, col, 0.5, 0.5);
      int32_t bc = xc < lo ? 0 : (xc > hi ? B - 1 : bin_index(xc, lo, hi, B));
      bop[i] = bc;
      xcen[i] = (float)xc;
      {
        // smooth profile: between the two bin centres around the pixel centre
        const double u = (xc - lo) / (hi - lo) * (double)B - 0.5;
        if (!(u > 0.0)) {
          out->interp_a[i] = 0;
          out->interp_t[i] = 0.0f;
        } else if (u >= (double)(B - 1)) {
          out->interp_a[i] = B - 1;
          out->interp_t[i] = 0.0f;
        } else {
          const double a = floor(u);
          out->interp_a[i] = (int32_t)a;
          out->interp_t[i] = (float)(u - a);
        }
      }
      if (exact) {
        int32_t* eb = &pb[(size_t)i * maxe];
        uint8_t* ek = &pk[(size_t)i * maxe];
        double* ec = &pc[(size_t)i * maxe];
        const double x0 = ((double)col - g.cx) * g.px, x1 = x0 + g.px;
        const double y0 = ((double)row - g.cy) * g.py, y1 = y0 + g.py;
        const double nx = x0 > 0 ? x0 : (x1 < 0 ? x1 : 0.0), ny = y0 > 0 ? y0 : (y1 < 0 ? y1 : 0.0);
        const double fx = std::max(fabs(x0), fabs(x1)), fy = std::max(fabs(y0), fabs(y1));
        const double umin = unit_of(g, sqrt(nx * nx + ny * ny)), umax = unit_of(g, sqrt(fx * fx + fy * fy));
        int n = 0;
        bool has_centre = false;
        if (umax >= lo && umin <= hi) {
          const int32_t b0 = bin_index(std::max(umin, lo), lo, hi, B), b1 = bin_index(std::min(umax, hi), lo, hi, B);
          const double area = g.px * g.py;
          for (int32_t b = b0; b <= b1 && b >= 0; ++b) {
            const double elo = lo + (hi - lo) * (double)b / (double)B;
            const double ehi = lo + (hi - lo) * (double)(b + 1) / (double)B;
            const double c = (rect_disc_area(x0, x1, y0, y1, radius_of(g, ehi)) -
                              rect_disc_area(x0, x1, y0, y1, radius_of(g, elo))) / area;
            if (!(c > 1e-12)) continue;
            if (n == kMaxExact) {
#pragma omp atomic write
              too_many = 1;
              break;
            }
            eb[n] = b;
            ek[n] = 1;
            ec[n] = std::min(c, 1.0);
            ++n;
            if (b == bc) has_centre = true;
          }
        }
        if (!has_centre) {   // threshold carrier of zero weight, kept in bin order
          int p = n;
          while (p > 0 && eb[p - 1] > bc) {
            eb[p] = eb[p - 1];
            ek[p] = ek[p - 1];
            ec[p] = ec[p - 1];
            --p;
          }
          eb[p] = bc;
          ek[p] = 0;
          ec[p] = 0.0;
          ++n;
        }
        pn[i] = (uint8_t)n;
        continue;
      }
      int32_t sb[4];
      int m = 0;
      for (int a = 0; a < s; ++a)
        for (int b = 0; b < s; ++b) sb[m++] = bin_index(radial(g, row, col, off[a], off[b]), lo, hi, B);
      for (int x = 1; x < m; ++x)   // m <= 4: insertion sort
        for (int y = x; y > 0 && sb[y - 1] > sb[y]; --y) std::swap(sb[y - 1], sb[y]);
      int32_t* eb = &pb[(size_t)i * maxe];
      uint8_t* ek = &pk[(size_t)i * maxe];
      int n = 0;
      bool has_centre = false;
      for (int t = 0; t < m; ++t) {
        if (sb[t] < 0) continue;
        if (n > 0 && eb[n - 1] == sb[t]) {
          ek[n - 1] += 1;
        } else {
          eb[n] = sb[t];
          ek[n] = 1;
          ++n;
        }
        if (sb[t] == bc) has_centre = true;
      }
      if (!has_centre) {  // threshold carrier of zero weight, kept in bin order
        int p = n;
        while (p > 0 && eb[p - 1] > bc) {
          eb[p] = eb[p - 1];
          ek[p] = ek[p - 1];
          --p;
        }
        eb[p] = bc;
        ek[p] = 0;
        ++n;
      }
      pn[i] = (uint8_t)n;
    }
  }

  if (too_many) return "exact area fractions: a pixel spans more than 15 bins (bins far narrower than pixels)";

  // Staging order of the pixels: grouped by tiles of kTileH x kTileW and,
  // inside a tile, by centre bin (then radius, then pixel index). Only
  // pixels with at least one entry take part. It orders the entries inside
  // every coefficient group of a row (below), so the entries of one bin in
  // one tile are consecutive.
  {
    const int64_t tx = (cols + kTileW - 1) / kTileW, ty = (rows + kTileH - 1) / kTileH;
    out->tiles_x = (int32_t)tx;
    out->tiles_y = (int32_t)ty;
    out->tile_base.assign((size_t)(tx * ty) + 1, 0);
    out->tile_rank.assign((size_t)npix, (int16_t)-1);
    out->perm_inv.clear();
    out->perm_inv.reserve((size_t)npix);
    std::vector<int32_t> pos_of((size_t)npix, -1);
    struct Px { int32_t bin; float x; int32_t i; };
    std::vector<Px> tile_px;
    tile_px.reserve((size_t)kTileH * kTileW);
    for (int64_t t = 0; t < tx * ty; ++t) {
      const int64_t r0 = (t / tx) * kTileH, c0 = (t % tx) * kTileW;
      tile_px.clear();
      for (int64_t r = r0; r < std::min<int64_t>(r0 + kTileH, rows); ++r)
        for (int64_t c = c0; c < std::min<int64_t>(c0 + kTileW, cols); ++c) {
          const int64_t i = r * cols + c;
          if (pn[i] > 0) tile_px.push_back({bop[i], xcen[i], (int32_t)i});
        }
      // by centre bin, then radius: the pixels of a bin that spill into the
      // next (previous) bin sit at the end (start) of its run, next to that bin
      std::sort(tile_px.begin(), tile_px.end(), [](const Px& a, const Px& b) {
        if (a.bin != b.bin) return a.bin < b.bin;
        if (a.x != b.x) return a.x < b.x;
        return a.i < b.i;
      });
      out->tile_base[t] = (int32_t)out->perm_inv.size();
      for (size_t k = 0; k < tile_px.size(); ++k) {
        const int32_t i = tile_px[k].i;
        out->tile_rank[i] = (int16_t)k;
        pos_of[i] = (int32_t)out->perm_inv.size();
        out->perm_inv.push_back(i);
      }
    }
    out->tile_base[tx * ty] = (int32_t)out->perm_inv.size();
    out->pos_of = pos_of;
    out->npos = (int64_t)out->perm_inv.size();
  }

  // Row layout (one row per bin): entries grouped by coefficient class,
  // largest coefficient first (class c holds k = s*s - c sub-pixels, c = 0 ..
  // s*s - 1), then the weight-0 centre carriers; inside a group the entries
  // follow the staging order, so those of one staging tile form a run. Each
  // run is padded with flagged entries to a multiple of kRunAlign (8) slots:
  // the staging kernel, which writes a tile's runs into the frame's staged
  // row (slot = entry), then writes whole 32-byte sectors. Groups and rows
  // hold multiples of 8 entries, so the kernels move 4 entries per vector
  // access and apply a class's weight once per group.
  constexpr int64_t kRunAlign = 8;
  const int NC = s * s + 1;                 // coefficient classes + carriers
  struct Ent {
    uint64_t key;   // (bin * NC + class) << 32 | staging position
    int64_t i;      // pixel
    int t;          // its entry
  };
  std::vector<Ent> all;
  {
    int64_t n_real = 0;
    for (int64_t i = 0; i < npix; ++i) n_real += pn[i];
    all.reserve((size_t)n_real);
  }
  for (int64_t i = 0; i < npix; ++i)
    for (int t = 0; t < pn[i]; ++t) {
      const int32_t b = pb[(size_t)i * maxe + t];
      const int k = pk[(size_t)i * maxe + t];
      const int c = k == 0 ? NC - 1 : s * s - k;
      all.push_back({((uint64_t)((int64_t)b * NC + c) << 32) | (uint32_t)out->pos_of[i], i, t});
    }
  std::sort(all.begin(), all.end(), [](const Ent& x, const Ent& y) { return x.key < y.key; });
  auto tile_of = [&](int64_t i) { return (i / cols) / kTileH * (int64_t)out->tiles_x + (i % cols) / kTileW; };
  // slots: entries and their runs' padding, row by row
  out->rowptr.assign((size_t)B + 1, 0);
  out->grp.assign((size_t)B * 4, 0);
  std::vector<int64_t> slot_of_ent(all.size());
  int64_t pos = 0;
  int32_t max_row = 0;
  {
    size_t j = 0;
    for (int32_t b = 0; b < B; ++b) {
      const int64_t r0 = pos;
      for (int c = 0; c < NC; ++c) {
        const uint64_t g = (uint64_t)((int64_t)b * NC + c);
        int64_t run_tile = -1;
        while (j < all.size() && (all[j].key >> 32) == g) {
          const int64_t tl = tile_of(all[j].i);
          if (tl != run_tile) {   // a new run starts on a sector boundary
            pos = (pos + kRunAlign - 1) / kRunAlign * kRunAlign;
            run_tile = tl;
          }
          slot_of_ent[j++] = pos++;
        }
        pos = (pos + kRunAlign - 1) / kRunAlign * kRunAlign;
        if (c < 4) out->grp[(size_t)b * 4 + c] = (int32_t)(pos - r0);
      }
      for (int c = NC - 1; c < 4; ++c) out->grp[(size_t)b * 4 + c] = out->grp[(size_t)b * 4 + (NC - 2)];
      if (pos > (int64_t)std::numeric_limits<int32_t>::max()) return "too many nonzeros";
      out->rowptr[b + 1] = (int32_t)pos;
      max_row = std::max(max_row, (int32_t)(pos - r0));
    }
  }
  const int64_t nnz = pos;
  out->ent.assign((size_t)nnz, kPad);
  out->coef.assign((size_t)nnz, 0.0f);
  if (norm || exact) out->w.assign((size_t)nnz, 0.0f);   // per-entry weights c * norm
  const double inv = 1.0 / (double)(s * s);
  for (size_t j = 0; j < all.size(); ++j) {
    const int64_t i = all[j].i;
    const int t = all[j].t;
    const int32_t b = pb[(size_t)i * maxe + t];
    const int k = pk[(size_t)i * maxe + t];
    const int64_t e = slot_of_ent[j];
    uint32_t u = (uint32_t)i;
    if (k == 0) u |= kZero;
    else u |= (uint32_t)(k - 1) << kKShift;
    if (b == bop[i]) u |= kCentre;
    out->ent[e] = u;
    const double cf = exact ? pc[(size_t)i * maxe + t] : (double)k * inv;
    out->coef[e] = (float)cf;
    if (norm || exact) out->w[e] = (float)(cf * (norm ? (double)norm[i] : 1.0));
  }
  // per entry: its pixel if the entry carries the pixel's centre bin (one
  // such entry per pixel with entries), else -1; the clip kernel marks kept
  // pixels through these, and the consumers read a pixel's staged value at
  // its centre entry's slot
  out->cpix.assign((size_t)nnz, -1);
  out->slot_of.assign((size_t)npix, -1);
  for (int64_t e = 0; e < nnz; ++e) {
    const uint32_t u = out->ent[e];
    if ((u & kCentre) && !(u & kPad)) {
      out->cpix[(size_t)e] = (int32_t)(u & kColMask);
      out->slot_of[u & kColMask] = (int32_t)e;
    }
  }
  // Staged copy of a frame: one value per entry, in row order (slot e holds
  // entry e's pixel value; padding slots hold NaN). The staging kernel works
  // by image tiles: each tile lists the slots of its pixels' entries in
  // ascending order with the pixel's index inside the tile (row * kTileW +
  // column), -1 for the padding slots of its runs (a run's padding follows
  // its entries, so the tile writes whole sectors).
  {
    const int64_t tx = out->tiles_x, nt = (int64_t)out->tiles_x * out->tiles_y;
    std::vector<int32_t> slot_tile((size_t)nnz, 0);
    for (int64_t e = 0, cur = 0; e < nnz; ++e) {
      const uint32_t u = out->ent[(size_t)e];
      if (!(u & kPad)) {
        const int64_t i = u & kColMask, r = i / cols, c = i % cols;
        cur = (r / kTileH) * tx + c / kTileW;
      }
      slot_tile[(size_t)e] = (int32_t)cur;
    }
    auto tile_of = [&](int64_t e) -> int64_t { return slot_tile[(size_t)e]; };
    (void)nt;
    out->tile_ebase.assign((size_t)nt + 1, 0);
    for (int64_t e = 0; e < nnz; ++e) out->tile_ebase[(size_t)tile_of(e) + 1] += 1;
    for (int64_t t = 0; t < nt; ++t) out->tile_ebase[(size_t)t + 1] += out->tile_ebase[(size_t)t];
    std::vector<int64_t> fill_t(out->tile_ebase.begin(), out->tile_ebase.end() - 1);
    out->tile_sc.assign((size_t)nnz * 2, -1);
    for (int64_t e = 0; e < nnz; ++e) {
      const int64_t t = tile_of(e), k = fill_t[(size_t)t]++;
      const uint32_t u = out->ent[(size_t)e];
      int32_t loc = -1;
      if (!(u & kPad)) {
        const int64_t i = u & kColMask;
        loc = (int32_t)((i / cols) % kTileH * kTileW + (i % cols) % kTileW);
      }
      out->tile_sc[(size_t)k * 2] = (int32_t)e;
      out->tile_sc[(size_t)k * 2 + 1] = loc;
    }
  }
  out->rows = gm.rows;
  out->cols = gm.cols;
  out->nbins = B;
  out->split = gm.split;   // 0: exact area fractions
  out->lo = lo;
  out->hi = hi;
  out->max_row = max_row;
  out->bop.swap(bop);
  out->centers.resize(B);
  for (int32_t b = 0; b < B; ++b) out->centers[b] = (float)(lo + ((double)b + 0.5) * (hi - lo) / (double)B);
  // a matrix the kernels cannot follow safely never leaves the host
  const std::string why = validate_host_csr(*out);
  return why.empty() ? why : "internal matrix check failed: " + why;
}


// Matrix in the export layout (Section 2.2's CSR: rows are bins; col -1 marks
// a padding slot). Every index the kernels follow is checked against the
// array it indexes; the first violation is returned.
std::string validate_matrix(const int32_t* rowptr, const int32_t* col, const float* coef, const int32_t* bop,
                            int32_t nbins, int64_t nnz, int64_t npix) {
  auto at = [](const char* what, int64_t i) { return std::string(what) + " at " + std::to_string(i); };
  if (nbins <= 0) return "nbins must be > 0";
  if (nnz < 0 || npix <= 0) return "nnz must be >= 0 and npix > 0";
  if (!rowptr) return "rowptr is NULL";
  if (nnz > 0 && (!col || !coef)) return "col / coef is NULL";
  if (rowptr[0] != 0) return "rowptr[0] != 0";
  for (int32_t b = 0; b < nbins; ++b)
    if (rowptr[b + 1] < rowptr[b]) return at("rowptr decreases (non-monotone row pointer) at bin", b);
  if ((int64_t)rowptr[nbins] != nnz) return "rowptr[nbins] differs from nnz";
  // coefficients of one pixel over all bins sum to its area share, at most 1
  std::vector<double> area((size_t)npix, 0.0);
  for (int64_t e = 0; e < nnz; ++e) {
    const int32_t c = col[e];
    const float w = coef[e];
    if (c < -1 || (int64_t)c >= npix) return at("column out of range [-1, npix) at entry", e);
    if (!(w >= 0.0f && w <= 1.0f)) return at("coefficient outside [0, 1] at entry", e);
    if (c == -1) {
      if (w != 0.0f) return at("padding slot with a nonzero coefficient at entry", e);
      continue;
    }
    area[(size_t)c] += w;
  }
  for (int64_t i = 0; i < npix; ++i)
    if (area[(size_t)i] > 1.0 + 1e-6) return at("coefficients of a pixel sum above 1 at pixel", i);
  if (bop)
    for (int64_t i = 0; i < npix; ++i)
      if (bop[i] < -1 || bop[i] >= nbins) return at("bin_of_pixel out of range [-1, nbins) at pixel", i);
  return std::string();
}

// The packed layout the kernels read: the matrix checks above on its
// exported view, then the kernel-side tables (class ends, centre entries,
// staging tables).
std::string validate_host_csr(const HostCsr& h) {
  const int64_t npix = (int64_t)h.rows * h.cols, nnz = (int64_t)h.ent.size();
  if ((int64_t)h.rowptr.size() != (int64_t)h.nbins + 1) return "rowptr size differs from nbins + 1";
  if ((int64_t)h.coef.size() != nnz || (int64_t)h.cpix.size() != nnz) return "entry tables differ in size";
  if ((int64_t)h.bop.size() != npix) return "bin_of_pixel size differs from npix";
  std::vector<int32_t> col((size_t)nnz);
  for (int64_t e = 0; e < nnz; ++e) {
    const uint32_t u = h.ent[(size_t)e];
    col[(size_t)e] = (u & kPad) ? -1 : (int32_t)(u & kColMask);
  }
  std::string why = validate_matrix(h.rowptr.data(), col.data(), h.coef.data(), h.bop.data(), h.nbins, nnz, npix);
  if (!why.empty()) return why;
  if ((int64_t)h.grp.size() != 4 * (int64_t)h.nbins) return "class table size differs from 4 nbins";
  for (int32_t b = 0; b < h.nbins; ++b) {
    const int32_t n = h.rowptr[b + 1] - h.rowptr[b];
    if (n % 4) return "row length not a multiple of 4 at bin " + std::to_string(b);
    int32_t prev = 0;
    for (int c = 0; c < 4; ++c) {
      const int32_t g = h.grp[(size_t)b * 4 + c];
      if (g < prev || g > n || g % 4) return "class ends out of order at bin " + std::to_string(b);
      prev = g;
    }
  }
  for (int64_t e = 0; e < nnz; ++e)
    if (h.cpix[(size_t)e] < -1 || h.cpix[(size_t)e] >= npix) return "centre entry pixel out of range at " + std::to_string(e);
  if ((int64_t)h.slot_of.size() != npix) return "centre slot table size differs from npix";
  for (int64_t i = 0; i < npix; ++i)
    if (h.slot_of[(size_t)i] < -1 || h.slot_of[(size_t)i] >= nnz) return "centre slot out of range at pixel " + std::to_string(i);
  if (h.tile_ebase.empty() || h.tile_ebase.front() != 0 || (int64_t)h.tile_ebase.back() * 2 != (int64_t)h.tile_sc.size())
    return "staging scatter table bounds";
  for (size_t t = 0; t + 1 < h.tile_ebase.size(); ++t)
    if (h.tile_ebase[t + 1] < h.tile_ebase[t]) return "staging scatter table decreases at tile " + std::to_string(t);
  for (size_t k = 0; k < h.tile_sc.size(); k += 2) {
    if (h.tile_sc[k] < 0 || h.tile_sc[k] >= nnz) return "staging slot out of range";
    if (h.tile_sc[k + 1] < -1 || h.tile_sc[k + 1] >= kTileH * kTileW) return "staging tile index out of range";
  }
  return std::string();
}
}  // namespace sep
