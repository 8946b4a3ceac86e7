// Film probe of the rupture criterion (Sec. 3.1 / Sec. 4 of the paper) as a
// device routine over any accessor with rho(x,y,z) and p(x,y,z) in FP64
// (wrapped coordinates are the accessor's job).
//
// Along `len` cells from c0 in direction e: x1 = first upward crossing of
// rho_mid, x2 = next downward crossing (linear interpolation), h = x2 - x1;
// d2p/dn2 at the nearest line cell to the midpoint (mean of the two cells
// when exactly half-way); R_d = half the number of rows along ep, contiguous
// with the midpoint row, whose liquid run along e through the midpoint
// column is no thicker than h + 2.  out = {found, x1, x2, h, d2p_mid, R_d}.
#pragma once

#include <stdint.h>

namespace sclbm {

template <class Acc>
__device__ double film_run_thickness(const Acc &acc, int64_t x, int64_t y, int64_t z,
                                     const int *e, double mid, int64_t maxlen) {
  if (acc.rho(x, y, z) < mid) return -1.0;
  double lo = 0, hi = 0;
  int64_t m;
  for (m = 1; m <= maxlen; ++m) {
    const double ra = acc.rho(x - (m - 1) * e[0], y - (m - 1) * e[1], z - (m - 1) * e[2]);
    const double rb = acc.rho(x - m * e[0], y - m * e[1], z - m * e[2]);
    if (rb < mid) {
      lo = -((double)(m - 1) + (mid - ra) / (rb - ra));
      break;
    }
  }
  if (m > maxlen) return -1.0;
  for (m = 1; m <= maxlen; ++m) {
    const double ra = acc.rho(x + (m - 1) * e[0], y + (m - 1) * e[1], z + (m - 1) * e[2]);
    const double rb = acc.rho(x + m * e[0], y + m * e[1], z + m * e[2]);
    if (rb < mid) {
      hi = (double)(m - 1) + (mid - ra) / (rb - ra);
      break;
    }
  }
  if (m > maxlen) return -1.0;
  return hi - lo;
}

template <class Acc>
__device__ void film_probe_dev(const Acc &acc, int64_t x0, int64_t y0, int64_t z0, const int *e,
                               const int *ep, int64_t len, double mid, double *out) {
  for (int q = 0; q < 6; ++q) out[q] = 0.0;
  double x1 = -1, x2 = -1;
  int64_t m;
  for (m = 1; m < len; ++m) {
    const double ra = acc.rho(x0 + (m - 1) * e[0], y0 + (m - 1) * e[1], z0 + (m - 1) * e[2]);
    const double rb = acc.rho(x0 + m * e[0], y0 + m * e[1], z0 + m * e[2]);
    if (ra < mid && rb >= mid) {
      x1 = (double)(m - 1) + (mid - ra) / (rb - ra);
      break;
    }
  }
  if (x1 < 0) return;
  for (++m; m < len; ++m) {
    const double ra = acc.rho(x0 + (m - 1) * e[0], y0 + (m - 1) * e[1], z0 + (m - 1) * e[2]);
    const double rb = acc.rho(x0 + m * e[0], y0 + m * e[1], z0 + m * e[2]);
    if (ra >= mid && rb < mid) {
      x2 = (double)(m - 1) + (ra - mid) / (ra - rb);
      break;
    }
  }
  if (x2 < 0) return;
  const double h = x2 - x1, xm = 0.5 * (x1 + x2), fl = floor(xm);
  const int64_t c = (int64_t)fl;
  auto d2 = [&](int64_t cc) {
    return acc.p(x0 + (cc + 1) * e[0], y0 + (cc + 1) * e[1], z0 + (cc + 1) * e[2]) -
           2.0 * acc.p(x0 + cc * e[0], y0 + cc * e[1], z0 + cc * e[2]) +
           acc.p(x0 + (cc - 1) * e[0], y0 + (cc - 1) * e[1], z0 + (cc - 1) * e[2]);
  };
  const double dmid = xm - fl == 0.5 ? 0.5 * (d2(c) + d2(c + 1)) : d2(xm - fl < 0.5 ? c : c + 1);
  const int64_t cm = (int64_t)floor(xm + 0.5);
  const int64_t xc = x0 + cm * e[0], yc = y0 + cm * e[1], zc = z0 + cm * e[2];
  int64_t extent = 0;
  for (int sg = -1; sg <= 1; sg += 2) {
    for (int64_t j = (sg < 0 ? 1 : 0); j <= len; ++j) {
      const double t = film_run_thickness(acc, xc + sg * j * ep[0], yc + sg * j * ep[1],
                                          zc + sg * j * ep[2], e, mid, len);
      if (t < 0 || t > h + 2.0) break;
      ++extent;
    }
  }
  out[0] = 1.0;
  out[1] = x1;
  out[2] = x2;
  out[3] = h;
  out[4] = dmid;
  out[5] = 0.5 * (double)extent;
}

}  // namespace sclbm
