// Film probe of the rupture criterion (Sec. 3.1 / Sec. 4 of the paper) as a
// CTA-wide device routine over any accessor with rho(x,y,z) and p(x,y,z) in
// FP64 (wrapped coordinates are the accessor's job).
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


// Every thread of the CTA calls it with the same arguments; thread 0 writes
// out.  Crossings and disc rows are searched in parallel chunks: each
// candidate is evaluated exactly as a sequential scan would evaluate it, and
// the first hit is a block-wide minimum, so the result equals the
// sequential scan's.
template <class Acc>
__device__ void film_probe_block(const Acc &acc, int64_t x0, int64_t y0, int64_t z0,
                                 const int *e, const int *ep, int64_t len, double mid,
                                 double *out) {
  __shared__ unsigned long long s_first;
  const int tid = threadIdx.x, nt = blockDim.x;
  const unsigned long long NONE = ~0ull;
  auto rho_at = [&](int64_t m) { return acc.rho(x0 + m * e[0], y0 + m * e[1], z0 + m * e[2]); };
  // first m in [lo, hi) with hit(m), or NONE; block-uniform
  auto first = [&](int64_t lo, int64_t hi, auto hit) -> unsigned long long {
    for (int64_t m0 = lo; m0 < hi; m0 += nt) {
      if (tid == 0) s_first = NONE;
      __syncthreads();
      const int64_t m = m0 + tid;
      if (m < hi && hit(m)) atomicMin(&s_first, (unsigned long long)m);
      __syncthreads();
      const unsigned long long f = s_first;
      __syncthreads();
      if (f != NONE) return f;
    }
    return NONE;
  };
  if (tid == 0)
    for (int q = 0; q < 6; ++q) out[q] = 0.0;
  const unsigned long long m1 = first(1, len, [&](int64_t m) {
    return rho_at(m - 1) < mid && rho_at(m) >= mid;
  });
  if (m1 == NONE) return;
  const unsigned long long m2 = first((int64_t)m1 + 1, len, [&](int64_t m) {
    return rho_at(m - 1) >= mid && rho_at(m) < mid;
  });
  if (m2 == NONE) return;
  double ra = rho_at((int64_t)m1 - 1), rb = rho_at((int64_t)m1);
  const double x1 = (double)((int64_t)m1 - 1) + (mid - ra) / (rb - ra);
  ra = rho_at((int64_t)m2 - 1);
  rb = rho_at((int64_t)m2);
  const double x2 = (double)((int64_t)m2 - 1) + (ra - mid) / (ra - rb);
  const double h = x2 - x1, xm = 0.5 * (x1 + x2), fl = floor(xm);
  const int64_t c = (int64_t)fl;
  auto d2 = [&](int64_t cc) {
    return acc.p(x0 + (cc + 1) * e[0], y0 + (cc + 1) * e[1], z0 + (cc + 1) * e[2]) -
           2.0 * acc.p(x0 + cc * e[0], y0 + cc * e[1], z0 + cc * e[2]) +
           acc.p(x0 + (cc - 1) * e[0], y0 + (cc - 1) * e[1], z0 + (cc - 1) * e[2]);
  };
  const int64_t cm = (int64_t)floor(xm + 0.5);
  const int64_t xc = x0 + cm * e[0], yc = y0 + cm * e[1], zc = z0 + cm * e[2];
  // rows of the disc: the first row (outward from the midpoint row) whose
  // liquid run is missing or thicker than h + 2 ends it on each side.  A run
  // whose crossing on either side lies beyond floor(h + 2) + 1 cells is
  // thicker than h + 2 whether or not a crossing follows within len, so the
  // walks stop there: the same decisions as walking len cells, at a bounded
  // cost for rows outside the disc.
  const int64_t walk = (int64_t)floor(h + 2.0) + 2 < len ? (int64_t)floor(h + 2.0) + 2 : len;
  auto fails = [&](int sg) {
    return [&, sg](int64_t j) {
      const double t = film_run_thickness(acc, xc + sg * j * ep[0], yc + sg * j * ep[1],
                                          zc + sg * j * ep[2], e, mid, walk);
      return t < 0 || t > h + 2.0;
    };
  };
  const unsigned long long fp = first(0, len + 1, fails(1));
  const unsigned long long fm = first(1, len + 1, fails(-1));
  const int64_t extent = (fp == NONE ? len + 1 : (int64_t)fp) + (fm == NONE ? len : (int64_t)fm - 1);
  if (tid == 0) {
    out[0] = 1.0;
    out[1] = x1;
    out[2] = x2;
    out[3] = h;
    out[4] = xm - fl == 0.5 ? 0.5 * (d2(c) + d2(c + 1)) : d2(xm - fl < 0.5 ? c : c + 1);
    out[5] = 0.5 * (double)extent;
  }
}

}  // namespace sclbm
