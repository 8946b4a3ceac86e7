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

// Accessors give rho(x,y,z) and p(x,y,z) in FP64, and below(x,y,z,mid): the
// decision rho < mid exactly as the FP64 rho makes it.  The crossings are
// found with below(); only the cells around a crossing are read in FP64.
// first m in 1..maxlen with a gas cell at (x, y, z) + sg m e, or -1; four
// cells a round, their reads independent of one another
template <class Acc>
__device__ int64_t film_edge(const Acc &acc, int64_t x, int64_t y, int64_t z, const int *e,
                             int sg, double mid, int64_t maxlen) {
  for (int64_t m0 = 1; m0 <= maxlen; m0 += 4) {
    bool g[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t m = m0 + q;
      g[q] = m <= maxlen &&
             acc.below(x + sg * m * e[0], y + sg * m * e[1], z + sg * m * e[2], mid);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (g[q]) return m0 + q;
  }
  return -1;
}

// Thickness of the liquid run through (x, y, z) along e, its crossings of
// mid interpolated (FP64) between the last liquid and the first gas cell at
// ml cells back and mh cells ahead.
template <class Acc>
__device__ double film_run_between(const Acc &acc, int64_t x, int64_t y, int64_t z, const int *e,
                                   double mid, int64_t ml, int64_t mh) {
  double ra = acc.rho(x - (ml - 1) * e[0], y - (ml - 1) * e[1], z - (ml - 1) * e[2]);
  double rb = acc.rho(x - ml * e[0], y - ml * e[1], z - ml * e[2]);
  const double lo = -((double)(ml - 1) + (mid - ra) / (rb - ra));
  ra = acc.rho(x + (mh - 1) * e[0], y + (mh - 1) * e[1], z + (mh - 1) * e[2]);
  rb = acc.rho(x + mh * e[0], y + mh * e[1], z + mh * e[2]);
  const double hi = (double)(mh - 1) + (mid - ra) / (rb - ra);
  return hi - lo;
}

// Does the row through (x, y, z) end the disc: no liquid run there within
// maxlen cells either way, or one thicker than limit?  Each interpolated
// crossing lies within its cell pair, so the thickness lies in
// [ml + mh - 2, ml + mh]; it is interpolated in FP64 only when that range
// does not decide the comparison.
template <class Acc>
__device__ bool film_row_fails(const Acc &acc, int64_t x, int64_t y, int64_t z, const int *e,
                               double mid, int64_t maxlen, double limit) {
  if (acc.below(x, y, z, mid)) return true;
  const int64_t ml = film_edge(acc, x, y, z, e, -1, mid, maxlen);
  if (ml < 0) return true;
  const int64_t mh = film_edge(acc, x, y, z, e, 1, mid, maxlen);
  if (mh < 0) return true;
  if ((double)(ml + mh) < limit - 1e-6) return false;
  if ((double)(ml + mh - 2) > limit + 1e-6) return true;
  return film_run_between(acc, x, y, z, e, mid, ml, mh) > limit;
}


// Every thread of the CTA calls it with the same arguments; thread 0 writes
// out.  Crossings and disc rows are searched in parallel chunks: each
// candidate is evaluated exactly as a sequential scan would evaluate it, and
// the first hit is a block-wide minimum, so the result equals the
// sequential scan's.  need_disc(h, d2p), evaluated by every thread on the
// same values, says whether R_d is wanted: when it is not, the disc rows are
// not scanned and out[5] = -1 (the other outputs are unchanged).
template <class Acc, class NeedDisc>
__device__ void film_probe_block(const Acc &acc, int64_t x0, int64_t y0, int64_t z0,
                                 const int *e, const int *ep, int64_t len, double mid,
                                 double *out, NeedDisc need_disc) {
  __shared__ unsigned long long s_first;
  const int tid = threadIdx.x, nt = blockDim.x;
  const unsigned long long NONE = ~0ull;
  auto rho_at = [&](int64_t m) { return acc.rho(x0 + m * e[0], y0 + m * e[1], z0 + m * e[2]); };
  auto gas_at = [&](int64_t m) { return acc.below(x0 + m * e[0], y0 + m * e[1], z0 + m * e[2], mid); };
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
    return gas_at(m - 1) && !gas_at(m);
  });
  if (m1 == NONE) return;
  const unsigned long long m2 = first((int64_t)m1 + 1, len, [&](int64_t m) {
    return !gas_at(m - 1) && gas_at(m);
  });
  if (m2 == NONE) return;
  // the FP64 densities around the two crossings, one thread each
  __shared__ double s_v[8];
  if (tid < 4) s_v[tid] = rho_at(tid < 2 ? (int64_t)m1 - 1 + tid : (int64_t)m2 - 3 + tid);
  __syncthreads();
  double ra = s_v[0], rb = s_v[1];
  const double x1 = (double)((int64_t)m1 - 1) + (mid - ra) / (rb - ra);
  ra = s_v[2];
  rb = s_v[3];
  const double x2 = (double)((int64_t)m2 - 1) + (ra - mid) / (ra - rb);
  const double h = x2 - x1, xm = 0.5 * (x1 + x2), fl = floor(xm);
  const int64_t c = (int64_t)fl;
  // pressures of the line cells c - 1 .. c + 2, one thread each; d2(cc) for
  // cc = c or c + 1 combines them in the order p(cc+1) - 2 p(cc) + p(cc-1)
  if (tid < 4) s_v[4 + tid] = acc.p(x0 + (c - 1 + tid) * e[0], y0 + (c - 1 + tid) * e[1],
                                    z0 + (c - 1 + tid) * e[2]);
  __syncthreads();
  auto d2 = [&](int64_t cc) {
    const double *q = s_v + 4 + (cc - c);
    return q[2] - 2.0 * q[1] + q[0];
  };
  const double d2p = xm - fl == 0.5 ? 0.5 * (d2(c) + d2(c + 1)) : d2(xm - fl < 0.5 ? c : c + 1);
  if (!need_disc(h, d2p)) {
    if (tid == 0) {
      out[0] = 1.0;
      out[1] = x1;
      out[2] = x2;
      out[3] = h;
      out[4] = d2p;
      out[5] = -1.0;
    }
    return;
  }
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
      return film_row_fails(acc, xc + sg * j * ep[0], yc + sg * j * ep[1], zc + sg * j * ep[2],
                            e, mid, walk, h + 2.0);
    };
  };
  // the first failing row on each side (side +1: rows 0..len, side -1: rows
  // 1..len), both sides at once on the two halves of the CTA; each side's
  // first hit is its own block-wide minimum, as in first()
  __shared__ unsigned long long s_two[2];
  unsigned long long fp = NONE, fm = NONE;
  {
    const int half = nt / 2, sd = tid < half ? 0 : 1, t = tid - sd * half;
    bool dp = false, dm = false;  // side settled; block-uniform
    for (int64_t k0 = 0;; k0 += half) {
      const bool scan_p = !dp && k0 <= len, scan_m = !dm && 1 + k0 <= len;
      if (!scan_p && !scan_m) break;
      if (tid == 0) s_two[0] = s_two[1] = NONE;
      __syncthreads();
      const int64_t j = sd + k0 + t;
      if ((sd == 0 ? scan_p : scan_m) && j <= len && fails(sd == 0 ? 1 : -1)(j))
        atomicMin(&s_two[sd], (unsigned long long)j);
      __syncthreads();
      const unsigned long long hp = s_two[0], hm = s_two[1];
      __syncthreads();
      if (scan_p && hp != NONE) fp = hp;
      if (scan_m && hm != NONE) fm = hm;
      dp = dp || !scan_p || hp != NONE;
      dm = dm || !scan_m || hm != NONE;
    }
  }
  const int64_t extent = (fp == NONE ? len + 1 : (int64_t)fp) + (fm == NONE ? len : (int64_t)fm - 1);
  if (tid == 0) {
    out[0] = 1.0;
    out[1] = x1;
    out[2] = x2;
    out[3] = h;
    out[4] = d2p;
    out[5] = 0.5 * (double)extent;
  }
}

template <class Acc>
__device__ void film_probe_block(const Acc &acc, int64_t x0, int64_t y0, int64_t z0,
                                 const int *e, const int *ep, int64_t len, double mid,
                                 double *out) {
  film_probe_block(acc, x0, y0, z0, e, ep, len, mid, out, [](double, double) { return true; });
}

}  // namespace sclbm
