// State conversion and diagnostics kernels, all in FP64 arithmetic:
// initial state, population gather/scatter, moments, EOS pressure and its
// Laplacian (the rupture criterion of Sec. 3.1 / Sec. 4 of the paper), FP64
// totals, and connected-component labelling of gas cells.
//
// Stored populations are in push form: stored_i(x) = f_i(x, t).
#include <type_traits>

#include "film.cuh"
#include "internal.h"
#include "lattice.cuh"

namespace sclbm {

namespace {

struct Idx {
  int x, y, z;
};
// Lattices hold fewer than 2^31 cells (lbm_create), so cell indices and
// their decomposition use 32-bit arithmetic: a 64-bit division is a long
// emulated sequence on the GPU, partly on the narrow FP64 pipe.
__device__ __forceinline__ Idx idx_of(int64_t k, const View &v) {
  Idx c;
  const uint32_t kk = (uint32_t)k, nx = (uint32_t)v.NX, ny = (uint32_t)v.NY;
  const uint32_t r = fdiv(kk, v.fx, nx);
  c.x = (int)(kk - r * nx);
  const uint32_t zq = fdiv(r, v.fy, ny);
  c.y = (int)(r - zq * ny);
  c.z = (int)zq;
  return c;
}
// periodic wrap: one add or subtract for a neighbour's coordinate, the
// remainder only for coordinates further out
__device__ __forceinline__ int wr(int a, int n) {
  if (a >= n) a -= n;
  else if (a < 0) a += n;
  if ((unsigned)a >= (unsigned)n) {
    a %= n;
    if (a < 0) a += n;
  }
  return a;
}
__device__ __forceinline__ int64_t lin(int x, int y, int z, const View &v) {
  return (int64_t)(((uint32_t)z * (uint32_t)v.NY + (uint32_t)y) * (uint32_t)v.NX + (uint32_t)x);
}
__device__ __forceinline__ int64_t sidx(int i, int x, int y, int z, const View &v) {
  return (int64_t)i * v.px * v.NY * v.NZ + ((int64_t)z * v.NY + y) * v.px + x;
}

template <int ST>
__device__ __forceinline__ double load_d(const void *p, int64_t k, double wref) {
  return decode_f<ST>(static_cast<const typename Storage<ST>::T *>(p)[k], wref);
}
// f_i at cell (x, y, z) in double: the stored value, and for population 0 of
// a lattice that keeps a rounding residual, that residual too (added last,
// so a view without one gets the same bits as load_d)
template <int ST>
__device__ __forceinline__ double pop_d(const View &v, const void *p, int i, int x, int y, int z,
                                        double wref) {
  const int64_t k = sidx(i, x, y, z, v);
  double f = load_d<ST>(p, k, wref);
  if (i == 0 && v.resid) f = __dadd_rn(f, (double)v.resid[k]);
  return f;
}
template <int ST>
__device__ __forceinline__ void store_d(void *p, int64_t k, double v, double wref) {
  static_cast<typename Storage<ST>::T *>(p)[k] = encode_f<ST>(v, wref);
}

// SplitMix64 (Steele, Lea & Flood 2014): the k-th output of the generator
// whose state starts at key.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t key, uint64_t k) {
  uint64_t z = key + (k + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

constexpr int TPB = 256;
inline int nblocks(int64_t n) {
  const int64_t b = (n + TPB - 1) / TPB;
  return (int)(b < 1 ? 1 : (b > 262144 ? 262144 : b));
}
#define GRID_LOOP(k, n) \
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < (n); \
       k += (int64_t)gridDim.x * blockDim.x)

__device__ __forceinline__ double min_image(double d, double n) {
  d = fmod(d, n);
  if (d < 0) d += n;
  if (d > 0.5 * n) d -= n;
  return d;
}

// Initial density.  The nearest bubble (smallest distance minus radius) is
// found with FP32 distances, then every bubble within 1e-3 of that FP32
// minimum is re-evaluated in FP64 with the exact formula, so the result
// equals the all-FP64 minimum (FP32 distance errors are < 1e-4 here).
__device__ __forceinline__ float min_image_f(float d, float n) {
  d = fmodf(d, n);
  if (d < 0) d += n;
  if (d > 0.5f * n) d -= n;
  return d;
}
// signed FP32 distance from the point (px, py, pz) to bubble b's surface
__device__ __forceinline__ float bubble_dist_f(float px, float py, float pz, const double *b,
                                               float nxf, float nyf, float nzf) {
  const float dx = min_image_f(px - (float)b[0], nxf);
  const float dy = min_image_f(py - (float)b[1], nyf);
  const float dz = min_image_f(pz - (float)b[2], nzf);
  return sqrtf(dx * dx + dy * dy + dz * dz) - (float)b[3];
}

// One block per brick of cells (8 x 8 x 8; 16 x 16 in the D2Q9 view).  The
// block first keeps the bubbles that can matter to any of its cells.  With
// c the brick's centre, h its half-diagonal and d_c the smallest signed
// distance from c, every cell x of the brick has a bubble within d_c + h,
// and a bubble b within that of x has d_c(b) <= d_x(b) + h <= d_c + 2h
// (the periodic distance is a metric).  The margin covers the FP32 errors
// and the 1e-3 window of the FP64 re-evaluation, so each cell meets the
// same bubbles as in a scan of all of them.  A brick with more candidates
// than the list holds scans all bubbles.
constexpr int INIT_CAND = 1024;
__global__ void __launch_bounds__(TPB) k_init_rho(const View v, int bx, int by, int bz,
                                                  const double *bub, int32_t nb, double rho_l,
                                                  double rho_g, double width, double amp,
                                                  uint64_t key, double *rho) {
  __shared__ int cand[INIT_CAND];
  __shared__ int ncand;
  __shared__ float wmin[TPB / 32];
  const int NX = (int)v.NX, NY = (int)v.NY, NZ = (int)v.NZ;
  const int nbx = (NX + bx - 1) / bx, nby = (NY + by - 1) / by;
  const int ix = (int)(blockIdx.x % (unsigned)nbx);
  const int r1 = (int)(blockIdx.x / (unsigned)nbx);
  const int iy = r1 % nby, iz = r1 / nby;
  const int x0 = ix * bx, y0 = iy * by, z0 = iz * bz;
  const int ex = min(bx, NX - x0), ey = min(by, NY - y0), ez = min(bz, NZ - z0);
  const float nxf = (float)v.NX, nyf = (float)v.NY, nzf = (float)v.NZ;
  bool use_all = true;
  if (nb > 0) {
    const float cx = (float)x0 + 0.5f * (float)(ex - 1);
    const float cy = (float)y0 + 0.5f * (float)(ey - 1);
    const float cz = (float)z0 + 0.5f * (float)(ez - 1);
    const float h = 0.5f * sqrtf((float)((ex - 1) * (ex - 1) + (ey - 1) * (ey - 1) +
                                         (ez - 1) * (ez - 1)));
    float m = INFINITY;
    for (int b = threadIdx.x; b < nb; b += TPB)
      m = fminf(m, bubble_dist_f(cx, cy, cz, bub + 4 * b, nxf, nyf, nzf));
    for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = m;
    if (threadIdx.x == 0) ncand = 0;
    __syncthreads();
    float dc = wmin[0];
    for (int w = 1; w < TPB / 32; ++w) dc = fminf(dc, wmin[w]);
    const float t0 = dc + 2.0f * h;
    for (int b = threadIdx.x; b < nb; b += TPB) {
      const float d = bubble_dist_f(cx, cy, cz, bub + 4 * b, nxf, nyf, nzf);
      if (d - t0 <= 0.05f + 1e-6f * (fabsf(d) + fabsf((float)bub[4 * b + 3]) + fabsf(t0))) {
        const int q = atomicAdd(&ncand, 1);
        if (q < INIT_CAND) cand[q] = b;
      }
    }
    __syncthreads();
    use_all = ncand > INIT_CAND;
  }
  const int nc = use_all ? nb : ncand;
  const int cells = ex * ey * ez;
  for (int t = threadIdx.x; t < cells; t += TPB) {
    const int x = x0 + t % ex, y = y0 + (t / ex) % ey, z = z0 + t / (ex * ey);
    const int64_t k = ((int64_t)z * NY + y) * NX + x;
    double r = rho_l;
    if (nb > 0) {
      float s32 = INFINITY;
      for (int j = 0; j < nc; ++j) {
        const int b = use_all ? j : cand[j];
        s32 = fminf(s32, bubble_dist_f((float)x, (float)y, (float)z, bub + 4 * b, nxf, nyf, nzf));
      }
      double s = INFINITY;
      for (int j = 0; j < nc; ++j) {
        const int b = use_all ? j : cand[j];
        if (bubble_dist_f((float)x, (float)y, (float)z, bub + 4 * b, nxf, nyf, nzf) > s32 + 1e-3f)
          continue;
        const double dx = min_image((double)x - bub[4 * b + 0], (double)v.NX);
        const double dy = min_image((double)y - bub[4 * b + 1], (double)v.NY);
        const double dz = min_image((double)z - bub[4 * b + 2], (double)v.NZ);
        const double d =
            __dadd_rn(sqrt(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz))),
                      -bub[4 * b + 3]);
        s = d < s ? d : s;
      }
      r = rho_g + 0.5 * (rho_l - rho_g) * (1.0 + tanh(2.0 * s / width));
    }
    if (amp != 0.0) {
      const double u = (double)(splitmix64_at(key, (uint64_t)k) >> 11) * (1.0 / 9007199254740992.0);
      r += amp * (2.0 * u - 1.0);
    }
    rho[k] = r;
  }
}

template <int LAT, int ST>
__global__ void k_store_from(const View v, const double *src, int from_f, void *stored) {
  using L = Lattice<LAT>;
  const int64_t N = v.NX * v.NY * v.NZ;
  GRID_LOOP(k, N) {
    const Idx c = idx_of(k, v);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const double val = from_f ? src[(int64_t)i * N + k] : L::w(i) * src[k];
      store_d<ST>(stored, sidx(i, c.x, c.y, c.z, v), val, L::w(i) * v.rho_ref);
    }
  }
}

template <int LAT, int ST>
__global__ void k_gather_f(const View v, const void *stored, double *f) {
  using L = Lattice<LAT>;
  const int64_t N = v.NX * v.NY * v.NZ;
  GRID_LOOP(k, N) {
    const Idx c = idx_of(k, v);
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
      f[(int64_t)i * N + k] = pop_d<ST>(v, stored, i, c.x, c.y, c.z, L::w(i) * v.rho_ref);
  }
}

// one population: out(x) = f_i(x) = stored_i(x)
template <int LAT, int ST>
__global__ void k_gather_pop(const View v, const void *stored, int i, double *out) {
  using L = Lattice<LAT>;
  int cx = 0, cy = 0, cz = 0;
  double w = 0;
#pragma unroll
  for (int m = 0; m < L::Q; ++m)
    if (m == i) {
      cx = L::cx(m);
      cy = L::cy(m);
      cz = L::cz(m);
      w = L::w(m);
    }
  const int64_t N = v.NX * v.NY * v.NZ;
  GRID_LOOP(k, N) {
    const Idx c = idx_of(k, v);
    out[k] = pop_d<ST>(v, stored, i, c.x, c.y, c.z, w * v.rho_ref);
  }
}

// one population: stored_i(x) = f_i(x) from canonical f_i (N doubles)
template <int LAT, int ST>
__global__ void k_store_pop(const View v, const double *f, int i, void *stored) {
  using L = Lattice<LAT>;
  int cx = 0, cy = 0, cz = 0;
  double w = 0;
#pragma unroll
  for (int m = 0; m < L::Q; ++m)
    if (m == i) {
      cx = L::cx(m);
      cy = L::cy(m);
      cz = L::cz(m);
      w = L::w(m);
    }
  const int64_t N = v.NX * v.NY * v.NZ;
  GRID_LOOP(k, N) {
    const Idx c = idx_of(k, v);
    store_d<ST>(stored, sidx(i, c.x, c.y, c.z, v), f[k], w * v.rho_ref);
  }
}

// per-cell FP64 moments (sum in velocity order) in the view's axes
template <int LAT, int ST>
__device__ __forceinline__ void cell_moments(const View &v, const void *stored, const Idx &c,
                                             double &rho, double &jx, double &jy, double &jz) {
  using L = Lattice<LAT>;
  rho = jx = jy = jz = 0.0;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const double f = pop_d<ST>(v, stored, i, c.x, c.y, c.z, L::w(i) * v.rho_ref);
    rho += f;
    jx += L::cx(i) * f;
    jy += L::cy(i) * f;
    jz += L::cz(i) * f;
  }
}

// density alone, in the same order (and so the same bits) as cell_moments
template <int LAT, int ST>
__device__ __forceinline__ double cell_rho(const View &v, const void *stored, int x, int y, int z) {
  using L = Lattice<LAT>;
  double rho = 0.0;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) rho += pop_d<ST>(v, stored, i, x, y, z, L::w(i) * v.rho_ref);
  return rho;
}

// FP64 EOS pressure p = rho/3 + G/6 psi^2, psi = rho0 (1 - exp(-rho/rho0))
__device__ __forceinline__ double eos_p(double r, double G, double rho0) {
  const double s = rho0 * (1.0 - exp(-r / rho0));
  return r / 3.0 + G / 6.0 * s * s;
}

template <int LAT, int ST, bool J>
__global__ void k_moments(const View v, const void *stored, double G, double rho0, double *rho,
                          double *jx, double *jy, double *jz, double *psi, double *p, int *err) {
  const int64_t N = v.NX * v.NY * v.NZ;
  bool bad = false;
  GRID_LOOP(k, N) {
    const Idx c = idx_of(k, v);
    double r, a = 0, b = 0, d = 0;
    if (J)
      cell_moments<LAT, ST>(v, stored, c, r, a, b, d);
    else
      r = cell_rho<LAT, ST>(v, stored, c.x, c.y, c.z);
    if (!isfinite(r)) bad = true;
    const double s = rho0 * (1.0 - exp(-r / rho0));
    if (rho) rho[k] = r;
    if (jx) jx[k] = a;
    if (jy) jy[k] = b;
    if (jz) jz[k] = d;
    if (psi) psi[k] = s;
    if (p) p[k] = eos_p(r, G, rho0);
  }
  if (bad && err) atomicOr(err, ERR_NONFINITE);
}

template <int LAT>
__global__ void k_velocity(const View v, double G, const double *rho, const double *jx,
                           const double *jy, const double *jz, const double *psi, double *u) {
  using L = Lattice<LAT>;
  const int64_t N = v.NX * v.NY * v.NZ;
  GRID_LOOP(k, N) {
    const Idx c = idx_of(k, v);
    double sx = 0, sy = 0, sz = 0;
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
      const double wp = L::w(i) * psi[lin(wr(c.x + L::cx(i), (int)v.NX),
                                          wr(c.y + L::cy(i), (int)v.NY),
                                          wr(c.z + L::cz(i), (int)v.NZ), v)];
      sx += L::cx(i) * wp;
      sy += L::cy(i) * wp;
      sz += L::cz(i) * wp;
    }
    const double gp = -G * psi[k];
    const double ux = (jx[k] + 0.5 * gp * sx) / rho[k];
    const double uy = (jy[k] + 0.5 * gp * sy) / rho[k];
    const double uz = (jz[k] + 0.5 * gp * sz) / rho[k];
    if (LAT == D2Q9) {  // view (x, 1, y) -> user (x, y)
      u[k] = ux;
      u[N + k] = uz;
      u[2 * N + k] = 0.0;
    } else {
      u[k] = ux;
      u[N + k] = uy;
      u[2 * N + k] = uz;
    }
  }
}

__global__ void k_laplacian(const View v, const double *p, double *lap) {
  const int64_t N = v.NX * v.NY * v.NZ;
  GRID_LOOP(k, N) {
    const Idx c = idx_of(k, v);
    const double pc = p[k];
    double s = p[lin(wr(c.x + 1, (int)v.NX), c.y, c.z, v)] - 2.0 * pc +
               p[lin(wr(c.x - 1, (int)v.NX), c.y, c.z, v)];
    s += p[lin(c.x, wr(c.y + 1, (int)v.NY), c.z, v)] - 2.0 * pc +
         p[lin(c.x, wr(c.y - 1, (int)v.NY), c.z, v)];
    s += p[lin(c.x, c.y, wr(c.z + 1, (int)v.NZ), v)] - 2.0 * pc +
         p[lin(c.x, c.y, wr(c.z - 1, (int)v.NZ), v)];
    lap[k] = s;
  }
}

__global__ void k_line_d2(const View v, const double *p, int x0, int y0, int z0, int axis,
                          int64_t len, double *out) {
  GRID_LOOP(m, len) {
    const int ex = axis == 0, ey = axis == 1, ez = axis == 2;
    const int x = wr((int)(x0 + m * ex), (int)v.NX), y = wr((int)(y0 + m * ey), (int)v.NY),
              z = wr((int)(z0 + m * ez), (int)v.NZ);
    out[m] = p[lin(wr(x + ex, (int)v.NX), wr(y + ey, (int)v.NY), wr(z + ez, (int)v.NZ), v)] -
             2.0 * p[lin(x, y, z, v)] +
             p[lin(wr(x - ex, (int)v.NX), wr(y - ey, (int)v.NY), wr(z - ez, (int)v.NZ), v)];
  }
}

// Fixed-order FP64 block sums: block b sums a fixed set of cells in a fixed
// tree, so repeated calls give identical bits.
constexpr int TOT_BLOCKS = 1024;
template <int LAT, int ST>
__global__ void __launch_bounds__(TPB) k_totals(const View v, const void *stored, double *part) {
  __shared__ double sh[4][TPB];
  const int64_t N = v.NX * v.NY * v.NZ;
  double m = 0, a = 0, b = 0, d = 0;
  for (int64_t k = blockIdx.x * (int64_t)TPB + threadIdx.x; k < N; k += (int64_t)TOT_BLOCKS * TPB) {
    double r, x, y, z;
    cell_moments<LAT, ST>(v, stored, idx_of(k, v), r, x, y, z);
    m += r;
    a += x;
    b += y;
    d += z;
  }
  sh[0][threadIdx.x] = m;
  sh[1][threadIdx.x] = a;
  sh[2][threadIdx.x] = b;
  sh[3][threadIdx.x] = d;
  __syncthreads();
  for (int w = TPB / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 4; ++q) part[4 * blockIdx.x + q] = sh[q][0];
}

template <int LAT>
__global__ void __launch_bounds__(TPB) k_totals_final(const double *part, double *out) {
  __shared__ double sh[4][TPB];
  double acc[4] = {0, 0, 0, 0};
  for (int b = threadIdx.x; b < TOT_BLOCKS; b += TPB)
    for (int q = 0; q < 4; ++q) acc[q] += part[4 * b + q];
  for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int w = TPB / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sh[0][0];
    out[1] = sh[1][0];
    if (LAT == D2Q9) {  // view (x, 1, y) -> user (x, y)
      out[2] = sh[3][0];
      out[3] = 0.0;
    } else {
      out[2] = sh[2][0];
      out[3] = sh[3][0];
    }
  }
}

// ---- one pass for the diagnostic interval (FP32-arithmetic storages) -------
// The offsets g_i are summed with an error-free FP32 transformation (TwoSum,
// Knuth TAOCP vol. 2, 4.2.2) into a per-thread pair (hi, lo): every addition
// to hi is exact, its rounding error goes to lo.  Every SCAN_FLUSH cells
// hi + lo is added to the thread's FP64 accumulator (FP64 is a narrow pipe
// on this part: two FP64 operations per cell instead of sixteen); threads
// and blocks are combined in FP64 in a fixed order, so the mass
// (N rho_ref + sum of offsets) is an FP64 reduction that repeated calls
// reproduce bit for bit.  Momentum (sum g c_i; the w_i rho_ref part cancels)
// is reduced the same way.
// The gas decision rho < threshold is taken in FP64, exactly as the FP64
// moments of the decoded populations would take it, whenever the FP32
// density is within 1e-5 of the threshold; elsewhere hi decides.
constexpr int SCAN_BLOCKS = 1024;
constexpr int SCAN_FLUSH = 8;
__device__ __forceinline__ void two_sum(float &hi, float &lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float err = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += err;
}
template <int LAT, int ST>
__global__ void __launch_bounds__(TPB) k_scan(const View v, const void *stored, double thr,
                                              int32_t *labels, double *part, int *err) {
  using L = Lattice<LAT>;
  using S = Storage<ST>;
  using T = typename S::T;
  __shared__ double sh[4][TPB];
  const int64_t N = v.NX * v.NY * v.NZ;
  const int64_t pop = v.px * v.NY * v.NZ;
  const T *f = static_cast<const T *>(stored);
  const float rho_ref = (float)v.rho_ref, thr_f = (float)thr;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  float hi[4] = {0, 0, 0, 0}, lo[4] = {0, 0, 0, 0};
  int pending = 0;
  bool bad = false;
  for (int64_t k = blockIdx.x * (int64_t)TPB + threadIdx.x; k < N;
       k += (int64_t)SCAN_BLOCKS * TPB) {
    const Idx c = idx_of(k, v);
    const int64_t o = ((int64_t)c.z * v.NY + c.y) * v.px + c.x;
    float g[L::Q];
    float cell = 0.0f;  // the cell's FP32 offset sum, for the gas decision
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      g[i] = S::load(f[i * pop + o]);
      cell += g[i];
      two_sum(hi[0], lo[0], g[i]);
      if (L::cx(i) != 0) two_sum(hi[1], lo[1], L::cx(i) > 0 ? g[i] : -g[i]);
      if (L::cy(i) != 0) two_sum(hi[2], lo[2], L::cy(i) > 0 ? g[i] : -g[i]);
      if (L::cz(i) != 0) two_sum(hi[3], lo[3], L::cz(i) > 0 ? g[i] : -g[i]);
    }
    // a lattice with a rounding residual: it is part of the rest population
    const float res = v.resid ? v.resid[o] : 0.0f;
    if (v.resid) {
      cell += res;
      two_sum(hi[0], lo[0], res);
    }
    if (!isfinite(cell)) bad = true;
    if (labels) {
      const float r32 = rho_ref + cell;
      bool gas;
      if (fabsf(r32 - thr_f) > 1e-5f) {
        gas = r32 < thr_f;
      } else {
        double r64 = 0;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) r64 += __dadd_rn(__dmul_rn(L::w(i), v.rho_ref), (double)g[i]);
        if (v.resid) r64 = __dadd_rn(r64, (double)res);
        gas = r64 < thr;
      }
      labels[k] = gas ? (int32_t)k : -1;
    }
    if (++pending == SCAN_FLUSH) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[q] += (double)hi[q] + (double)lo[q];
        hi[q] = lo[q] = 0.0f;
      }
      pending = 0;
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q] += (double)hi[q] + (double)lo[q];
  if (bad && err) atomicOr(err, ERR_NONFINITE);
  if (!part) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int w = TPB / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 4; ++q) part[4 * blockIdx.x + q] = sh[q][0];
}

template <int LAT>
__global__ void __launch_bounds__(TPB) k_scan_final(const double *part, double mass0, double *out) {
  __shared__ double sh[4][TPB];
  double a[4] = {0, 0, 0, 0};
  for (int b = threadIdx.x; b < SCAN_BLOCKS; b += TPB)
    for (int q = 0; q < 4; ++q) a[q] += part[4 * b + q];
  for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] = a[q];
  __syncthreads();
  for (int w = TPB / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = mass0 + sh[0][0];
    out[1] = sh[1][0];
    if (LAT == D2Q9) {  // view (x, 1, y) -> user (x, y)
      out[2] = sh[3][0];
      out[3] = 0.0;
    } else {
      out[2] = sh[2][0];
      out[3] = sh[3][0];
    }
  }
}

// ---- connected components (union-find, links always from the larger root
// to the smaller, so every root is its component's minimum index) ---------
__device__ __forceinline__ int32_t uf_find(const int32_t *L, int32_t x) {
  int32_t p = L[x];
  while (p != x) {
    x = p;
    p = L[x];
  }
  return x;
}
__device__ __forceinline__ void uf_union(int32_t *L, int32_t a, int32_t b) {
  bool done = false;
  while (!done) {
    a = uf_find(L, a);
    b = uf_find(L, b);
    if (a < b) {
      const int32_t old = atomicMin(&L[b], a);
      done = old == b;
      b = old;
    } else if (b < a) {
      const int32_t old = atomicMin(&L[a], b);
      done = old == a;
      a = old;
    } else {
      done = true;
    }
  }
}

__global__ void k_ccl_init(int64_t N, const double *rho, double thr, int32_t *L) {
  GRID_LOOP(k, N) L[k] = rho[k] < thr ? (int32_t)k : -1;
}
// (gas or liquid is fixed before the pass: only gas entries change)
__global__ void k_ccl_union(const View v, int32_t *L) {
  const int64_t N = v.NX * v.NY * v.NZ;
  quad_pass(N, L, [&](int64_t k, int32_t lk) {
    if (lk < 0) return;
    const Idx c = idx_of(k, v);
    const int64_t nbr[3] = {lin(wr(c.x + 1, (int)v.NX), c.y, c.z, v),
                            lin(c.x, wr(c.y + 1, (int)v.NY), c.z, v),
                            lin(c.x, c.y, wr(c.z + 1, (int)v.NZ), v)};
    for (int q = 0; q < 3; ++q) {
      const int64_t m = nbr[q];
      if (m != k && L[m] >= 0) uf_union(L, (int32_t)k, (int32_t)m);
    }
  });
}
__global__ void k_ccl_compress(int64_t N, int32_t *L, unsigned long long *ncomp) {
  unsigned int roots = 0;
  quad_pass(N, L, [&](int64_t k, int32_t lk) {
    if (lk < 0) return;
    const int32_t r = uf_find(L, (int32_t)k);
    L[k] = r;
    roots += (r == (int32_t)k);
  });
  if (roots) atomicAdd(ncomp, (unsigned long long)roots);
}
__global__ void k_gather_labels(const int32_t *L, const int32_t *cells, int32_t n, int32_t *out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) out[s] = L[cells[s]];
}


// ---- film test at every lattice point (Sec. 4) -------------------------------
using FilmRec = lbm_film_cell;  // written as the C ABI hands it out

// One thread per cell.  For each lattice axis: walk to the first gas cell on
// each side (at most h_max cells), classify film / midpoint, and update the
// arming bit of (cell, axis) as the two-bubble criterion does.  The FP64
// pressure of a midpoint and its two neighbours along the axis is computed
// from their populations (the bits diag_moments would store).  Records: the
// fired (cell, axis) pairs (slot counts[3]); with all_mid, every midpoint
// instead (slot counts[4], axis | fired << 8).
template <int LAT, int ST>
__global__ void __launch_bounds__(TPB)
    k_film_cells(const View v, const int32_t *labels, const void *stored, double G, double rho0,
                 int h_max, double eps_arm, uint8_t *state, unsigned long long *counts,
                 int64_t cap, FilmRec *rec, int all_mid) {
  __shared__ unsigned long long sh[4];
  if (threadIdx.x < 4) sh[threadIdx.x] = 0;
  __syncthreads();
  const int64_t N = v.NX * v.NY * v.NZ;
  const int naxes = v.lat == D2Q9 ? 2 : 3;
  unsigned long long nfilm = 0, nmid = 0, narmed = 0;
  GRID_LOOP(k, N) {
    const Idx c = idx_of(k, v);
    const int x = c.x, y = c.y, z = c.z;
    uint8_t st = state[k];
    const bool liquid = labels[k] < 0;
    for (int ua = 0; ua < naxes; ++ua) {
      // user axis ua -> view axis (D2Q9: x, z)
      const int va = v.lat == D2Q9 && ua == 1 ? 2 : ua;
      const int n_a = va == 0 ? (int)v.NX : (va == 1 ? (int)v.NY : (int)v.NZ);
      const int c_a = va == 0 ? x : (va == 1 ? y : z);
      // periodic coordinate along the axis: |s| <= h_max, so one add or
      // subtract suffices unless the axis is shorter than h_max (tiny
      // lattices only take the remainder)
      auto wrap_a = [&](int q) -> int {
        if (q >= n_a) q -= n_a;
        else if (q < 0) q += n_a;
        if ((unsigned)q >= (unsigned)n_a) q = ((q % n_a) + n_a) % n_a;
        return q;
      };
      // the cell s steps along the axis: the cell's own index plus s strides,
      // one period added or removed at the seam (|s| <= h_max < n_a; axes no
      // longer than h_max take the general wrap)
      const int stride = va == 0 ? 1 : (va == 1 ? (int)v.NX : (int)(v.NX * v.NY));
      const int period = n_a * stride;
      const bool short_axis = n_a <= h_max;
      auto cell_at = [&](int s) -> int64_t {
        if (!short_axis) {
          const int q = c_a + s;
          int idx = (int)k + s * stride;
          if (q >= n_a) idx -= period;
          else if (q < 0) idx += period;
          return idx;
        }
        const int q = wrap_a(c_a + s);
        const int xx = va == 0 ? q : x, yy = va == 1 ? q : y, zz = va == 2 ? q : z;
        return lin(xx, yy, zz, v);
      };
      auto p_at = [&](int s) -> double {
        const int q = wrap_a(c_a + s);
        const int xx = va == 0 ? q : x, yy = va == 1 ? q : y, zz = va == 2 ? q : z;
        return eos_p(cell_rho<LAT, ST>(v, stored, xx, yy, zz), G, rho0);
      };
      const uint8_t bit = (uint8_t)(1u << ua);
      bool mid = false;
      int32_t Lp = -1, Lm = -1;
      int dp = 0, dm = 0;
      if (liquid) {
        // first gas cell within h_max along +e (then -e): the labels of a
        // whole walk of FILM_CHUNK cells are loaded at once, so that a cell
        // with no gas near it waits for one round trip per direction
        constexpr int FILM_CHUNK = 12;
        auto first_gas = [&](int sign, int32_t &lab_out) -> int {
          for (int s0 = 1; s0 <= h_max; s0 += FILM_CHUNK) {
            int32_t lq[FILM_CHUNK];
#pragma unroll
            for (int q = 0; q < FILM_CHUNK; ++q)
              lq[q] = s0 + q <= h_max ? labels[cell_at(sign * (s0 + q))] : -1;
#pragma unroll
            for (int q = 0; q < FILM_CHUNK; ++q)
              if (lq[q] >= 0) {
                lab_out = lq[q];
                return s0 + q;
              }
          }
          return 0;
        };
        dp = first_gas(1, Lp);
        if (Lp >= 0) dm = first_gas(-1, Lm);
        const bool film = Lp >= 0 && Lm >= 0 && Lp != Lm && dp + dm - 1 <= h_max;
        nfilm += film;
        mid = film && dp - dm <= 1 && dm - dp <= 1;
      }
      if (!mid) {
        st = (uint8_t)(st & ~bit);
        continue;
      }
      ++nmid;
      const double d2 = p_at(1) - 2.0 * p_at(0) + p_at(-1);
      bool fired = false;
      if (d2 < -eps_arm) {
        st = (uint8_t)(st | bit);
      } else if ((st & bit) && d2 >= 0.0) {
        st = (uint8_t)(st & ~bit);
        fired = true;
      }
      unsigned long long q = ~0ull;
      if (all_mid) {
        // one atomic per warp for the midpoints recorded together
        const unsigned am = __activemask();
        const int lane = (int)(threadIdx.x & 31), leader = __ffs(am) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(&counts[4], (unsigned long long)__popc(am));
        base = __shfl_sync(am, base, leader);
        q = base + (unsigned long long)__popc(am & ((1u << lane) - 1u));
        if (fired) atomicAdd(&counts[3], 1ull);
      } else if (fired) {
        q = atomicAdd(&counts[3], 1ull);
      }
      if ((int64_t)q < cap && q != ~0ull) {
        FilmRec r;
        r.cell = k;
        r.axis = all_mid ? (ua | (fired ? 0x100 : 0)) : ua;
        r.label_minus = Lm;
        r.label_plus = Lp;
        r.thickness = dp + dm - 1;
        r.d2p = d2;
        rec[q] = r;
      }
    }
    state[k] = st;
    narmed += __popc((unsigned)st);
  }
  // every thread of the block reaches this point (grid-stride loop)
  const unsigned wf = __reduce_add_sync(0xffffffffu, (unsigned)nfilm);
  const unsigned wm = __reduce_add_sync(0xffffffffu, (unsigned)nmid);
  const unsigned wa = __reduce_add_sync(0xffffffffu, (unsigned)narmed);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&sh[0], (unsigned long long)wf);
    atomicAdd(&sh[1], (unsigned long long)wm);
    atomicAdd(&sh[2], (unsigned long long)wa);
  }
  __syncthreads();
  if (threadIdx.x < 3 && sh[threadIdx.x]) atomicAdd(&counts[threadIdx.x], sh[threadIdx.x]);
}

// ---- the film test along lattice lines (h_max <= 63; Sec. 4) ------------------
// The classification of k_film_cells, taken one lattice line at a time: the
// first gas cells on either side of a liquid cell are the two gas cells that
// close the liquid run holding it (periodically: the run through the line's
// end closes at its first gas cell).  A run is a film when its two gas cells
// carry different labels and it holds at most h_max cells; its midpoints are
// the cell at equal distance from both ends, or the two cells one apart.  The
// walk clears the axis bit of every cell it passes and queues each midpoint
// with its old bit, kept in a window of the walk's last 64 cells (for the
// run through the end: also of its first 64).  A second kernel takes the
// queued midpoints one per thread: the FP64 pressure, the criterion, the new
// bit and the record.  Midpoints beyond the queue's capacity are taken in
// the walk itself.  The counts, states and records equal k_film_cells'; the
// records come in another order (the callers sort them, or their order does
// not matter).
constexpr int FILM_LINE_HMAX = 63;

struct FilmArgs {
  View v;
  const int32_t *labels;
  const void *stored;
  double G, rho0, eps_arm;
  int h_max, all_mid;
  uint8_t *state;
  unsigned long long *counts;  // film, midpoints, armed, fired, midpoint slots, queued
  int64_t cap;
  FilmRec *rec;
  FilmMid *mids;  // the midpoint queue
  int64_t mid_cap;
};

// The criterion at the midpoint (cell k, user axis ua, old bit ob): the new
// bit, set in the state (atomically: the queue holds midpoints of every axis,
// and a cell's axes share its state byte), and the record.  Returns the new bit.
template <int LAT, int ST>
__device__ __noinline__ unsigned film_midpoint(const FilmArgs &A, int64_t k, int ua, int ob,
                                               int32_t lm, int32_t lp, int len) {
  const View &v = A.v;
  const Idx c = idx_of(k, v);
  const int va = LAT == D2Q9 && ua == 1 ? 2 : ua;
  const int n = (int)(va == 0 ? v.NX : (va == 1 ? v.NY : v.NZ));
  const int ca = va == 0 ? c.x : (va == 1 ? c.y : c.z);
  auto p_at = [&](int s) -> double {
    const int q = wr(ca + s, n);
    const int xx = va == 0 ? q : c.x, yy = va == 1 ? q : c.y, zz = va == 2 ? q : c.z;
    return eos_p(cell_rho<LAT, ST>(v, A.stored, xx, yy, zz), A.G, A.rho0);
  };
  const double d2 = p_at(1) - 2.0 * p_at(0) + p_at(-1);
  bool fired = false;
  int nb = ob;
  if (d2 < -A.eps_arm) {
    nb = 1;
  } else if (ob && d2 >= 0.0) {
    nb = 0;
    fired = true;
  }
  if (nb) {
    const uint64_t a = reinterpret_cast<uint64_t>(A.state + k);
    atomicOr(reinterpret_cast<unsigned *>(a & ~3ull), (1u << ua) << (8 * (unsigned)(a & 3)));
  }
  unsigned long long q = ~0ull;
  if (A.all_mid) {
    q = atomicAdd(&A.counts[4], 1ull);
    if (fired) atomicAdd(&A.counts[3], 1ull);
  } else if (fired) {
    q = atomicAdd(&A.counts[3], 1ull);
  }
  if ((int64_t)q < A.cap && q != ~0ull) {
    FilmRec r;
    r.cell = k;
    r.axis = A.all_mid ? (ua | (fired ? 0x100 : 0)) : ua;
    r.label_minus = lm;
    r.label_plus = lp;
    r.thickness = len;
    r.d2p = d2;
    A.rec[q] = r;
  }
  return (unsigned)nb;
}

// block sums of the film, midpoint and armed counts into counts[0..2]
__device__ __forceinline__ void film_counts_add(unsigned nfilm, unsigned nmid, unsigned narmed,
                                                unsigned long long *counts,
                                                unsigned long long *sh) {
  const unsigned wf = __reduce_add_sync(0xffffffffu, nfilm);
  const unsigned wm = __reduce_add_sync(0xffffffffu, nmid);
  const unsigned wa = __reduce_add_sync(0xffffffffu, narmed);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&sh[0], (unsigned long long)wf);
    atomicAdd(&sh[1], (unsigned long long)wm);
    atomicAdd(&sh[2], (unsigned long long)wa);
  }
  __syncthreads();
  if (threadIdx.x < 3 && sh[threadIdx.x]) atomicAdd(&counts[threadIdx.x], sh[threadIdx.x]);
}

// bits 0 .. j of a word (j <= 31)
__device__ __forceinline__ uint32_t low_bits(int j) {
  return j >= 31 ? 0xffffffffu : (2u << j) - 1u;
}

// The walk along one line: cell p at base + p * stride, n cells, user axis
// ua, taken cell by cell (step), or in groups of up to 32 cells (group): the
// group's gas cells and old bits as bit masks (bit j: cell p0 + j), its gas
// cells then one by one.
template <int LAT, int ST>
struct FilmWalk {
  int64_t base, stride;
  int n, ua, h;
  int f0 = -1, lf = 0, a = -1, la = 0;  // first and last gas cell so far, their labels
  uint64_t win = 0, first = 0;          // old bits: of cell p - j, of cell j
  unsigned nfilm = 0, nmid = 0, narmed = 0;

  // one cell: p, its label and state byte
  __device__ __forceinline__ void step(const FilmArgs &A, int p, int32_t lab, uint32_t st) {
    const uint64_t ob = (st >> ua) & 1u;
    win = (win << 1) | ob;
    if (p < 64) first |= ob << p;
    if (ob) A.state[base + (int64_t)p * stride] = (uint8_t)(st & ~(1u << ua));
    if (lab >= 0) {
      if (a >= 0)
        run(A, a, p, la, lab, win, false);
      else
        f0 = p, lf = lab;
      a = p;
      la = lab;
    }
  }
  // cells p0 .. p0 + cnt - 1: gas mask gm, old-bit mask om; lab(j), st(j):
  // label and state byte of cell p0 + j
  template <class Lab, class St>
  __device__ __forceinline__ void group(const FilmArgs &A, int p0, int cnt, uint32_t gm,
                                        uint32_t om, Lab lab, St st) {
    for (uint32_t m = om; m; m &= m - 1) {  // clear the old bits as the walk passes
      const int j = __ffs(m) - 1;
      A.state[base + (int64_t)(p0 + j) * stride] = (uint8_t)(st(j) & ~(1u << ua));
    }
    if (p0 < 64) first |= (uint64_t)om << p0;
    const uint64_t w0 = win;
    for (uint32_t m = gm; m; m &= m - 1) {
      const int j = __ffs(m) - 1, b = p0 + j;
      const int32_t lb = lab(j);
      if (a >= 0) {
        // old bits with cell b at bit 0
        const uint64_t wb = (w0 << (j + 1)) | (uint64_t)(__brev(om & low_bits(j)) >> (31 - j));
        run(A, a, b, la, lb, wb, false);
      } else {
        f0 = b;
        lf = lb;
      }
      a = b;
      la = lb;
    }
    win = (w0 << cnt) | (uint64_t)(__brev(om) >> (32 - cnt));
  }
  // the run from the last gas cell through the line's end to the first one
  __device__ __forceinline__ void finish(const FilmArgs &A) {
    if (f0 >= 0) run(A, a, f0 + n, la, lf, win, true);
  }
  // liquid cells a_ + 1 .. b - 1 between gas cells a_ and b (b may pass n);
  // w: old bits with the walk's current cell at bit 0 (b, or n - 1 at the end)
  __device__ __forceinline__ void run(const FilmArgs &A, int a_, int b, int32_t lm, int32_t lp,
                                      uint64_t w, bool wrap) {
    const int len = b - a_ - 1;
    if (len < 1 || len > h || lm == lp) return;
    nfilm += (unsigned)len;
    const int c1 = (a_ + b) >> 1;
    for (int c = c1; c <= c1 + ((a_ + b) & 1); ++c) {
      const int pos = c >= n ? c - n : c;
      uint64_t ob;
      if (!wrap)
        ob = (w >> (b - c)) & 1u;
      else if (c >= n)
        ob = (first >> pos) & 1u;
      else
        ob = (w >> (n - 1 - c)) & 1u;
      ++nmid;
      const int64_t k = base + (int64_t)pos * stride;
      const unsigned long long slot = atomicAdd(&A.counts[5], 1ull);
      if ((int64_t)slot < A.mid_cap)
        A.mids[slot] = FilmMid{k, lm, lp, ua | ((int)ob << 2) | (len << 3)};
      else
        narmed += film_midpoint<LAT, ST>(A, k, ua, (int)ob, lm, lp, len);
    }
  }
};

// Lines along x: one thread per row (y, z), FILM_ROWS rows per block.  The
// block stages FILM_COLS columns of its rows at a time: a warp reads one row's
// columns with one coalesced load per lane, and its ballots give the row's
// gas and old-bit masks; the labels go to shared memory (row padded against
// bank conflicts) for the gas cells the walk then takes.
constexpr int FILM_ROWS = 128, FILM_COLS = 32;
template <int LAT, int ST>
__global__ void __launch_bounds__(FILM_ROWS) k_film_rows(const __grid_constant__ FilmArgs A) {
  __shared__ int32_t slab[FILM_ROWS][FILM_COLS + 1];
  __shared__ uint32_t sgm[FILM_ROWS], som[FILM_ROWS];
  __shared__ unsigned long long sh[3];
  if (threadIdx.x < 3) sh[threadIdx.x] = 0;
  const int NX = (int)A.v.NX, rows = (int)(A.v.NY * A.v.NZ);
  const int r0 = blockIdx.x * FILM_ROWS, t = (int)threadIdx.x, row = r0 + t;
  const int lane = t & 31, wp = t >> 5;
  FilmWalk<LAT, ST> w;
  w.base = (int64_t)row * NX;
  w.stride = 1;
  w.n = NX;
  w.ua = 0;
  w.h = A.h_max;
  constexpr int RPW = FILM_ROWS / (FILM_ROWS / 32);  // rows staged per warp
  for (int c0 = 0; c0 < NX; c0 += FILM_COLS) {
    const int wd = min(FILM_COLS, NX - c0);
    __syncthreads();
#pragma unroll 8
    for (int u = 0; u < RPW; ++u) {
      const int rr = wp * RPW + u;
      int32_t lv = -1;
      uint32_t sv = 0;
      if (r0 + rr < rows && lane < wd) {
        const int64_t k = (int64_t)(r0 + rr) * NX + c0 + lane;
        lv = A.labels[k];
        sv = A.state[k];
      }
      const uint32_t gm = __ballot_sync(0xffffffffu, lv >= 0);
      const uint32_t om = __ballot_sync(0xffffffffu, sv & 1u);  // x is user axis 0
      slab[rr][lane] = lv;
      if (lane == 0) {
        sgm[rr] = gm;
        som[rr] = om;
      }
    }
    __syncthreads();
    if (row < rows) {
      const int32_t *lr = slab[t];
      const int64_t b0 = w.base + c0;
      w.group(A, c0, wd, sgm[t], som[t], [&](int j) { return lr[j]; },
              [&](int j) { return (uint32_t)A.state[b0 + j]; });
    }
  }
  if (row < rows) w.finish(A);
  film_counts_add(w.nfilm, w.nmid, w.narmed, A.counts, sh);
}

// Lines along view axis va (y, or z): one thread per line, x fastest across
// the threads, so that each step's loads are coalesced; FILM_AHEAD cells
// loaded ahead of their walk.
constexpr int FILM_AHEAD = 16;
template <int LAT, int ST>
__global__ void __launch_bounds__(TPB) k_film_cols(const __grid_constant__ FilmArgs A, int ua,
                                                   int va) {
  __shared__ unsigned long long sh[3];
  if (threadIdx.x < 3) sh[threadIdx.x] = 0;
  __syncthreads();
  const int NX = (int)A.v.NX, NY = (int)A.v.NY, NZ = (int)A.v.NZ;
  const int64_t nlines = (int64_t)NX * (va == 1 ? NZ : NY);
  const int64_t line = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  FilmWalk<LAT, ST> w;
  if (line < nlines) {
    const int o = (int)(line / NX);
    const int x = (int)(line - (int64_t)o * NX), y = va == 1 ? 0 : o, z = va == 1 ? o : 0;
    w.base = lin(x, y, z, A.v);
    w.stride = va == 1 ? (int64_t)NX : (int64_t)NX * NY;
    w.n = va == 1 ? NY : NZ;
    w.ua = ua;
    w.h = A.h_max;
    const int n = w.n;
    for (int p0 = 0; p0 < n; p0 += FILM_AHEAD) {
      int32_t lab[FILM_AHEAD];
      uint32_t st[FILM_AHEAD];
#pragma unroll
      for (int j = 0; j < FILM_AHEAD; ++j) {
        lab[j] = -1;
        st[j] = 0;
        if (p0 + j < n) {
          const int64_t k = w.base + (int64_t)(p0 + j) * w.stride;
          lab[j] = A.labels[k];
          st[j] = A.state[k];
        }
      }
#pragma unroll
      for (int j = 0; j < FILM_AHEAD; ++j)
        if (p0 + j < n) w.step(A, p0 + j, lab[j], st[j]);
    }
    w.finish(A);
  }
  film_counts_add(w.nfilm, w.nmid, w.narmed, A.counts, sh);
}

// The queued midpoints, one per thread (grid-stride over the queue's length).
template <int LAT, int ST>
__global__ void __launch_bounds__(TPB) k_film_mids(const __grid_constant__ FilmArgs A) {
  __shared__ unsigned long long sh[3];
  if (threadIdx.x < 3) sh[threadIdx.x] = 0;
  __syncthreads();
  const int64_t nq = (int64_t)min((unsigned long long)A.mid_cap, A.counts[5]);
  unsigned narmed = 0;
  GRID_LOOP(q, nq) {
    const FilmMid m = A.mids[q];
    narmed += film_midpoint<LAT, ST>(A, m.cell, m.meta & 3, (m.meta >> 2) & 1, m.label_minus,
                                     m.label_plus, m.meta >> 3);
  }
  film_counts_add(0u, 0u, narmed, A.counts, sh);
}


// ---- film probe on FP64 density and pressure fields -------------------------
struct FieldAcc {
  View v;
  const double *rho_f, *p_f;
  __device__ int64_t at(int64_t x, int64_t y, int64_t z) const {
    return lin(wr((int)(x % v.NX), (int)v.NX), wr((int)(y % v.NY), (int)v.NY),
               wr((int)(z % v.NZ), (int)v.NZ), v);
  }
  __device__ double rho(int64_t x, int64_t y, int64_t z) const { return rho_f[at(x, y, z)]; }
  __device__ double p(int64_t x, int64_t y, int64_t z) const { return p_f[at(x, y, z)]; }
  __device__ bool below(int64_t x, int64_t y, int64_t z, double mid) const {
    return rho(x, y, z) < mid;
  }
};
__global__ void k_film_probe(const View v, const double *rho, const double *p, int64_t x0,
                             int64_t y0, int64_t z0, int ex, int ey, int ez, int px_, int py_,
                             int pz_, int64_t len, double mid, double *out) {
  if (blockIdx.x != 0) return;
  const FieldAcc acc{v, rho, p};
  const int e[3] = {ex, ey, ez}, ep[3] = {px_, py_, pz_};
  film_probe_block(acc, x0, y0, z0, e, ep, len, mid, out);
}
}  // namespace

// ---- host wrappers ----------------------------------------------------------
// Calls fn(integral_constant<lattice>, integral_constant<storage>).
template <typename Fn>
static void dispatch(const View &v, Fn &&fn) {
  using D3 = std::integral_constant<int, D3Q19>;
  using D2 = std::integral_constant<int, D2Q9>;
  using F64 = std::integral_constant<int, ST_F64>;
  using F32 = std::integral_constant<int, ST_F32>;
  using F16 = std::integral_constant<int, ST_F16>;
  using B16 = std::integral_constant<int, ST_BF16>;
  if (v.lat == D3Q19) {
    switch (v.st) {
      case ST_F64: fn(D3{}, F64{}); break;
      case ST_F32: fn(D3{}, F32{}); break;
      case ST_F16: fn(D3{}, F16{}); break;
      default: fn(D3{}, B16{}); break;
    }
  } else {
    switch (v.st) {
      case ST_F64: fn(D2{}, F64{}); break;
      case ST_F32: fn(D2{}, F32{}); break;
      case ST_F16: fn(D2{}, F16{}); break;
      default: fn(D2{}, B16{}); break;
    }
  }
}

static int64_t ncells(const View &v) { return v.NX * v.NY * v.NZ; }

cudaError_t diag_init_rho(const View &v, const double *bub, int32_t nb, double rho_l,
                          double rho_g, double width, double noise_amp, uint64_t seed,
                          double *rho, cudaStream_t s) {
  // bricks of 8 x 8 x 8 cells, 16 x 16 in the D2Q9 view (NY == 1)
  const int bx = v.NY == 1 ? 16 : 8, by = v.NY == 1 ? 1 : 8, bz = v.NY == 1 ? 16 : 8;
  const int64_t nbricks = ((v.NX + bx - 1) / bx) * ((v.NY + by - 1) / by) * ((v.NZ + bz - 1) / bz);
  k_init_rho<<<(unsigned)nbricks, TPB, 0, s>>>(v, bx, by, bz, bub, nb, rho_l, rho_g, width,
                                               noise_amp, seed ^ 0x6E6F697365000000ull, rho);
  return cudaGetLastError();
}

static cudaError_t store_from(const View &v, const double *src, int from_f, void *stored,
                              cudaStream_t s) {
  dispatch(v, [&](auto L, auto S) {
    k_store_from<decltype(L)::value, decltype(S)::value>
        <<<nblocks(ncells(v)), TPB, 0, s>>>(v, src, from_f, stored);
  });
  return cudaGetLastError();
}
cudaError_t diag_store_from_f(const View &v, const double *f, void *stored, cudaStream_t s) {
  return store_from(v, f, 1, stored, s);
}
cudaError_t diag_store_from_rho(const View &v, const double *rho, void *stored, cudaStream_t s) {
  return store_from(v, rho, 0, stored, s);
}

cudaError_t diag_gather_f(const View &v, const void *stored, double *f, cudaStream_t s) {
  dispatch(v, [&](auto L, auto S) {
    k_gather_f<decltype(L)::value, decltype(S)::value>
        <<<nblocks(ncells(v)), TPB, 0, s>>>(v, stored, f);
  });
  return cudaGetLastError();
}

cudaError_t diag_gather_pop(const View &v, const void *stored, int i, double *out,
                            cudaStream_t s) {
  dispatch(v, [&](auto L, auto S) {
    k_gather_pop<decltype(L)::value, decltype(S)::value>
        <<<nblocks(ncells(v)), TPB, 0, s>>>(v, stored, i, out);
  });
  return cudaGetLastError();
}

cudaError_t diag_store_pop(const View &v, const double *f, int i, void *stored, cudaStream_t s) {
  dispatch(v, [&](auto L, auto S) {
    k_store_pop<decltype(L)::value, decltype(S)::value>
        <<<nblocks(ncells(v)), TPB, 0, s>>>(v, f, i, stored);
  });
  return cudaGetLastError();
}

cudaError_t diag_moments(const View &v, const void *stored, double G, double rho0, double *rho,
                         double *jx, double *jy, double *jz, double *psi, double *p, int *err,
                         cudaStream_t s) {
  const bool want_j = jx || jy || jz;
  dispatch(v, [&](auto L, auto S) {
    if (want_j)
      k_moments<decltype(L)::value, decltype(S)::value, true>
          <<<nblocks(ncells(v)), TPB, 0, s>>>(v, stored, G, rho0, rho, jx, jy, jz, psi, p, err);
    else
      k_moments<decltype(L)::value, decltype(S)::value, false>
          <<<nblocks(ncells(v)), TPB, 0, s>>>(v, stored, G, rho0, rho, jx, jy, jz, psi, p, err);
  });
  return cudaGetLastError();
}

cudaError_t diag_velocity(const View &v, double G, const double *rho, const double *jx,
                          const double *jy, const double *jz, const double *psi, double *u,
                          cudaStream_t s) {
  if (v.lat == D3Q19)
    k_velocity<D3Q19><<<nblocks(ncells(v)), TPB, 0, s>>>(v, G, rho, jx, jy, jz, psi, u);
  else
    k_velocity<D2Q9><<<nblocks(ncells(v)), TPB, 0, s>>>(v, G, rho, jx, jy, jz, psi, u);
  return cudaGetLastError();
}

cudaError_t diag_laplacian(const View &v, const double *p, double *lap, cudaStream_t s) {
  k_laplacian<<<nblocks(ncells(v)), TPB, 0, s>>>(v, p, lap);
  return cudaGetLastError();
}

cudaError_t diag_line_d2(const View &v, const double *p, int64_t x0, int64_t y0, int64_t z0,
                         int axis, int64_t len, double *out, cudaStream_t s) {
  k_line_d2<<<nblocks(len), TPB, 0, s>>>(v, p, (int)x0, (int)y0, (int)z0, axis, len, out);
  return cudaGetLastError();
}

cudaError_t diag_film_probe(const View &v, const double *rho, const double *p, int64_t x0,
                            int64_t y0, int64_t z0, const int e[3], const int ep[3], int64_t len,
                            double mid, double *out, cudaStream_t s) {
  k_film_probe<<<1, 256, 0, s>>>(v, rho, p, x0, y0, z0, e[0], e[1], e[2], ep[0], ep[1], ep[2],
                                 len, mid, out);
  return cudaGetLastError();
}

int diag_totals_blocks() { return TOT_BLOCKS; }

cudaError_t diag_totals(const View &v, const void *stored, double *partials, double *out4,
                        cudaStream_t s) {
  dispatch(v, [&](auto L, auto S) {
    k_totals<decltype(L)::value, decltype(S)::value><<<TOT_BLOCKS, TPB, 0, s>>>(v, stored, partials);
  });
  if (v.lat == D3Q19)
    k_totals_final<D3Q19><<<1, TPB, 0, s>>>(partials, out4);
  else
    k_totals_final<D2Q9><<<1, TPB, 0, s>>>(partials, out4);
  return cudaGetLastError();
}

int diag_scan_blocks() { return SCAN_BLOCKS; }

cudaError_t diag_scan(const View &v, const void *stored, double thr, int32_t *labels,
                      double *partials, double *out4, int *err, cudaStream_t s) {
  dispatch(v, [&](auto L, auto S) {
    constexpr int lat = decltype(L)::value, st = decltype(S)::value;
    if constexpr (st != ST_F64) {
      k_scan<lat, st><<<SCAN_BLOCKS, TPB, 0, s>>>(v, stored, thr, labels, partials, err);
      if (out4)
        k_scan_final<lat><<<1, TPB, 0, s>>>(partials, (double)ncells(v) * v.rho_ref, out4);
    }
  });
  return cudaGetLastError();
}

cudaError_t diag_label_links(const View &v, int32_t *labels, unsigned long long *ncomp_dev,
                             cudaStream_t s) {
  const int64_t N = ncells(v);
  cudaError_t e = cudaMemsetAsync(ncomp_dev, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_ccl_union<<<nblocks((N + 3) / 4), TPB, 0, s>>>(v, labels);
  k_ccl_compress<<<nblocks((N + 3) / 4), TPB, 0, s>>>(N, labels, ncomp_dev);
  return cudaGetLastError();
}

cudaError_t diag_label(const View &v, const double *rho, double thr, int32_t *labels,
                       unsigned long long *ncomp_dev, cudaStream_t s) {
  const int64_t N = ncells(v);
  cudaError_t e = cudaMemsetAsync(ncomp_dev, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_ccl_init<<<nblocks(N), TPB, 0, s>>>(N, rho, thr, labels);
  k_ccl_union<<<nblocks((N + 3) / 4), TPB, 0, s>>>(v, labels);
  k_ccl_compress<<<nblocks((N + 3) / 4), TPB, 0, s>>>(N, labels, ncomp_dev);
  return cudaGetLastError();
}

size_t film_record_bytes() { return sizeof(FilmRec); }

cudaError_t diag_film_cells(const View &v, const int32_t *labels, const void *stored, double G,
                            double rho0, int h_max, double eps_arm, uint8_t *state,
                            unsigned long long *counts, int64_t cap, void *records,
                            bool all_mid, FilmMid *mids, int64_t mid_cap, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * FILM_COUNT_SLOTS, s);
  if (e != cudaSuccess) return e;
  FilmRec *rec = static_cast<FilmRec *>(records);
  const int am = all_mid ? 1 : 0;
  dispatch(v, [&](auto L, auto S) {
    constexpr int LAT = decltype(L)::value, STV = decltype(S)::value;
    if (h_max > FILM_LINE_HMAX || !mids) {
      k_film_cells<LAT, STV><<<nblocks(ncells(v)), TPB, 0, s>>>(
          v, labels, stored, G, rho0, h_max, eps_arm, state, counts, cap, rec, am);
      return;
    }
    const FilmArgs A{v,     labels, stored, G,   rho0, eps_arm, h_max, am,
                     state, counts, cap,    rec, mids, mid_cap};
    // one walk per lattice line: rows along x, then the other axes in turn;
    // then the queued midpoints
    const int64_t rows = v.NY * v.NZ;
    k_film_rows<LAT, STV><<<(int)((rows + FILM_ROWS - 1) / FILM_ROWS), FILM_ROWS, 0, s>>>(A);
    const int naxes = LAT == D2Q9 ? 2 : 3;
    for (int ua = 1; ua < naxes; ++ua) {
      const int va = LAT == D2Q9 ? 2 : ua;  // D2Q9's second axis is the view's z
      const int64_t nl = v.NX * (va == 1 ? v.NZ : v.NY);
      k_film_cols<LAT, STV><<<(int)((nl + TPB - 1) / TPB), TPB, 0, s>>>(A, ua, va);
    }
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    k_film_mids<LAT, STV><<<std::max(nsm, 1) * 4, TPB, 0, s>>>(A);
  });
  return cudaGetLastError();
}

cudaError_t diag_gather_labels(const int32_t *labels, const int32_t *cells, int32_t n,
                               int32_t *out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_gather_labels<<<(n + TPB - 1) / TPB, TPB, 0, s>>>(labels, cells, n, out);
  return cudaGetLastError();
}

}  // namespace sclbm
