/*
 * Plain FP64 CPU oracle for the single-component Shan-Chen pseudopotential
 * lattice Boltzmann method used to study bubble merging in liquid metal
 * (Barzegari, Bayani, Mirbagheri, "A criterion for bubble merging in liquid
 * metal", arXiv 1708.01608).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the GPU path computes.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * source, header, table or helper with the CUDA library.
 *
 * Everything is double precision, plain loops, no blocking or fusion: every
 * phase of a step runs over the whole lattice before the next one starts.
 * The optional OpenMP pragmas only split the outermost loop of a phase; they
 * do not change any arithmetic or summation order.
 *
 * Conventions
 *   lattice  0 = D2Q9 (nz must be 1), 1 = D3Q19
 *   cell     linear index  x + nx*(y + ny*z), periodic in every axis
 *   f        populations f[i*N + cell], N = nx*ny*nz, "post-streaming" form:
 *            f_i(x,t) is the population that has arrived at x at time t
 *   velocity order (both lattices): rest, the axis directions, then the
 *            diagonals, exactly as in the tables below.
 *
 * Paper passages followed (section numbers of arXiv 1708.01608):
 *   Sec. 3.1  Shan-Chen model with long-range attraction between the
 *             distribution functions; EOS p = rho cs^2 + (G cs^2/2) psi^2 (the
 *             printed 0.166 is read as cs^2/2 = 1/6); psi = 1 - exp(-rho)
 *             (generalised to rho0 (1 - exp(-rho/rho0)), rho0 = 1 recovers it);
 *             single-relaxation collision followed by streaming.
 *   Sec. 3    random nucleation sites; a virtual blowing agent adds gas to
 *             every bubble each time step until it is used up.
 *   Sec. 3.1, Sec. 4  second derivative of the pressure across the film
 *             between two bubbles as the rupture criterion.
 * The paper does not state the forcing scheme, lattice, boundaries or how gas
 * regions are identified.  This oracle takes: the Shan-Chen velocity shift
 * u_eq = (j + tau F)/rho; D2Q9 and D3Q19; periodic boundaries in every axis;
 * gas = rho below a threshold, face-connected, labelled by the smallest
 * linear index of its component.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_D2Q9 0
#define ORC_D3Q19 1

/* ---- velocity sets (standard D2Q9 / D3Q19, weights 4/9,1/9,1/36 and
 *      1/3,1/18,1/36) ---------------------------------------------------- */
static const int C9[9][3] = {
    {0, 0, 0},  {1, 0, 0},  {0, 1, 0},   {-1, 0, 0}, {0, -1, 0},
    {1, 1, 0},  {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
static const double W9[9] = {4.0 / 9,  1.0 / 9,  1.0 / 9,  1.0 / 9, 1.0 / 9,
                             1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

static const int C19[19][3] = {
    {0, 0, 0},   {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
    {0, 0, 1},   {0, 0, -1}, {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
    {-1, 1, 0},  {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const double W19[19] = {
    1.0 / 3,  1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18,
    1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
    1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

static int lat_q(int lat) { return lat == ORC_D2Q9 ? 9 : 19; }
static const int *lat_c(int lat, int i) { return lat == ORC_D2Q9 ? C9[i] : C19[i]; }
static double lat_w(int lat, int i) { return lat == ORC_D2Q9 ? W9[i] : W19[i]; }

int orc_q(int lat) { return lat_q(lat); }

void orc_velocities(int lat, int *c, double *w) {
  int q = lat_q(lat);
  for (int i = 0; i < q; ++i) {
    for (int a = 0; a < 3; ++a) c[3 * i + a] = lat_c(lat, i)[a];
    w[i] = lat_w(lat, i);
  }
}

static int64_t wrap(int64_t a, int64_t n) {
  int64_t r = a % n;
  return r < 0 ? r + n : r;
}

/* linear index of the periodic neighbour (x+dx, y+dy, z+dz) */
static int64_t nb(int64_t x, int64_t y, int64_t z, int dx, int dy, int dz,
                  int64_t nx, int64_t ny, int64_t nz) {
  return wrap(x + dx, nx) + nx * (wrap(y + dy, ny) + ny * wrap(z + dz, nz));
}

/* ---- SplitMix64 (Steele, Lea & Flood 2014), counter form ---------------
 * value k of the stream keyed by `key` is the k-th output of a SplitMix64
 * generator whose state starts at `key`: state = key + (k+1)*gamma, then the
 * published output mix. */
static uint64_t sm64_at(uint64_t key, uint64_t k) {
  uint64_t z = key + (k + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static double sm64_unit(uint64_t key, uint64_t k) {
  return (double)(sm64_at(key, k) >> 11) * (1.0 / 9007199254740992.0);
}
/* stream keys: the seed xor a fixed tag per purpose */
#define TAG_NOISE 0x6E6F697365000000ULL /* "noise" */
#define TAG_SITES 0x7369746573000000ULL /* "sites" */

uint64_t orc_splitmix64(uint64_t key, uint64_t k) { return sm64_at(key, k); }

/* ---- pseudopotential, EOS ------------------------------------------------ */
/* Sec. 3.1: psi(rho) = rho0 (1 - exp(-rho/rho0)) */
static double psi_of(double rho, double rho0) { return rho0 * (1.0 - exp(-rho / rho0)); }

/* Sec. 3.1: p = rho cs^2 + G cs^2/2 psi^2, cs^2 = 1/3 */
static double p_of(double rho, double G, double rho0) {
  double s = psi_of(rho, rho0);
  return rho / 3.0 + G / 6.0 * s * s;
}

void orc_eos(int64_t n, const double *rho, double G, double rho0, double *psi,
             double *p) {
  for (int64_t k = 0; k < n; ++k) {
    if (psi) psi[k] = psi_of(rho[k], rho0);
    if (p) p[k] = p_of(rho[k], G, rho0);
  }
}

/* ---- moments: rho = sum_i f_i, j = sum_i f_i c_i (velocity order) -------- */
void orc_moments(int lat, int64_t nx, int64_t ny, int64_t nz, const double *f,
                 double *rho, double *jx, double *jy, double *jz) {
  int q = lat_q(lat);
  int64_t N = nx * ny * nz;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < N; ++k) {
    double r = 0, a = 0, b = 0, c = 0;
    for (int i = 0; i < q; ++i) {
      double v = f[(int64_t)i * N + k];
      const int *ci = lat_c(lat, i);
      r += v;
      a += v * ci[0];
      b += v * ci[1];
      c += v * ci[2];
    }
    rho[k] = r;
    if (jx) jx[k] = a;
    if (jy) jy[k] = b;
    if (jz) jz[k] = c;
  }
}

/* ---- Shan-Chen force  F(x) = -G psi(x) sum_i w_i psi(x+c_i) c_i ---------- */
void orc_force(int lat, int64_t nx, int64_t ny, int64_t nz, const double *psi,
               double G, double *Fx, double *Fy, double *Fz) {
  int q = lat_q(lat);
#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t z = 0; z < nz; ++z)
    for (int64_t y = 0; y < ny; ++y)
      for (int64_t x = 0; x < nx; ++x) {
        int64_t k = x + nx * (y + ny * z);
        double sx = 0, sy = 0, sz = 0;
        for (int i = 1; i < q; ++i) {
          const int *ci = lat_c(lat, i);
          double s = lat_w(lat, i) * psi[nb(x, y, z, ci[0], ci[1], ci[2], nx, ny, nz)];
          sx += s * ci[0];
          sy += s * ci[1];
          sz += s * ci[2];
        }
        Fx[k] = -G * psi[k] * sx;
        Fy[k] = -G * psi[k] * sy;
        Fz[k] = -G * psi[k] * sz;
      }
}

/* equilibrium f_eq_i = w_i rho (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u) */
static double feq(int lat, int i, double rho, double ux, double uy, double uz) {
  const int *c = lat_c(lat, i);
  double cu = c[0] * ux + c[1] * uy + c[2] * uz;
  double uu = ux * ux + uy * uy + uz * uz;
  return lat_w(lat, i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

/*
 * One time step, in the order of the method:
 *   1 moments  2 psi everywhere  3 Shan-Chen force  4 velocity shift
 *   u_eq = (j + tau F)/rho  5 equilibrium  6 BGK  f* = f - (f - f_eq)/tau
 *   7 injection of the virtual blowing agent (Sec. 3): for each site s with
 *     budget left, dm = min(rate_s, budget_s), budget_s -= dm and
 *     f*_i(x_s) += w_i dm (zero momentum)
 *   8 streaming f_i(x + c_i, t+1) = f*_i(x)
 * f is updated in place; work must hold (Q + 8) * N doubles.
 * site_cell / rate / budget may be NULL when nsites == 0.
 */
void orc_step(int lat, int64_t nx, int64_t ny, int64_t nz, double tau,
              double G, double rho0, double *f, double *work, int32_t nsites,
              const int64_t *site_cell, const double *rate, double *budget) {
  int q = lat_q(lat);
  int64_t N = nx * ny * nz;
  double *rho = work, *jx = work + N, *jy = work + 2 * N, *jz = work + 3 * N;
  double *psi = work + 4 * N, *Fx = work + 5 * N, *Fy = work + 6 * N,
         *Fz = work + 7 * N;
  double *fs = work + 8 * N; /* post-collision populations, Q*N */

  orc_moments(lat, nx, ny, nz, f, rho, jx, jy, jz);
  for (int64_t k = 0; k < N; ++k) psi[k] = psi_of(rho[k], rho0);
  orc_force(lat, nx, ny, nz, psi, G, Fx, Fy, Fz);

#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < N; ++k) {
    double ux = (jx[k] + tau * Fx[k]) / rho[k];
    double uy = (jy[k] + tau * Fy[k]) / rho[k];
    double uz = (jz[k] + tau * Fz[k]) / rho[k];
    for (int i = 0; i < q; ++i) {
      double fi = f[(int64_t)i * N + k];
      fs[(int64_t)i * N + k] = fi - (fi - feq(lat, i, rho[k], ux, uy, uz)) / tau;
    }
  }

  for (int32_t s = 0; s < nsites; ++s) {
    if (budget[s] <= 0) continue;
    double dm = rate[s] < budget[s] ? rate[s] : budget[s];
    budget[s] -= dm;
    for (int i = 0; i < q; ++i) fs[(int64_t)i * N + site_cell[s]] += lat_w(lat, i) * dm;
  }

#pragma omp parallel for collapse(2) schedule(static)
  for (int64_t z = 0; z < nz; ++z)
    for (int64_t y = 0; y < ny; ++y)
      for (int64_t x = 0; x < nx; ++x) {
        int64_t k = x + nx * (y + ny * z);
        for (int i = 0; i < q; ++i) {
          const int *c = lat_c(lat, i);
          f[(int64_t)i * N + nb(x, y, z, c[0], c[1], c[2], nx, ny, nz)] =
              fs[(int64_t)i * N + k];
        }
      }
}

void orc_run(int lat, int64_t nx, int64_t ny, int64_t nz, double tau, double G,
             double rho0, double *f, int64_t nsteps, int32_t nsites,
             const int64_t *site_cell, const double *rate, double *budget) {
  int q = lat_q(lat);
  int64_t N = nx * ny * nz;
  double *work = (double *)malloc(sizeof(double) * (size_t)((q + 8) * N));
  for (int64_t t = 0; t < nsteps; ++t)
    orc_step(lat, nx, ny, nz, tau, G, rho0, f, work, nsites, site_cell, rate, budget);
  free(work);
}

/*
 * Post-collision population f*_i at one cell, computed from scratch (used to
 * check sampled cells of very large lattices one by one): the moments of the
 * cell, psi of the cell and of its neighbours, the force, the shifted
 * velocity, the equilibrium and BGK, exactly as in orc_step.  Injection is
 * not included.
 */
static double fstar_at(int lat, int64_t nx, int64_t ny, int64_t nz, double tau,
                       double G, double rho0, const double *f, int64_t x,
                       int64_t y, int64_t z, int i) {
  int q = lat_q(lat);
  int64_t N = nx * ny * nz;
  int64_t k = x + nx * (y + ny * z);
  double rho = 0, jx = 0, jy = 0, jz = 0;
  for (int a = 0; a < q; ++a) {
    double v = f[(int64_t)a * N + k];
    const int *c = lat_c(lat, a);
    rho += v;
    jx += v * c[0];
    jy += v * c[1];
    jz += v * c[2];
  }
  double sx = 0, sy = 0, sz = 0;
  for (int a = 1; a < q; ++a) {
    const int *c = lat_c(lat, a);
    int64_t m = nb(x, y, z, c[0], c[1], c[2], nx, ny, nz);
    double rm = 0;
    for (int b = 0; b < q; ++b) rm += f[(int64_t)b * N + m];
    double s = lat_w(lat, a) * psi_of(rm, rho0);
    sx += s * c[0];
    sy += s * c[1];
    sz += s * c[2];
  }
  double ps = psi_of(rho, rho0);
  double Fx = -G * ps * sx, Fy = -G * ps * sy, Fz = -G * ps * sz;
  double ux = (jx + tau * Fx) / rho, uy = (jy + tau * Fy) / rho,
         uz = (jz + tau * Fz) / rho;
  double fi = f[(int64_t)i * N + k];
  return fi - (fi - feq(lat, i, rho, ux, uy, uz)) / tau;
}

/* f_i(x, t+1) for the listed destination cells: out[c*Q + i] */
void orc_step_cells(int lat, int64_t nx, int64_t ny, int64_t nz, double tau,
                    double G, double rho0, const double *f, int64_t ncells,
                    const int64_t *cells, double *out) {
  int q = lat_q(lat);
#pragma omp parallel for schedule(dynamic)
  for (int64_t c = 0; c < ncells; ++c) {
    int64_t k = cells[c];
    int64_t x = k % nx, y = (k / nx) % ny, z = k / (nx * ny);
    for (int i = 0; i < q; ++i) {
      const int *ci = lat_c(lat, i);
      int64_t src = nb(x, y, z, -ci[0], -ci[1], -ci[2], nx, ny, nz);
      int64_t sx = src % nx, sy = (src / nx) % ny, sz = src / (nx * ny);
      out[c * q + i] = fstar_at(lat, nx, ny, nz, tau, G, rho0, f, sx, sy, sz, i);
    }
  }
}

/* ---- initial state --------------------------------------------------------
 * Gas bubbles (x, y, z, r) in liquid: with s = min_k (d_k - r_k), d_k the
 * minimum-image distance to centre k,
 *   rho = rho_g + (rho_l - rho_g)/2 (1 + tanh(2 s / width))
 * plus uniform noise amp*(2u-1), u from the "noise" stream at the cell index;
 * then f_i = f_eq(rho, 0) = w_i rho.  With no bubbles rho = rho_l + noise.
 */
static double min_image(double d, double n) {
  d = fmod(d, n);
  if (d < 0) d += n;
  if (d > 0.5 * n) d -= n;
  return d;
}

void orc_init(int lat, int64_t nx, int64_t ny, int64_t nz, int32_t nb_,
              const double *bub /* nb x 4 */, double rho_l, double rho_g,
              double width, double noise_amp, uint64_t seed, double *f,
              double *rho_out) {
  int q = lat_q(lat);
  int64_t N = nx * ny * nz;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < N; ++k) {
    int64_t x = k % nx, y = (k / nx) % ny, z = k / (nx * ny);
    double rho = rho_l;
    if (nb_ > 0) {
      double s = INFINITY;
      for (int32_t b = 0; b < nb_; ++b) {
        double dx = min_image((double)x - bub[4 * b + 0], (double)nx);
        double dy = min_image((double)y - bub[4 * b + 1], (double)ny);
        double dz = min_image((double)z - bub[4 * b + 2], (double)nz);
        double d = sqrt(dx * dx + dy * dy + dz * dz) - bub[4 * b + 3];
        if (d < s) s = d;
      }
      rho = rho_g + 0.5 * (rho_l - rho_g) * (1.0 + tanh(2.0 * s / width));
    }
    if (noise_amp != 0.0)
      rho += noise_amp * (2.0 * sm64_unit(seed ^ TAG_NOISE, (uint64_t)k) - 1.0);
    if (rho_out) rho_out[k] = rho;
    for (int i = 0; i < q; ++i) f[(int64_t)i * N + k] = lat_w(lat, i) * rho;
  }
}

/* ---- random nucleation sites (Sec. 3 "random function") -------------------
 * Candidate m draws four values u0..u3 from the "sites" stream at indices
 * 4m..4m+3: centre (floor(u0 nx), floor(u1 ny), floor(u2 nz)) and radius
 * r_min + (r_max - r_min) u3.  Candidates are accepted in order when their
 * minimum-image distance to every accepted centre is at least
 * max(min_spacing, r_a + r_b + min_gap).  Returns the number accepted (n on
 * success), stopping after max_tries candidates. */
int32_t orc_sample_sites(int64_t nx, int64_t ny, int64_t nz, int32_t n,
                         double r_min, double r_max, double min_spacing,
                         double min_gap, uint64_t seed, int64_t max_tries,
                         double *out /* n x 4 */) {
  uint64_t key = seed ^ TAG_SITES;
  int32_t got = 0;
  for (int64_t m = 0; m < max_tries && got < n; ++m) {
    double cx = floor(sm64_unit(key, 4 * (uint64_t)m + 0) * (double)nx);
    double cy = floor(sm64_unit(key, 4 * (uint64_t)m + 1) * (double)ny);
    double cz = floor(sm64_unit(key, 4 * (uint64_t)m + 2) * (double)nz);
    double r = r_min + (r_max - r_min) * sm64_unit(key, 4 * (uint64_t)m + 3);
    int ok = 1;
    for (int32_t a = 0; a < got && ok; ++a) {
      double dx = min_image(cx - out[4 * a + 0], (double)nx);
      double dy = min_image(cy - out[4 * a + 1], (double)ny);
      double dz = min_image(cz - out[4 * a + 2], (double)nz);
      double d = sqrt(dx * dx + dy * dy + dz * dz);
      double need = r + out[4 * a + 3] + min_gap;
      if (min_spacing > need) need = min_spacing;
      if (d < need) ok = 0;
    }
    if (ok) {
      out[4 * got + 0] = cx;
      out[4 * got + 1] = cy;
      out[4 * got + 2] = cz;
      out[4 * got + 3] = r;
      ++got;
    }
  }
  return got;
}

/* ---- pressure Laplacian (Sec. 3.1 / Sec. 4 criterion) ---------------------
 * lap(x) = sum over the d axes of p(x+e) - 2 p(x) + p(x-e), periodic;
 * d = 2 for D2Q9 (5-point), 3 for D3Q19 (7-point). */
void orc_laplacian(int lat, int64_t nx, int64_t ny, int64_t nz, const double *p,
                   double *lap) {
  int dims = lat == ORC_D2Q9 ? 2 : 3;
  for (int64_t z = 0; z < nz; ++z)
    for (int64_t y = 0; y < ny; ++y)
      for (int64_t x = 0; x < nx; ++x) {
        int64_t k = x + nx * (y + ny * z);
        double s = 0;
        for (int a = 0; a < dims; ++a) {
          int e[3] = {0, 0, 0};
          e[a] = 1;
          s += p[nb(x, y, z, e[0], e[1], e[2], nx, ny, nz)] - 2.0 * p[k] +
               p[nb(x, y, z, -e[0], -e[1], -e[2], nx, ny, nz)];
        }
        lap[k] = s;
      }
}

/* second difference d2p/dn2 along one axis at `len` consecutive cells
 * starting at (x0,y0,z0): p(x+e) - 2 p(x) + p(x-e) */
void orc_line_d2(int64_t nx, int64_t ny, int64_t nz, const double *p, int64_t x0,
                 int64_t y0, int64_t z0, int axis, int64_t len, double *out) {
  int e[3] = {0, 0, 0};
  e[axis] = 1;
  for (int64_t m = 0; m < len; ++m) {
    int64_t x = wrap(x0 + m * e[0], nx), y = wrap(y0 + m * e[1], ny),
            z = wrap(z0 + m * e[2], nz);
    int64_t k = x + nx * (y + ny * z);
    out[m] = p[nb(x, y, z, e[0], e[1], e[2], nx, ny, nz)] - 2.0 * p[k] +
             p[nb(x, y, z, -e[0], -e[1], -e[2], nx, ny, nz)];
  }
}

/* ---- gas connected components ---------------------------------------------
 * gas = rho < thr; face neighbours (4 in 2-D, 6 in 3-D), periodic.  Every gas
 * cell gets the smallest linear index of its component, liquid cells -1.
 * Breadth-first search started from unlabelled gas cells in increasing index
 * order, so the start cell is the component's minimum.  Returns the number
 * of components. */
int64_t orc_label_gas(int lat, int64_t nx, int64_t ny, int64_t nz,
                      const double *rho, double thr, int32_t *label) {
  int64_t N = nx * ny * nz;
  int dims = lat == ORC_D2Q9 ? 2 : 3;
  int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
  int64_t ncomp = 0;
  for (int64_t k = 0; k < N; ++k) label[k] = -1;
  for (int64_t s = 0; s < N; ++s) {
    if (!(rho[s] < thr) || label[s] != -1) continue;
    ++ncomp;
    int64_t head = 0, tail = 0;
    queue[tail++] = s;
    label[s] = (int32_t)s;
    while (head < tail) {
      int64_t k = queue[head++];
      int64_t x = k % nx, y = (k / nx) % ny, z = k / (nx * ny);
      for (int a = 0; a < dims; ++a)
        for (int sg = -1; sg <= 1; sg += 2) {
          int e[3] = {0, 0, 0};
          e[a] = sg;
          int64_t m = nb(x, y, z, e[0], e[1], e[2], nx, ny, nz);
          if (rho[m] < thr && label[m] == -1) {
            label[m] = (int32_t)s;
            queue[tail++] = m;
          }
        }
    }
  }
  free(queue);
  return ncomp;
}

/* ---- global FP64 sums: mass and momentum ---------------------------------- */
void orc_totals(int lat, int64_t nx, int64_t ny, int64_t nz, const double *f,
                double *out /* M, Jx, Jy, Jz */) {
  int q = lat_q(lat);
  int64_t N = nx * ny * nz;
  double M = 0, a = 0, b = 0, c = 0;
  for (int64_t k = 0; k < N; ++k)
    for (int i = 0; i < q; ++i) {
      double v = f[(int64_t)i * N + k];
      const int *ci = lat_c(lat, i);
      M += v;
      a += v * ci[0];
      b += v * ci[1];
      c += v * ci[2];
    }
  out[0] = M;
  out[1] = a;
  out[2] = b;
  out[3] = c;
}

/* ---- film probe (Sec. 3.1 / Sec. 4: pressure second derivative across the
 * film between two bubbles) ----------------------------------------------------
 * Along `len` cells from (x0,y0,z0) in direction e_axis (from inside bubble A
 * towards bubble B), with rho_mid the density separating gas from liquid:
 *   x1 = first upward crossing of rho_mid (linear interpolation between the
 *        two cells), x2 = the next downward crossing; h = x2 - x1 is the film
 *        thickness.
 *   d2p/dn2 at the film midpoint xm = (x1+x2)/2: p(c+e)-2p(c)+p(c-e) at the
 *        nearest line cell c (mean of the two cells when xm is exactly half-way).
 *   R_d: through the midpoint cell, walk along e_perp (axis+1, modulo the
 *        lattice dimension); in every row whose midpoint cell is liquid the
 *        local thickness is the length of the liquid run along e_axis through
 *        it (interpolated crossings on both sides).  The rows contiguous with
 *        the centre row whose thickness is <= h + 2 form the film disc, and
 *        R_d is half its extent in cells.
 * out = {found, x1, x2, h, d2p_mid, R_d}; found = 0 when no film exists. */
static double lerp_cross(double ra, double rb, double mid) { return (mid - ra) / (rb - ra); }

static int64_t cell_at(int64_t nx, int64_t ny, int64_t nz, int64_t x, int64_t y, int64_t z) {
  return wrap(x, nx) + nx * (wrap(y, ny) + ny * wrap(z, nz));
}

/* thickness of the liquid run along e through cell (x,y,z); -1 if gas */
static double run_thickness(int64_t nx, int64_t ny, int64_t nz, const double *rho, int64_t x,
                            int64_t y, int64_t z, const int e[3], double mid, int64_t maxlen) {
  if (rho[cell_at(nx, ny, nz, x, y, z)] < mid) return -1.0;
  double lo = 0, hi = 0;
  int64_t m;
  for (m = 1; m <= maxlen; ++m) { /* backwards */
    double ra = rho[cell_at(nx, ny, nz, x - (m - 1) * e[0], y - (m - 1) * e[1], z - (m - 1) * e[2])];
    double rb = rho[cell_at(nx, ny, nz, x - m * e[0], y - m * e[1], z - m * e[2])];
    if (rb < mid) {
      lo = -((double)(m - 1) + lerp_cross(ra, rb, mid));
      break;
    }
  }
  if (m > maxlen) return -1.0;
  for (m = 1; m <= maxlen; ++m) { /* forwards */
    double ra = rho[cell_at(nx, ny, nz, x + (m - 1) * e[0], y + (m - 1) * e[1], z + (m - 1) * e[2])];
    double rb = rho[cell_at(nx, ny, nz, x + m * e[0], y + m * e[1], z + m * e[2])];
    if (rb < mid) {
      hi = (double)(m - 1) + lerp_cross(ra, rb, mid);
      break;
    }
  }
  if (m > maxlen) return -1.0;
  return hi - lo;
}

void orc_film_probe(int lat, int64_t nx, int64_t ny, int64_t nz, const double *rho,
                    const double *p, int64_t x0, int64_t y0, int64_t z0, int axis, int64_t len,
                    double mid, double *out) {
  int e[3] = {0, 0, 0}, ep[3] = {0, 0, 0};
  int dims = lat == ORC_D2Q9 ? 2 : 3;
  e[axis] = 1;
  ep[(axis + 1) % dims] = 1;
  for (int q = 0; q < 6; ++q) out[q] = 0.0;
  double x1 = -1, x2 = -1;
  int64_t m;
  for (m = 1; m < len; ++m) {
    double ra = rho[cell_at(nx, ny, nz, x0 + (m - 1) * e[0], y0 + (m - 1) * e[1], z0 + (m - 1) * e[2])];
    double rb = rho[cell_at(nx, ny, nz, x0 + m * e[0], y0 + m * e[1], z0 + m * e[2])];
    if (ra < mid && rb >= mid) {
      x1 = (double)(m - 1) + lerp_cross(ra, rb, mid);
      break;
    }
  }
  if (x1 < 0) return;
  for (++m; m < len; ++m) {
    double ra = rho[cell_at(nx, ny, nz, x0 + (m - 1) * e[0], y0 + (m - 1) * e[1], z0 + (m - 1) * e[2])];
    double rb = rho[cell_at(nx, ny, nz, x0 + m * e[0], y0 + m * e[1], z0 + m * e[2])];
    if (ra >= mid && rb < mid) {
      x2 = (double)(m - 1) + lerp_cross(ra, rb, mid);
      break;
    }
  }
  if (x2 < 0) return;
  double h = x2 - x1, xm = 0.5 * (x1 + x2);
  double fl = floor(xm);
  int64_t c = (int64_t)fl;
  double d2;
  if (xm - fl == 0.5) {
    double dd[2];
    for (int k = 0; k < 2; ++k) {
      int64_t cc = c + k;
      dd[k] = p[cell_at(nx, ny, nz, x0 + (cc + 1) * e[0], y0 + (cc + 1) * e[1], z0 + (cc + 1) * e[2])] -
              2.0 * p[cell_at(nx, ny, nz, x0 + cc * e[0], y0 + cc * e[1], z0 + cc * e[2])] +
              p[cell_at(nx, ny, nz, x0 + (cc - 1) * e[0], y0 + (cc - 1) * e[1], z0 + (cc - 1) * e[2])];
    }
    d2 = 0.5 * (dd[0] + dd[1]);
  } else {
    int64_t cc = xm - fl < 0.5 ? c : c + 1;
    d2 = p[cell_at(nx, ny, nz, x0 + (cc + 1) * e[0], y0 + (cc + 1) * e[1], z0 + (cc + 1) * e[2])] -
         2.0 * p[cell_at(nx, ny, nz, x0 + cc * e[0], y0 + cc * e[1], z0 + cc * e[2])] +
         p[cell_at(nx, ny, nz, x0 + (cc - 1) * e[0], y0 + (cc - 1) * e[1], z0 + (cc - 1) * e[2])];
  }
  /* film disc along e_perp through the midpoint cell */
  int64_t cm = (int64_t)floor(xm + 0.5);
  int64_t xc = x0 + cm * e[0], yc = y0 + cm * e[1], zc = z0 + cm * e[2];
  int64_t extent = 0;
  for (int sg = -1; sg <= 1; sg += 2) {
    for (int64_t j = (sg < 0 ? 1 : 0); j <= len; ++j) {
      double t = run_thickness(nx, ny, nz, rho, xc + sg * j * ep[0], yc + sg * j * ep[1],
                               zc + sg * j * ep[2], e, mid, len);
      if (t < 0 || t > h + 2.0) break;
      ++extent;
    }
  }
  out[0] = 1.0;
  out[1] = x1;
  out[2] = x2;
  out[3] = h;
  out[4] = d2;
  out[5] = 0.5 * (double)extent;
}

/* ---- bubble census (Sec. 4: bubble sizes, merging defects) ----------------
 * From gas labels (orc_label_gas: label = smallest linear index of the
 * component, -1 liquid): the size in cells of every component, listed in
 * increasing order of its label.  roots/sizes hold up to cap entries (either
 * may be NULL); returns the number of components. */
int64_t orc_bubble_sizes(int64_t N, const int32_t *label, int64_t cap, int64_t *roots,
                         int64_t *sizes) {
  int64_t *count = (int64_t *)calloc((size_t)(N > 0 ? N : 1), sizeof(int64_t));
  for (int64_t k = 0; k < N; ++k)
    if (label[k] >= 0) count[label[k]] += 1;
  int64_t n = 0;
  for (int64_t r = 0; r < N; ++r) {
    if (count[r] == 0) continue;
    if (n < cap) {
      if (roots) roots[n] = r;
      if (sizes) sizes[n] = count[r];
    }
    ++n;
  }
  free(count);
  return n;
}

/* Histogram of component sizes in powers of two: bin b counts sizes s with
 * 2^b <= s < 2^(b+1); the last bin also takes everything larger. */
void orc_size_histogram(int64_t n, const int64_t *sizes, int nbins, int64_t *hist) {
  for (int b = 0; b < nbins; ++b) hist[b] = 0;
  for (int64_t q = 0; q < n; ++q) {
    int b = 0;
    while (b + 1 < nbins && ((int64_t)1 << (b + 1)) <= sizes[q]) ++b;
    hist[b] += 1;
  }
}

/* ---- the film test at every lattice point (Sec. 4) ------------------------
 * Sec. 4 applies the rupture criterion "at each lattice point" of a foam.
 * For every liquid cell (label -1) and every lattice axis a:
 *   walk from the cell along +e_a for at most h_max cells to the first gas
 *   cell (label L+, distance d+), and likewise along -e_a (L-, d-);
 *   the cell lies in a film along a when both exist, L+ != L- (two different
 *   bubbles) and the liquid run between them, t = d+ + d- - 1 cells, is at
 *   most h_max;
 *   it is a midpoint of that film when |d+ - d-| <= 1 (the middle cell of an
 *   odd run, the two middle cells of an even one);
 *   at a midpoint, d2 = p(x+e_a) - 2 p(x) + p(x-e_a) (FP64 EOS pressure) drives
 *   the criterion of the two-bubble probe, per (cell, axis): it is armed when
 *   d2 < -eps_arm, and fires when armed and d2 >= 0 (the arming is then
 *   cleared).  A (cell, axis) that is not a film midpoint is disarmed.
 * state[k] bit a holds the arming of (k, a) across calls.
 * counts = {film (cell, axis) pairs, midpoints, armed after the update,
 * fired}; the fired records, in increasing (cell, axis) order, fill up to
 * cap entries of rec (cell, axis, L-, L+, t) and d2 (either may be NULL). */
/* One pass of the film test.  all_mid = 0: rec (5 columns) and d2out hold
 * the fired (cell, axis) pairs.  all_mid = 1: rec (6 columns: cell, axis,
 * label on the -axis side, label on the +axis side, thickness, fired) and
 * d2out hold every film midpoint, and counts[4] their number. */
static void film_pass(int lat, int64_t nx, int64_t ny, int64_t nz, const int32_t *label,
                      const double *p, int h_max, double eps_arm, uint8_t *state,
                      int64_t *counts, int64_t cap, int64_t *rec, double *d2out, int all_mid) {
  int dims = lat == ORC_D2Q9 ? 2 : 3;
  int64_t N = nx * ny * nz;
  int64_t nfilm = 0, nmid = 0, narmed = 0, nfired = 0;
  for (int64_t k = 0; k < N; ++k) {
    int64_t x = k % nx, y = (k / nx) % ny, z = k / (nx * ny);
    for (int a = 0; a < dims; ++a) {
      uint8_t bit = (uint8_t)(1u << a);
      int film = 0, mid = 0;
      int32_t Lp = -1, Lm = -1;
      int dp = 0, dm = 0;
      if (label[k] < 0) {
        for (int s = 1; s <= h_max; ++s) {
          int e[3] = {0, 0, 0};
          e[a] = s;
          int64_t m = nb(x, y, z, e[0], e[1], e[2], nx, ny, nz);
          if (label[m] >= 0) {
            Lp = label[m];
            dp = s;
            break;
          }
        }
        for (int s = 1; s <= h_max; ++s) {
          int e[3] = {0, 0, 0};
          e[a] = -s;
          int64_t m = nb(x, y, z, e[0], e[1], e[2], nx, ny, nz);
          if (label[m] >= 0) {
            Lm = label[m];
            dm = s;
            break;
          }
        }
        film = Lp >= 0 && Lm >= 0 && Lp != Lm && dp + dm - 1 <= h_max;
        mid = film && (dp - dm <= 1 && dm - dp <= 1);
      }
      if (film) ++nfilm;
      if (!mid) {
        state[k] = (uint8_t)(state[k] & ~bit);
        continue;
      }
      int e[3] = {0, 0, 0};
      e[a] = 1;
      double d2 = p[nb(x, y, z, e[0], e[1], e[2], nx, ny, nz)] - 2.0 * p[k] +
                  p[nb(x, y, z, -e[0], -e[1], -e[2], nx, ny, nz)];
      int fired = 0;
      if (d2 < -eps_arm) {
        state[k] = (uint8_t)(state[k] | bit);
      } else if ((state[k] & bit) && d2 >= 0.0) {
        state[k] = (uint8_t)(state[k] & ~bit);
        fired = 1;
      }
      if (all_mid && nmid < cap) {
        if (rec) {
          int64_t *r = rec + 6 * nmid;
          r[0] = k;
          r[1] = a;
          r[2] = Lm;
          r[3] = Lp;
          r[4] = dp + dm - 1;
          r[5] = fired;
        }
        if (d2out) d2out[nmid] = d2;
      }
      ++nmid;
      if (fired) {
        if (!all_mid && nfired < cap) {
          if (rec) {
            int64_t *r = rec + 5 * nfired;
            r[0] = k;
            r[1] = a;
            r[2] = Lm;
            r[3] = Lp;
            r[4] = dp + dm - 1;
          }
          if (d2out) d2out[nfired] = d2;
        }
        ++nfired;
      }
    }
  }
  for (int64_t k = 0; k < N; ++k)
    for (int a = 0; a < dims; ++a) narmed += (state[k] >> a) & 1;
  counts[0] = nfilm;
  counts[1] = nmid;
  counts[2] = narmed;
  counts[3] = nfired;
  if (all_mid) counts[4] = nmid;
}

void orc_film_cells(int lat, int64_t nx, int64_t ny, int64_t nz, const int32_t *label,
                    const double *p, int h_max, double eps_arm, uint8_t *state,
                    int64_t *counts, int64_t cap, int64_t *rec, double *d2out) {
  film_pass(lat, nx, ny, nz, label, p, h_max, eps_arm, state, counts, cap, rec, d2out, 0);
}

/* The same pass recording every film midpoint: counts has 5 entries (film,
 * midpoints, armed, fired, midpoint records), rec 6 columns per midpoint in
 * increasing (cell, axis) order. */
void orc_film_midpoints(int lat, int64_t nx, int64_t ny, int64_t nz, const int32_t *label,
                        const double *p, int h_max, double eps_arm, uint8_t *state,
                        int64_t *counts, int64_t cap, int64_t *rec, double *d2out) {
  film_pass(lat, nx, ny, nz, label, p, h_max, eps_arm, state, counts, cap, rec, d2out, 1);
}

/* ==== multi-lattice Shan-Chen (Sec. 3.1, Fig. 1) ============================
 * A reading of the paper's modified model: the fluid (liquid metal) on
 * lattice 0 and the gas of bubble k on lattice k = 1 .. nl-1 ("each bubble
 * in its own lattice and fluid in a separate lattice", Fig. 1 steps 3-5),
 * coupled by interaction forces ("coupling the lattices and calculating the
 * interactions", step 6) in the multicomponent Shan-Chen form
 *   F_s(x) = -psi_s(x) sum_t Gm[s][t] sum_i w_i psi_t(x + c_i) c_i,
 * psi_s = rho0 (1 - exp(-rho_s/rho0)) on every lattice; Gm is the caller's
 * coupling matrix (fluid self-attraction G, fluid-gas coupling, and the
 * eta_m-switched barrier between different bubbles).  All lattices relax
 * with one tau towards f_eq(rho_s, u_s) with the common velocity
 *   u' = sum_s j_s / sum_s rho_s,   u_s = u' + tau F_s / rho_s
 * (u_s = u' where rho_s = 0: an empty lattice has f_eq = 0 whatever u_s).
 * The blowing agent of a site deposits w_i dm into the post-collision
 * populations of its own lattice at the site cell (Sec. 3: gas added to
 * each bubble).  Streaming as in orc_step, lattice by lattice.  f holds nl
 * lattices of Q*N values: f[(s*Q + i)*N + cell]. */

/* Multicomponent Shan-Chen force of every lattice from given psi fields
 * (nl x N): F_s = -psi_s sum_t Gm[s][t] sum_i w_i psi_t(x + c_i) c_i. */
void orc_ml_force(int lat, int64_t nx, int64_t ny, int64_t nz, int32_t nl, const double *psi,
                  const double *Gm, double *Fx, double *Fy, double *Fz) {
  int q = lat_q(lat);
  int64_t N = nx * ny * nz;
  for (int32_t s = 0; s < nl; ++s)
    for (int64_t z = 0; z < nz; ++z)
      for (int64_t y = 0; y < ny; ++y)
        for (int64_t x = 0; x < nx; ++x) {
          int64_t k = x + nx * (y + ny * z);
          double ax = 0, ay = 0, az = 0;
          for (int32_t t = 0; t < nl; ++t)
            for (int i = 1; i < q; ++i) {
              const int *ci = lat_c(lat, i);
              double v = Gm[s * nl + t] * lat_w(lat, i) *
                         psi[t * N + nb(x, y, z, ci[0], ci[1], ci[2], nx, ny, nz)];
              ax += v * ci[0];
              ay += v * ci[1];
              az += v * ci[2];
            }
          Fx[s * N + k] = -psi[s * N + k] * ax;
          Fy[s * N + k] = -psi[s * N + k] * ay;
          Fz[s * N + k] = -psi[s * N + k] * az;
        }
}

/* One step.  work must hold nl * (8 + Q) * N doubles. */
void orc_ml_step(int lat, int64_t nx, int64_t ny, int64_t nz, int32_t nl, double tau,
                 const double *Gm /* nl x nl */, double rho0, double *f, double *work,
                 int32_t nsites, const int64_t *site_cell, const int32_t *site_lattice,
                 const double *rate, double *budget) {
  int q = lat_q(lat);
  int64_t N = nx * ny * nz;
  double *rho = work;                                              /* nl * N */
  double *jx = rho + nl * N, *jy = jx + nl * N, *jz = jy + nl * N; /* nl * N each */
  double *psi = jz + nl * N;                                       /* nl * N */
  double *Fx = psi + nl * N, *Fy = Fx + nl * N, *Fz = Fy + nl * N; /* nl * N each */
  double *fs = Fz + nl * N;                                        /* nl * Q * N */

  /* 1 moments of every lattice */
  for (int32_t s = 0; s < nl; ++s)
    orc_moments(lat, nx, ny, nz, f + (int64_t)s * q * N, rho + s * N, jx + s * N, jy + s * N,
                jz + s * N);
  /* 2 psi of every lattice at every cell */
  for (int32_t s = 0; s < nl; ++s)
    for (int64_t k = 0; k < N; ++k) psi[s * N + k] = psi_of(rho[s * N + k], rho0);
  /* 3 the coupled forces */
  orc_ml_force(lat, nx, ny, nz, nl, psi, Gm, Fx, Fy, Fz);
  /* 4-6 common velocity, shifted velocities, BGK for every lattice */
  for (int64_t k = 0; k < N; ++k) {
    double rt = 0, jtx = 0, jty = 0, jtz = 0;
    for (int32_t s = 0; s < nl; ++s) {
      rt += rho[s * N + k];
      jtx += jx[s * N + k];
      jty += jy[s * N + k];
      jtz += jz[s * N + k];
    }
    double upx = jtx / rt, upy = jty / rt, upz = jtz / rt;
    for (int32_t s = 0; s < nl; ++s) {
      double r = rho[s * N + k];
      double ux = upx, uy = upy, uz = upz;
      if (r != 0.0) {
        ux += tau * Fx[s * N + k] / r;
        uy += tau * Fy[s * N + k] / r;
        uz += tau * Fz[s * N + k] / r;
      }
      for (int i = 0; i < q; ++i) {
        int64_t o = ((int64_t)s * q + i) * N + k;
        fs[o] = f[o] - (f[o] - feq(lat, i, r, ux, uy, uz)) / tau;
      }
    }
  }
  /* 7 blowing agent into the site's own lattice */
  for (int32_t m = 0; m < nsites; ++m) {
    if (budget[m] <= 0) continue;
    double dm = rate[m] < budget[m] ? rate[m] : budget[m];
    budget[m] -= dm;
    for (int i = 0; i < q; ++i)
      fs[((int64_t)site_lattice[m] * q + i) * N + site_cell[m]] += lat_w(lat, i) * dm;
  }
  /* 8 streaming, lattice by lattice */
  for (int32_t s = 0; s < nl; ++s)
    for (int64_t z = 0; z < nz; ++z)
      for (int64_t y = 0; y < ny; ++y)
        for (int64_t x = 0; x < nx; ++x) {
          int64_t k = x + nx * (y + ny * z);
          for (int i = 0; i < q; ++i) {
            const int *c = lat_c(lat, i);
            f[((int64_t)s * q + i) * N + nb(x, y, z, c[0], c[1], c[2], nx, ny, nz)] =
                fs[((int64_t)s * q + i) * N + k];
          }
        }
}

void orc_ml_run(int lat, int64_t nx, int64_t ny, int64_t nz, int32_t nl, double tau,
                const double *Gm, double rho0, double *f, int64_t nsteps, int32_t nsites,
                const int64_t *site_cell, const int32_t *site_lattice, const double *rate,
                double *budget) {
  int q = lat_q(lat);
  int64_t N = nx * ny * nz;
  double *work = (double *)malloc(sizeof(double) * (size_t)((nl * 8 + nl * q) * N));
  for (int64_t t = 0; t < nsteps; ++t)
    orc_ml_step(lat, nx, ny, nz, nl, tau, Gm, rho0, f, work, nsites, site_cell, site_lattice,
                rate, budget);
  free(work);
}

/* Pressure of the coupled lattices (the multicomponent form of the EOS of
 * Sec. 3.1): p = cs^2 sum_s rho_s + cs^2/2 sum_s sum_t Gm[s][t] psi_s psi_t,
 * cs^2 = 1/3.  rho: nl x N densities; p: N. */
void orc_ml_pressure(int64_t N, int32_t nl, const double *rho, const double *Gm, double rho0,
                     double *p) {
  for (int64_t k = 0; k < N; ++k) {
    double r = 0, e = 0;
    for (int32_t s = 0; s < nl; ++s) r += rho[s * N + k];
    for (int32_t s = 0; s < nl; ++s)
      for (int32_t t = 0; t < nl; ++t)
        e += Gm[s * nl + t] * psi_of(rho[s * N + k], rho0) * psi_of(rho[t * N + k], rho0);
    p[k] = r / 3.0 + e / 6.0;
  }
}
