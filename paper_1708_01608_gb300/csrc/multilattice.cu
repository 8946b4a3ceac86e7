// Multi-lattice Shan-Chen model: a reading of the modified model of Sec. 3.1
// and Fig. 1 ("each bubble in its own lattice and fluid in a separate
// lattice"; the lattices are coupled and their interactions computed; eta_m
// switches the barrier off at the rupture criterion and the bubbles merge).
//
// Lattice 0 holds the fluid, lattice k = 1 .. nl-1 the gas of bubble k.
// They interact through the multicomponent Shan-Chen force
//   F_s(x) = -psi_s(x) sum_t Gm[s][t] sum_i w_i psi_t(x + c_i) c_i
// with the coupling matrix Gm[0][0] = G (the fluid's own attraction, the
// single-component model of the hot path), Gm[0][k] = Gm[k][0] = G_x (fluid
// and gas), Gm[k][k] = 0 and Gm[k][l] = eta_m(k, l) G_b between two bubbles.
// Every lattice relaxes with one tau towards f_eq(rho_s, u_s),
//   u' = sum_s j_s / sum_s rho_s,   u_s = u' + tau F_s / rho_s
// (u_s = u' where the lattice is empty: f_eq is 0 there).  eta_m(k, l) = 0
// merges lattice l into k (f_k += f_l, f_l = 0) and removes their coupling.
//
// GB300 form: two passes per step (psi of every lattice into an FP64/FP32
// field, then collide and push every lattice of a cell in one thread),
// populations f[s][i][z][y][x] unpadded, plain values (no offset), FP64 or
// FP32.  The FP64 form keeps the oracle's operation order.  The blowing
// agent of site k deposits w_i dm into lattice k (one thread walks the
// sites in order after the step, on the pushed populations at x_k + c_i).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "lattice.cuh"
#include "lbm.h"

using namespace sclbm;

namespace {

constexpr int ML_MAX = 8;  // lattices: the fluid and up to seven bubbles
constexpr int TPB = 256;

struct MlArgs {
  const void *fin;
  void *fout;
  int64_t NX, NY, NZ;  // view extents (D2Q9 on (nx, 1, ny))
  int nl;
  double tau, rho0;
  double Gm[ML_MAX * ML_MAX];
};

inline int nblocks(int64_t n) {
  const int64_t b = (n + TPB - 1) / TPB;
  return (int)std::min<int64_t>(std::max<int64_t>(b, 1), 262144);
}

__device__ __forceinline__ int wrapv(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// psi = rho0 (1 - exp(-rho/rho0)) in the oracle's operation order
__device__ __forceinline__ double ml_psi(double rho, double rho0) {
  return rho0 * (1.0 - exp(-rho / rho0));
}
__device__ __forceinline__ float ml_psi(float rho, float rho0) {
  return rho0 * (1.0f - expf(-rho / rho0));
}

// pass 1: psi of every lattice at every cell (density summed in velocity order)
template <int LAT, class T>
__global__ void __launch_bounds__(TPB) k_ml_psi(const MlArgs a, T *psi) {
  using L = Lattice<LAT>;
  const int64_t N = a.NX * a.NY * a.NZ;
  const T *f = static_cast<const T *>(a.fin);
  const T rho0 = (T)a.rho0;
  for (int64_t k = blockIdx.x * (int64_t)TPB + threadIdx.x; k < N; k += (int64_t)gridDim.x * TPB)
    for (int s = 0; s < a.nl; ++s) {
      T r = 0;
#pragma unroll
      for (int i = 0; i < L::Q; ++i) r += f[((int64_t)s * L::Q + i) * N + k];
      psi[(int64_t)s * N + k] = ml_psi(r, rho0);
    }
}

// pass 2: moments, common velocity, forces, BGK and push of every lattice
// (the oracle's operation order: the force of lattice s sums over t and i
// jointly, F_s = -psi_s sum, u_s = u' + tau F_s / rho_s where rho_s != 0)
template <int LAT, class T>
__global__ void __launch_bounds__(TPB) k_ml_collide(const MlArgs a, const T *psi) {
  using L = Lattice<LAT>;
  constexpr int Q = L::Q;
  const int64_t N = a.NX * a.NY * a.NZ;
  const T *f = static_cast<const T *>(a.fin);
  T *g = static_cast<T *>(a.fout);
  const int NX = (int)a.NX, NY = (int)a.NY, NZ = (int)a.NZ;
  const T tau = (T)a.tau;
  for (int64_t k = blockIdx.x * (int64_t)TPB + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * TPB) {
    const int x = (int)(k % NX), y = (int)((k / NX) % NY), z = (int)(k / ((int64_t)NX * NY));
    // neighbour cells x + c_i, periodic
    int64_t nbk[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i)
      nbk[i] = ((int64_t)wrapv(z + L::cz(i), NZ) * NY + wrapv(y + L::cy(i), NY)) * NX +
               wrapv(x + L::cx(i), NX);
    T rho[ML_MAX];
    T rt = 0, jtx = 0, jty = 0, jtz = 0;
    for (int s = 0; s < a.nl; ++s) {
      T r = 0, ax = 0, ay = 0, az = 0;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const T v = f[((int64_t)s * Q + i) * N + k];
        r += v;
        ax += v * (T)L::cx(i);
        ay += v * (T)L::cy(i);
        az += v * (T)L::cz(i);
      }
      rho[s] = r;
      rt += r;
      jtx += ax;
      jty += ay;
      jtz += az;
    }
    const T upx = jtx / rt, upy = jty / rt, upz = jtz / rt;
    for (int s = 0; s < a.nl; ++s) {
      T ax = 0, ay = 0, az = 0;
      for (int t = 0; t < a.nl; ++t) {
        const T G = (T)a.Gm[s * ML_MAX + t];
#pragma unroll
        for (int i = 1; i < Q; ++i) {
          const T v = G * (T)L::w(i) * psi[(int64_t)t * N + nbk[i]];
          ax += v * (T)L::cx(i);
          ay += v * (T)L::cy(i);
          az += v * (T)L::cz(i);
        }
      }
      const T ps = psi[(int64_t)s * N + k];
      const T Fx = -ps * ax, Fy = -ps * ay, Fz = -ps * az;
      const T r = rho[s];
      T ux = upx, uy = upy, uz = upz;
      if (r != (T)0) {
        ux += tau * Fx / r;
        uy += tau * Fy / r;
        uz += tau * Fz / r;
      }
      const T uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const T cu = (T)L::cx(i) * ux + (T)L::cy(i) * uy + (T)L::cz(i) * uz;
        const T feq =
            (T)L::w(i) * r * ((T)1 + (T)3 * cu + (T)4.5 * cu * cu - (T)1.5 * uu);
        const T fi = f[((int64_t)s * Q + i) * N + k];
        g[((int64_t)s * Q + i) * N + nbk[i]] = fi - (fi - feq) / tau;
      }
    }
  }
}

// the blowing agent, site by site in order (one thread): dm = min(rate,
// budget) into lattice site_lat[m] at the pushed destinations x_m + c_i
template <int LAT, class T>
__global__ void k_ml_inject(const MlArgs a, int n, const int32_t *sx, const int32_t *sy,
                            const int32_t *sz, const int32_t *slat, const double *rate,
                            double *budget) {
  using L = Lattice<LAT>;
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int64_t N = a.NX * a.NY * a.NZ;
  T *g = static_cast<T *>(a.fout);
  for (int m = 0; m < n; ++m) {
    const double b = budget[m];
    if (b <= 0.0) continue;
    const double dm = rate[m] < b ? rate[m] : b;
    budget[m] = b - dm;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const int64_t cell =
          ((int64_t)wrapv(sz[m] + L::cz(i), (int)a.NZ) * a.NY + wrapv(sy[m] + L::cy(i), (int)a.NY)) *
              a.NX +
          wrapv(sx[m] + L::cx(i), (int)a.NX);
      T *o = g + ((int64_t)slat[m] * L::Q + i) * N + cell;
      *o = *o + (T)(L::w(i) * dm);
    }
  }
}

// eta_m(k, l) = 0: lattice l merged into lattice k
template <class T>
__global__ void __launch_bounds__(TPB) k_ml_merge(T *f, int64_t QN, int k, int l) {
  for (int64_t m = blockIdx.x * (int64_t)TPB + threadIdx.x; m < QN;
       m += (int64_t)gridDim.x * TPB) {
    f[(int64_t)k * QN + m] = f[(int64_t)k * QN + m] + f[(int64_t)l * QN + m];
    f[(int64_t)l * QN + m] = (T)0;
  }
}

// FP64 fields: densities of every lattice (rho: nl x N, may be null) and the
// pressure of the coupled lattices, p = rho_total/3 + 1/6 sum_s sum_t
// Gm[s][t] psi_s psi_t (p may be null)
template <int LAT, class T>
__global__ void __launch_bounds__(TPB) k_ml_fields(const MlArgs a, double *rho_out, double *p) {
  using L = Lattice<LAT>;
  const int64_t N = a.NX * a.NY * a.NZ;
  const T *f = static_cast<const T *>(a.fin);
  for (int64_t k = blockIdx.x * (int64_t)TPB + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * TPB) {
    double rho[ML_MAX];
    double rt = 0.0;
    for (int s = 0; s < a.nl; ++s) {
      double r = 0.0;
#pragma unroll
      for (int i = 0; i < L::Q; ++i) r += (double)f[((int64_t)s * L::Q + i) * N + k];
      rho[s] = r;
      rt += r;
      if (rho_out) rho_out[(int64_t)s * N + k] = r;
    }
    if (p) {
      double e = 0.0;
      for (int s = 0; s < a.nl; ++s)
        for (int t = 0; t < a.nl; ++t)
          e += a.Gm[s * ML_MAX + t] * ml_psi(rho[s], a.rho0) * ml_psi(rho[t], a.rho0);
      p[k] = rt / 3.0 + e / 6.0;
    }
  }
}

// f (device, storage type) <-> doubles f[(s*Q + i)*N + user cell]; the
// view's cell order equals the user's (D2Q9: (x, 1, y) has the same linear
// index as (x, y))
template <class T>
__global__ void __launch_bounds__(TPB) k_ml_to_double(const T *f, int64_t n, double *out) {
  for (int64_t m = blockIdx.x * (int64_t)TPB + threadIdx.x; m < n; m += (int64_t)gridDim.x * TPB)
    out[m] = (double)f[m];
}
template <class T>
__global__ void __launch_bounds__(TPB) k_ml_from_double(const double *in, int64_t n, T *f) {
  for (int64_t m = blockIdx.x * (int64_t)TPB + threadIdx.x; m < n; m += (int64_t)gridDim.x * TPB)
    f[m] = (T)in[m];
}
// f = w_i rho (at rest) for one lattice from an FP64 density field
template <int LAT, class T>
__global__ void __launch_bounds__(TPB) k_ml_rest(const double *rho, int64_t N, T *f) {
  using L = Lattice<LAT>;
  for (int64_t k = blockIdx.x * (int64_t)TPB + threadIdx.x; k < N; k += (int64_t)gridDim.x * TPB)
#pragma unroll
    for (int i = 0; i < L::Q; ++i) f[(int64_t)i * N + k] = (T)(L::w(i) * rho[k]);
}

thread_local std::string g_ml_err;

}  // namespace

struct lbm_ml_ctx {
  lbm_ml_config cfg;
  int lat = 0, Q = 0, nl = 0;
  bool f64 = true;
  View v{};
  int64_t N = 0;
  cudaStream_t s = nullptr;
  void *fA = nullptr, *fB = nullptr, *psi = nullptr;
  size_t lat_bytes = 0;
  double *d_rho = nullptr, *d_p = nullptr, *d_tmp = nullptr, *d_bub = nullptr;
  double *d_rate = nullptr, *d_budget = nullptr;
  int32_t *d_site = nullptr;  // x, y, z, lattice per site (view coordinates)
  int32_t nsites = 0;
  std::vector<int32_t> site_xyz;
  int cur = 0;
  bool seeded = false;
  int64_t steps = 0;
  double Gm[ML_MAX * ML_MAX] = {};
  std::vector<std::pair<void **, size_t>> owned;
};

namespace {

lbm_status ml_fail(lbm_status st, const std::string &m) {
  sclbm::set_error(st, m.c_str());
  return st;
}

#define MLCK(call)                                                                   \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      cudaGetLastError();                                                            \
      return ml_fail(LBM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    }                                                                                \
  } while (0)
#define MLCKS(expr)              \
  do {                           \
    lbm_status s_ = (expr);      \
    if (s_ != LBM_OK) return s_; \
  } while (0)

lbm_status ml_alloc(lbm_ml_ctx *c, void **p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (c->cfg.alloc) {
    *p = c->cfg.alloc(bytes, c->cfg.stream, c->cfg.alloc_user);
    if (!*p) return ml_fail(LBM_ENOMEM, "device allocation failed");
  } else if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return ml_fail(LBM_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  c->owned.push_back({p, bytes});
  return LBM_OK;
}

void ml_free_all(lbm_ml_ctx *c) {
  for (auto &o : c->owned)
    if (*o.first) {
      if (c->cfg.free)
        c->cfg.free(*o.first, o.second, c->cfg.stream, c->cfg.alloc_user);
      else
        cudaFree(*o.first);
      *o.first = nullptr;
    }
  c->owned.clear();
}

// a device staging buffer released when it goes out of scope (through the
// context's allocator when it has one)
struct MlTemp {
  lbm_ml_ctx *c;
  void *p = nullptr;
  size_t bytes = 0;
  MlTemp(lbm_ml_ctx *c_, size_t b) : c(c_), bytes(b) {
    if (c->cfg.alloc) {
      p = c->cfg.alloc(bytes, c->cfg.stream, c->cfg.alloc_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
  }
  ~MlTemp() {
    if (!p) return;
    cudaStreamSynchronize(c->s);
    if (c->cfg.free)
      c->cfg.free(p, bytes, c->cfg.stream, c->cfg.alloc_user);
    else
      cudaFree(p);
  }
};

MlArgs ml_args(const lbm_ml_ctx *c) {
  MlArgs a{};
  a.fin = c->cur == 0 ? c->fA : c->fB;
  a.fout = c->cur == 0 ? c->fB : c->fA;
  a.NX = c->v.NX;
  a.NY = c->v.NY;
  a.NZ = c->v.NZ;
  a.nl = c->nl;
  a.tau = c->cfg.tau;
  a.rho0 = c->cfg.rho0;
  std::memcpy(a.Gm, c->Gm, sizeof(a.Gm));
  return a;
}

template <class Fn>
cudaError_t ml_dispatch(const lbm_ml_ctx *c, Fn fn) {
  if (c->lat == D3Q19) {
    if (c->f64)
      fn(std::integral_constant<int, D3Q19>{}, double{});
    else
      fn(std::integral_constant<int, D3Q19>{}, float{});
  } else {
    if (c->f64)
      fn(std::integral_constant<int, D2Q9>{}, double{});
    else
      fn(std::integral_constant<int, D2Q9>{}, float{});
  }
  return cudaGetLastError();
}

lbm_status ml_sync(lbm_ml_ctx *c) {
  MLCK(cudaStreamSynchronize(c->s));
  return LBM_OK;
}

}  // namespace

extern "C" {

void lbm_ml_config_default(lbm_ml_config *cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->lattice = LBM_D2Q9;
  cfg->storage = LBM_F64;
  cfg->nx = cfg->ny = 128;
  cfg->nz = 1;
  cfg->nl = 3;
  cfg->tau = 1.0;
  cfg->rho0 = 1.0;
  cfg->G = -5.0;
  cfg->G_x = 1.0;
  cfg->G_b = 0.0;
}

lbm_status lbm_ml_create(const lbm_ml_config *cfg, lbm_ml_ctx **out) {
  if (!out) return ml_fail(LBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfg) return ml_fail(LBM_EINVAL, "cfg is NULL");
  if (cfg->lattice != LBM_D2Q9 && cfg->lattice != LBM_D3Q19)
    return ml_fail(LBM_EINVAL, "unknown lattice");
  if (cfg->storage != LBM_F64 && cfg->storage != LBM_F32)
    return ml_fail(LBM_EINVAL, "the multi-lattice model stores FP64 or FP32 populations");
  if (cfg->nl < 1 || cfg->nl > ML_MAX) return ml_fail(LBM_EINVAL, "nl must be 1..8");
  if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1 || (cfg->lattice == LBM_D2Q9 && cfg->nz != 1))
    return ml_fail(LBM_EINVAL, "extents must be >= 1 (nz = 1 for D2Q9)");
  if (cfg->nx > (1 << 20) || cfg->ny > (1 << 20) || cfg->nz > (1 << 20) ||
      cfg->nx * cfg->ny > ((int64_t)1 << 40) / cfg->nz)
    return ml_fail(LBM_EINVAL, "lattice too large");
  if (!(cfg->tau > 0.5) || !std::isfinite(cfg->tau) || !(cfg->rho0 > 0) ||
      !std::isfinite(cfg->rho0) || !std::isfinite(cfg->G) || !std::isfinite(cfg->G_x) ||
      !std::isfinite(cfg->G_b))
    return ml_fail(LBM_EINVAL, "tau finite and > 0.5, rho0 finite and > 0, couplings finite");
  if ((cfg->alloc == nullptr) != (cfg->free == nullptr))
    return ml_fail(LBM_EINVAL, "alloc and free callbacks must be given together");
  lbm_ml_ctx *c = new lbm_ml_ctx();
  c->cfg = *cfg;
  c->lat = cfg->lattice == LBM_D2Q9 ? D2Q9 : D3Q19;
  c->Q = c->lat == D3Q19 ? 19 : 9;
  c->nl = cfg->nl;
  c->f64 = cfg->storage == LBM_F64;
  c->s = static_cast<cudaStream_t>(cfg->stream);
  c->v.lat = c->lat;
  c->v.st = c->f64 ? ST_F64 : ST_F32;
  c->v.NX = cfg->nx;
  c->v.NY = c->lat == D2Q9 ? 1 : cfg->ny;
  c->v.NZ = c->lat == D2Q9 ? cfg->ny : cfg->nz;
  c->v.px = c->v.NX;
  c->v.rho_ref = 0.0;
  view_prepare(c->v);
  c->N = c->v.NX * c->v.NY * c->v.NZ;
  // coupling matrix of the reading above; eta_m = 1 for every pair
  for (int s = 0; s < c->nl; ++s)
    for (int t = 0; t < c->nl; ++t)
      c->Gm[s * ML_MAX + t] =
          (s == 0 && t == 0) ? cfg->G : ((s == 0 || t == 0) ? cfg->G_x : (s == t ? 0.0 : cfg->G_b));
  const size_t ts = c->f64 ? 8 : 4;
  c->lat_bytes = ts * (size_t)c->nl * c->Q * c->N;
  lbm_status st;
  auto bail = [&](lbm_status e) {
    lbm_ml_destroy(c);
    return e;
  };
  if ((st = ml_alloc(c, &c->fA, c->lat_bytes)) != LBM_OK) return bail(st);
  if ((st = ml_alloc(c, &c->fB, c->lat_bytes)) != LBM_OK) return bail(st);
  if ((st = ml_alloc(c, &c->psi, ts * (size_t)c->nl * c->N)) != LBM_OK) return bail(st);
  if ((st = ml_alloc(c, (void **)&c->d_rho, sizeof(double) * (size_t)c->nl * c->N)) != LBM_OK)
    return bail(st);
  if ((st = ml_alloc(c, (void **)&c->d_p, sizeof(double) * (size_t)c->N)) != LBM_OK) return bail(st);
  if ((st = ml_alloc(c, (void **)&c->d_tmp, sizeof(double) * (size_t)std::max<int64_t>(c->N, 8))) !=
      LBM_OK)
    return bail(st);
  if ((st = ml_alloc(c, (void **)&c->d_bub, sizeof(double) * 4 * ML_MAX)) != LBM_OK) return bail(st);
  if ((st = ml_alloc(c, (void **)&c->d_rate, sizeof(double) * ML_MAX)) != LBM_OK) return bail(st);
  if ((st = ml_alloc(c, (void **)&c->d_budget, sizeof(double) * ML_MAX)) != LBM_OK) return bail(st);
  if ((st = ml_alloc(c, (void **)&c->d_site, sizeof(int32_t) * 4 * ML_MAX)) != LBM_OK)
    return bail(st);
  if (cudaMemsetAsync(c->fA, 0, c->lat_bytes, c->s) != cudaSuccess ||
      cudaMemsetAsync(c->fB, 0, c->lat_bytes, c->s) != cudaSuccess) {
    cudaGetLastError();
    return bail(ml_fail(LBM_ECUDA, "memset failed"));
  }
  *out = c;
  return LBM_OK;
}

void lbm_ml_destroy(lbm_ml_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->s);
  cudaGetLastError();
  ml_free_all(c);
  delete c;
}

lbm_status lbm_ml_coupling(const lbm_ml_ctx *c, double *Gm) {
  if (!c || !Gm) return ml_fail(LBM_EINVAL, "NULL argument");
  for (int s = 0; s < c->nl; ++s)
    for (int t = 0; t < c->nl; ++t) Gm[s * c->nl + t] = c->Gm[s * ML_MAX + t];
  return LBM_OK;
}

lbm_status lbm_ml_seed(lbm_ml_ctx *c, const lbm_bubble *b, double rho_l, double rho_v,
                       double rho_gas, double width, double noise_amp, uint64_t seed) {
  if (!c) return ml_fail(LBM_EINVAL, "ctx is NULL");
  const int nb = c->nl - 1;
  if (nb > 0 && !b) return ml_fail(LBM_EINVAL, "need nl - 1 bubbles");
  if (!(width > 0) || !std::isfinite(rho_l) || !std::isfinite(rho_v) || !std::isfinite(rho_gas) ||
      !std::isfinite(noise_amp))
    return ml_fail(LBM_EINVAL, "width > 0, densities finite");
  std::vector<double> vb(4 * ML_MAX, 0.0);
  c->site_xyz.assign(4 * ML_MAX, 0);
  for (int k = 0; k < nb; ++k) {
    if (!std::isfinite(b[k].x) || !std::isfinite(b[k].y) || !std::isfinite(b[k].z) ||
        !std::isfinite(b[k].r))
      return ml_fail(LBM_EINVAL, "non-finite bubble");
    double vx = b[k].x, vy = b[k].y, vz = b[k].z;
    if (c->lat == D2Q9) {
      vz = b[k].y;
      vy = 0.0;
    }
    vb[4 * k + 0] = vx;
    vb[4 * k + 1] = vy;
    vb[4 * k + 2] = vz;
    vb[4 * k + 3] = b[k].r;
    auto wr = [](double p, int64_t n) {
      int64_t q = (int64_t)std::floor(p + 0.5) % n;
      return (int32_t)(q < 0 ? q + n : q);
    };
    c->site_xyz[4 * k + 0] = wr(vx, c->v.NX);
    c->site_xyz[4 * k + 1] = wr(vy, c->v.NY);
    c->site_xyz[4 * k + 2] = wr(vz, c->v.NZ);
    c->site_xyz[4 * k + 3] = k + 1;
  }
  MLCK(cudaMemcpyAsync(c->d_bub, vb.data(), sizeof(double) * vb.size(), cudaMemcpyHostToDevice, c->s));
  c->cur = 0;
  double *rho = c->d_tmp;
  const int64_t QN = (int64_t)c->Q * c->N;
  // the fluid: every bubble, liquid rho_l, its vapour rho_v inside, noise
  MLCK(diag_init_rho(c->v, c->d_bub, nb, rho_l, rho_v, width, noise_amp, seed, rho, c->s));
  MLCK(ml_dispatch(c, [&](auto L, auto T) {
    using TT = decltype(T);
    k_ml_rest<decltype(L)::value, TT><<<nblocks(c->N), TPB, 0, c->s>>>(rho, c->N,
                                                                        static_cast<TT *>(c->fA));
  }));
  // bubble k's gas: rho_gas inside bubble k, zero far outside, no noise
  for (int k = 0; k < nb; ++k) {
    MLCK(diag_init_rho(c->v, c->d_bub + 4 * k, 1, 0.0, rho_gas, width, 0.0, seed, rho, c->s));
    MLCK(ml_dispatch(c, [&](auto L, auto T) {
      using TT = decltype(T);
      k_ml_rest<decltype(L)::value, TT><<<nblocks(c->N), TPB, 0, c->s>>>(
          rho, c->N, static_cast<TT *>(c->fA) + (int64_t)(k + 1) * QN);
    }));
  }
  // every pair's barrier back on
  for (int s = 0; s < c->nl; ++s)
    for (int t = 0; t < c->nl; ++t)
      if (s != t && s > 0 && t > 0) c->Gm[s * ML_MAX + t] = c->cfg.G_b;
  c->nsites = 0;
  c->steps = 0;
  c->seeded = true;
  return ml_sync(c);
}

lbm_status lbm_ml_write_f(lbm_ml_ctx *c, const double *f, size_t bytes) {
  if (!c || !f) return ml_fail(LBM_EINVAL, "NULL argument");
  const int64_t n = (int64_t)c->nl * c->Q * c->N;
  if (bytes != (size_t)n * sizeof(double)) return ml_fail(LBM_EINVAL, "bytes must be nl*Q*N*8");
  MlTemp tmp(c, bytes);
  if (!tmp.p) return ml_fail(LBM_ENOMEM, "staging allocation failed");
  double *d = static_cast<double *>(tmp.p);
  MLCK(cudaMemcpyAsync(d, f, bytes, cudaMemcpyHostToDevice, c->s));
  void *dst = c->cur == 0 ? c->fA : c->fB;
  MLCK(ml_dispatch(c, [&](auto, auto T) {
    using TT = decltype(T);
    k_ml_from_double<TT><<<nblocks(n), TPB, 0, c->s>>>(d, n, static_cast<TT *>(dst));
  }));
  MLCKS(ml_sync(c));
  c->seeded = true;
  return LBM_OK;
}

lbm_status lbm_ml_read_f(lbm_ml_ctx *c, double *f, size_t bytes) {
  if (!c || !f) return ml_fail(LBM_EINVAL, "NULL argument");
  if (!c->seeded) return ml_fail(LBM_ESTATE, "seed the lattices first");
  const int64_t n = (int64_t)c->nl * c->Q * c->N;
  if (bytes != (size_t)n * sizeof(double)) return ml_fail(LBM_EINVAL, "bytes must be nl*Q*N*8");
  MlTemp tmp(c, bytes);
  if (!tmp.p) return ml_fail(LBM_ENOMEM, "staging allocation failed");
  double *d = static_cast<double *>(tmp.p);
  const void *src = c->cur == 0 ? c->fA : c->fB;
  MLCK(ml_dispatch(c, [&](auto, auto T) {
    using TT = decltype(T);
    k_ml_to_double<TT><<<nblocks(n), TPB, 0, c->s>>>(static_cast<const TT *>(src), n, d);
  }));
  MLCK(cudaMemcpyAsync(f, d, bytes, cudaMemcpyDeviceToHost, c->s));
  return ml_sync(c);
}

lbm_status lbm_ml_inject(lbm_ml_ctx *c, const double *rate, const double *budget, int32_t n) {
  if (!c) return ml_fail(LBM_EINVAL, "ctx is NULL");
  if (!c->seeded) return ml_fail(LBM_ESTATE, "seed the lattices first");
  if (n == 0) {
    c->nsites = 0;
    return LBM_OK;
  }
  if (n != c->nl - 1 || !rate || !budget)
    return ml_fail(LBM_EINVAL, "n must be 0 or the number of bubbles (nl - 1)");
  for (int k = 0; k < n; ++k)
    if (!(rate[k] >= 0) || !(budget[k] >= 0) || !std::isfinite(rate[k]) || !std::isfinite(budget[k]))
      return ml_fail(LBM_EINVAL, "rates and budgets must be finite and >= 0");
  MLCK(cudaMemcpyAsync(c->d_rate, rate, sizeof(double) * n, cudaMemcpyHostToDevice, c->s));
  MLCK(cudaMemcpyAsync(c->d_budget, budget, sizeof(double) * n, cudaMemcpyHostToDevice, c->s));
  // site lists x, y, z, lattice as four arrays of ML_MAX
  std::vector<int32_t> sites(4 * ML_MAX, 0);
  for (int k = 0; k < n; ++k)
    for (int q = 0; q < 4; ++q) sites[q * ML_MAX + k] = c->site_xyz[4 * k + q];
  MLCK(cudaMemcpyAsync(c->d_site, sites.data(), sizeof(int32_t) * sites.size(),
                       cudaMemcpyHostToDevice, c->s));
  MLCKS(ml_sync(c));
  c->nsites = n;
  return LBM_OK;
}

lbm_status lbm_ml_read_budgets(lbm_ml_ctx *c, double *budget, int32_t n) {
  if (!c || !budget) return ml_fail(LBM_EINVAL, "NULL argument");
  if (n != c->nsites) return ml_fail(LBM_EINVAL, "n must equal the number of injecting sites");
  if (n == 0) return LBM_OK;
  MLCK(cudaMemcpyAsync(budget, c->d_budget, sizeof(double) * n, cudaMemcpyDeviceToHost, c->s));
  return ml_sync(c);
}

lbm_status lbm_ml_step(lbm_ml_ctx *c, int64_t nsteps) {
  if (!c) return ml_fail(LBM_EINVAL, "ctx is NULL");
  if (nsteps < 0) return ml_fail(LBM_EINVAL, "nsteps < 0");
  if (!c->seeded) return ml_fail(LBM_ESTATE, "seed the lattices first");
  for (int64_t t = 0; t < nsteps; ++t) {
    const MlArgs a = ml_args(c);
    cudaError_t e = ml_dispatch(c, [&](auto L, auto T) {
      using TT = decltype(T);
      constexpr int lat = decltype(L)::value;
      k_ml_psi<lat, TT><<<nblocks(c->N), TPB, 0, c->s>>>(a, static_cast<TT *>(c->psi));
      k_ml_collide<lat, TT><<<nblocks(c->N), TPB, 0, c->s>>>(a, static_cast<const TT *>(c->psi));
      if (c->nsites > 0)
        k_ml_inject<lat, TT><<<1, 32, 0, c->s>>>(a, c->nsites, c->d_site, c->d_site + ML_MAX,
                                                  c->d_site + 2 * ML_MAX, c->d_site + 3 * ML_MAX,
                                                  c->d_rate, c->d_budget);
    });
    if (e != cudaSuccess) {
      cudaGetLastError();
      return ml_fail(LBM_ECUDA, std::string("multi-lattice step: ") + cudaGetErrorString(e));
    }
    c->cur = 1 - c->cur;
    ++c->steps;
  }
  return LBM_OK;
}

int64_t lbm_ml_step_count(const lbm_ml_ctx *c) { return c ? c->steps : -1; }

lbm_status lbm_ml_merge(lbm_ml_ctx *c, int32_t k, int32_t l) {
  if (!c) return ml_fail(LBM_EINVAL, "ctx is NULL");
  if (!c->seeded) return ml_fail(LBM_ESTATE, "seed the lattices first");
  if (k < 1 || l < 1 || k >= c->nl || l >= c->nl || k == l)
    return ml_fail(LBM_EINVAL, "k and l must be two different bubble lattices (1 .. nl-1)");
  const int64_t QN = (int64_t)c->Q * c->N;
  void *f = c->cur == 0 ? c->fA : c->fB;
  MLCK(ml_dispatch(c, [&](auto, auto T) {
    using TT = decltype(T);
    k_ml_merge<TT><<<nblocks(QN), TPB, 0, c->s>>>(static_cast<TT *>(f), QN, k, l);
  }));
  c->Gm[k * ML_MAX + l] = c->Gm[l * ML_MAX + k] = 0.0;
  return ml_sync(c);
}

lbm_status lbm_ml_fields(lbm_ml_ctx *c, double *rho, double *p) {
  if (!c) return ml_fail(LBM_EINVAL, "ctx is NULL");
  if (!c->seeded) return ml_fail(LBM_ESTATE, "seed the lattices first");
  const MlArgs a = ml_args(c);
  MLCK(ml_dispatch(c, [&](auto L, auto T) {
    k_ml_fields<decltype(L)::value, decltype(T)><<<nblocks(c->N), TPB, 0, c->s>>>(a, c->d_rho, c->d_p);
  }));
  if (rho)
    MLCK(cudaMemcpyAsync(rho, c->d_rho, sizeof(double) * (size_t)c->nl * c->N,
                         cudaMemcpyDeviceToHost, c->s));
  if (p) MLCK(cudaMemcpyAsync(p, c->d_p, sizeof(double) * (size_t)c->N, cudaMemcpyDeviceToHost, c->s));
  return ml_sync(c);
}

lbm_status lbm_ml_run_until_rupture(lbm_ml_ctx *c, const int64_t *line, double rho_mid,
                                     double eps_arm, double h_max, int64_t diag_every,
                                     int64_t max_steps, int32_t k, int32_t l, lbm_rupture *out) {
  if (!c || !line || !out) return ml_fail(LBM_EINVAL, "NULL argument");
  if (!c->seeded) return ml_fail(LBM_ESTATE, "seed the lattices first");
  const int dims = c->lat == D2Q9 ? 2 : 3;
  if (line[3] < 0 || line[3] >= dims || line[4] < 2)
    return ml_fail(LBM_EINVAL, "line = {x, y, z, axis (< dims), len >= 2}");
  if (diag_every < 1 || max_steps < 0 || !(eps_arm >= 0) || !(h_max > 0))
    return ml_fail(LBM_EINVAL, "diag_every >= 1, max_steps >= 0, eps_arm >= 0, h_max > 0");
  if (k < 1 || l < 1 || k >= c->nl || l >= c->nl || k == l)
    return ml_fail(LBM_EINVAL, "k and l must be two different bubble lattices (1 .. nl-1)");
  std::memset(out, 0, sizeof(*out));
  auto vaxis = [&](int a) { return c->lat == D2Q9 ? (a == 0 ? 0 : 2) : a; };
  int e[3] = {0, 0, 0}, ep[3] = {0, 0, 0};
  e[vaxis((int)line[3])] = 1;
  ep[vaxis(((int)line[3] + 1) % dims)] = 1;
  int64_t x0 = line[0], y0 = line[1], z0 = line[2];
  if (c->lat == D2Q9) {
    z0 = y0;
    y0 = 0;
  }
  auto wr = [](int64_t a, int64_t n) {
    const int64_t r = a % n;
    return r < 0 ? r + n : r;
  };
  bool armed = false;
  double h_prev = 0.0, d_prev = 0.0;
  double h[6];
  int64_t t = 0;
  while (t < max_steps) {
    const int64_t n = std::min(diag_every, max_steps - t);
    MLCKS(lbm_ml_step(c, n));
    t += n;
    // the film on the fluid lattice's density, with the coupled pressure
    MLCKS(lbm_ml_fields(c, nullptr, nullptr));
    MLCK(diag_film_probe(c->v, c->d_rho, c->d_p, wr(x0, c->v.NX), wr(y0, c->v.NY), wr(z0, c->v.NZ),
                         e, ep, line[4], rho_mid, c->d_tmp, c->s));
    MLCK(cudaMemcpyAsync(h, c->d_tmp, sizeof(h), cudaMemcpyDeviceToHost, c->s));
    MLCKS(ml_sync(c));
    out->steps = t;
    const bool found = h[0] != 0.0;
    const double hh = h[3], d2 = h[4];
    if (!found) {  // the film is gone before the criterion fired
      out->merged = 1;
      return LBM_OK;
    }
    if (hh > h_max) {
      armed = false;
    } else if (d2 < -eps_arm) {
      armed = true;
    } else if (armed && d2 >= 0.0) {
      // eta_m = 0: the barrier goes and the pair's lattices merge
      out->fired = 1;
      out->h_c = h_prev + (hh - h_prev) * (-d_prev / (d2 - d_prev));
      out->h_probe = hh;
      out->r_d = h[5];
      return lbm_ml_merge(c, k, l);
    }
    h_prev = hh;
    d_prev = d2;
  }
  return LBM_OK;
}

}  // extern "C"
