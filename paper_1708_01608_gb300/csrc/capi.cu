// C ABI of the library: context management, host-side bookkeeping
// (nucleation sites, injection buckets, merge events) and the calls that
// enqueue the kernels.  See include/lbm.h for the contract of every entry
// point.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "internal.h"
#include "lattice.cuh"
#include "lbm.h"

using namespace sclbm;

namespace {

thread_local std::string g_err;

lbm_status fail(lbm_status st, const std::string &msg) {
  g_err = msg;
  return st;
}

#define CK(call)                                                                             \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      cudaGetLastError();                                                                    \
      return fail(LBM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));           \
    }                                                                                        \
  } while (0)
#define CKS(expr)                       \
  do {                                  \
    lbm_status s_ = (expr);             \
    if (s_ != LBM_OK) return s_;        \
  } while (0)

struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
};
struct PinBuf {  // pinned host memory
  void *p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct lbm_ctx {
  lbm_config cfg;
  int lat = 0, st = 0, Q = 0;
  View v{};
  int64_t N = 0;
  cudaStream_t s = nullptr;
  int device = 0;
  size_t lat_bytes = 0;
  DevBuf fA, fB;
  int cur = 0;  // 0: state in fA, 1: state in fB
  // 16-bit storage with the per-cell FP32 rounding residual (mass_residual):
  // the step kernels run in the residual forms ST_F16R / ST_BF16R
  bool resid = false;
  int st_step = 0;  // storage form of the step kernels
  DevBuf d_resid;
  bool seeded = false;
  int64_t steps = 0;
  lbm_status sticky = LBM_OK;
  // nucleation sites (user coordinates) and their cells in the view
  std::vector<lbm_bubble> bubbles;
  std::vector<int32_t> sx, sy, sz;
  int32_t ninj = 0;  // > 0 while injection is on
  DevBuf d_sx, d_sy, d_sz, d_rate, d_budget, d_goff, d_gsite, d_boff, d_blist, d_cells, d_bub;
  int32_t ngroups = 0;
  // fused kernel
  int kernel = LBM_KERNEL_FUSED;
  FusedPlan plan{};
  FusedMaps tmA{}, tmB{};
  DevBuf psi_scratch;
  // diagnostics
  DevBuf d_err, d_rho, d_p, d_tmp, d_j, d_u, d_labels, d_ncomp, d_part, d_tot, d_site_lab;
  // bubble census and per-point film test
  DevBuf d_count, d_census, d_film_state, d_film_counts, d_film_rec, d_film_save, d_film_mids;
  int64_t film_mid_queue = 0;  // capacity of d_film_mids (queued film midpoints)
  bool film_state_clear = false;  // d_film_state must be zeroed before use
  int64_t census_cap = 4096;       // device capacity of the census list (grows)
  int64_t film_mid_cap = 1 << 16;  // device capacity of the midpoint records (grows)
  // injection mode: 0 at the site cell (inside the step kernels), 1 spread
  // over the site's bubble (inject.cu)
  int inj_mode = 0;
  DevBuf d_spread_groups, d_spread_sites, d_spread_count, d_dep;
  // d_rho / d_p hold the FP64 density and pressure of the current state;
  // d_labels its gas labels (cleared by stepping and by state writes)
  bool p_valid = false, labels_valid = false;
  std::vector<int32_t> site_labels, prev_site_labels;
  bool have_prev = false;
  int64_t merge_events = 0;
  // Pinned host memory for results read back after a call's one stream
  // synchronisation: the status word, the site labels of the last labelling
  // (copied to site_labels at that synchronisation) and a mailbox for the
  // results of one call.  Pageable targets would make each copy a staged,
  // serialising transfer.
  PinBuf h_err, h_site, h_mail;
  bool site_pending = false;
};

namespace {

void hfree(PinBuf &b) {
  if (b.p) cudaFreeHost(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

// grow a pinned host buffer (the stream is drained first: no copy may still
// target the old one)
lbm_status halloc(lbm_ctx *c, PinBuf &b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.p && b.bytes >= bytes) return LBM_OK;
  if (b.p) cudaStreamSynchronize(c->s);
  hfree(b);
  void *p = nullptr;
  if (cudaMallocHost(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(LBM_ENOMEM, "pinned host allocation of " + std::to_string(bytes) + " bytes failed");
  }
  b.p = p;
  b.bytes = bytes;
  return LBM_OK;
}

void dfree(lbm_ctx *c, DevBuf &b) {
  if (!b.p) return;
  if (c->cfg.alloc && c->cfg.free)
    c->cfg.free(b.p, b.bytes, c->s, c->cfg.alloc_user);
  else if (!c->cfg.alloc)
    cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

lbm_status dalloc(lbm_ctx *c, DevBuf &b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.p && b.bytes >= bytes) return LBM_OK;
  dfree(c, b);
  void *p = nullptr;
  if (c->cfg.alloc) {
    p = c->cfg.alloc(bytes, c->s, c->cfg.alloc_user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (!p) return fail(LBM_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  b.p = p;
  b.bytes = bytes;
  return LBM_OK;
}

template <typename T>
lbm_status upload(lbm_ctx *c, DevBuf &b, const std::vector<T> &h) {
  CKS(dalloc(c, b, h.size() * sizeof(T)));
  if (!h.empty()) CK(cudaMemcpyAsync(b.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, c->s));
  return LBM_OK;
}

int64_t wrap64(int64_t a, int64_t n) {
  int64_t r = a % n;
  return r < 0 ? r + n : r;
}

// SplitMix64 (Steele, Lea & Flood 2014): k-th output of the generator whose
// state starts at key.
uint64_t splitmix64_at(uint64_t key, uint64_t k) {
  uint64_t z = key + (k + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double unit_at(uint64_t key, uint64_t k) {
  return (double)(splitmix64_at(key, k) >> 11) * (1.0 / 9007199254740992.0);
}
double min_image(double d, double n) {
  d = std::fmod(d, n);
  if (d < 0) d += n;
  if (d > 0.5 * n) d -= n;
  return d;
}

lbm_status check_sticky(lbm_ctx *c) {
  if (c->sticky != LBM_OK) return fail(c->sticky, "an earlier device error is pending on this context");
  return LBM_OK;
}

// Read and clear nothing: report the device status word after a sync.
lbm_status sync_and_check(lbm_ctx *c) {
  CKS(halloc(c, c->h_err, sizeof(int)));
  int *herr = static_cast<int *>(c->h_err.p);
  CK(cudaMemcpyAsync(herr, c->d_err.p, sizeof(int), cudaMemcpyDeviceToHost, c->s));
  CK(cudaStreamSynchronize(c->s));
  const int err = *herr;
  if (c->site_pending) {
    const int32_t *hs = static_cast<const int32_t *>(c->h_site.p);
    c->site_labels.assign(hs, hs + c->sx.size());
    c->site_pending = false;
  }
  if (err & ERR_TMA_TIMEOUT) {
    c->sticky = LBM_ETIMEOUT;
    return fail(LBM_ETIMEOUT, "a step kernel gave up waiting for a TMA transfer");
  }
  if (err & ERR_NONFINITE) {
    CK(cudaMemsetAsync(c->d_err.p, 0, sizeof(int), c->s));
    CK(cudaStreamSynchronize(c->s));
    return fail(LBM_ENUMERIC, "non-finite density found");
  }
  return LBM_OK;
}

void *lattice_ptr(lbm_ctx *c, int which) { return which == 0 ? c->fA.p : c->fB.p; }

lbm_status build_buckets(lbm_ctx *c) {
  // per fused work item, the sites it owns sorted by (z, site index)
  const int n = (int)c->sx.size();
  std::vector<std::pair<std::pair<int, int>, int>> keyed;
  keyed.reserve(n);
  for (int s = 0; s < n; ++s)
    keyed.push_back({{fused_item_of(c->plan, c->sx[s], c->sy[s], c->sz[s]), c->sz[s]}, s});
  std::sort(keyed.begin(), keyed.end());
  std::vector<int32_t> off(c->plan.items + 1, 0), list(n);
  for (int q = 0; q < n; ++q) {
    off[keyed[q].first.first + 1]++;
    list[q] = keyed[q].second;
  }
  for (int it = 0; it < c->plan.items; ++it) off[it + 1] += off[it];
  CKS(upload(c, c->d_boff, off));
  CKS(upload(c, c->d_blist, list));
  return LBM_OK;
}

lbm_status ensure_diag(lbm_ctx *c) {
  const size_t nd = (size_t)c->N * sizeof(double);
  CKS(dalloc(c, c->d_rho, nd));
  CKS(dalloc(c, c->d_p, nd));
  CKS(dalloc(c, c->d_tmp, nd));
  CKS(dalloc(c, c->d_part,
             4 * sizeof(double) * std::max(diag_totals_blocks(), diag_scan_blocks())));
  CKS(dalloc(c, c->d_tot, 4 * sizeof(double)));
  CKS(dalloc(c, c->d_ncomp, sizeof(unsigned long long)));
  return LBM_OK;
}

lbm_status set_device(lbm_ctx *c) {
  int d = -1;
  CK(cudaGetDevice(&d));
  if (d != c->device) CK(cudaSetDevice(c->device));
  return LBM_OK;
}

}  // namespace

// record a failure for lbm_last_error() from another translation unit
lbm_status sclbm::set_error(lbm_status st, const char *msg) { return fail(st, msg); }


extern "C" {

const char *lbm_last_error(void) { return g_err.c_str(); }

const char *lbm_version(void) { return "sclbm-gb300 0.1 (sm_103a)"; }

void lbm_config_default(lbm_config *cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->lattice = LBM_D3Q19;
  cfg->storage = LBM_F32;
  cfg->nx = cfg->ny = cfg->nz = 64;
  cfg->tau = 1.0;
  cfg->G = -5.0;
  cfg->rho0 = 1.0;
  cfg->rho_ref = 1.0;
  cfg->gas_threshold = 1.0;
  cfg->kernel = LBM_KERNEL_AUTO;
  cfg->tile = 0;
  cfg->nucleus_radius = 3.0;
}

lbm_status lbm_create(const lbm_config *cfg, lbm_ctx **out) {
  if (!out) return fail(LBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!cfg) return fail(LBM_EINVAL, "cfg is NULL");
  if (cfg->lattice != LBM_D2Q9 && cfg->lattice != LBM_D3Q19) return fail(LBM_EINVAL, "unknown lattice");
  if (cfg->storage < LBM_F64 || cfg->storage > LBM_BF16_OFFSET) return fail(LBM_EINVAL, "unknown storage");
  if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1) return fail(LBM_EINVAL, "extents must be >= 1");
  if (cfg->lattice == LBM_D2Q9 && cfg->nz != 1) return fail(LBM_EINVAL, "D2Q9 needs nz == 1");
  if (cfg->nx > (1 << 20) || cfg->ny > (1 << 20) || cfg->nz > (1 << 20) ||
      ((cfg->nx + 7) / 8 * 8) * cfg->ny * cfg->nz > ((int64_t)1 << 31) - 1)
    return fail(LBM_EINVAL, "lattice too large (padded cells must fit 32-bit offsets)");
  if (!(cfg->tau > 0.5) || !std::isfinite(cfg->tau)) return fail(LBM_EINVAL, "tau must be > 0.5");
  if (!(cfg->rho0 > 0) || !std::isfinite(cfg->G)) return fail(LBM_EINVAL, "rho0 must be > 0, G finite");
  if (cfg->kernel < LBM_KERNEL_AUTO || cfg->kernel > LBM_KERNEL_TWO_PASS)
    return fail(LBM_EINVAL, "unknown kernel");
  if ((cfg->alloc == nullptr) != (cfg->free == nullptr))
    return fail(LBM_EINVAL, "alloc and free callbacks must be given together");
  if (cfg->mass_residual != 0 && cfg->mass_residual != 1)
    return fail(LBM_EINVAL, "mass_residual must be 0 or 1");
  if (cfg->mass_residual && cfg->storage != LBM_F16_OFFSET && cfg->storage != LBM_BF16_OFFSET)
    return fail(LBM_EINVAL, "mass_residual applies to the 16-bit offset storages");

  lbm_ctx *c = new lbm_ctx();
  c->cfg = *cfg;
  c->lat = cfg->lattice == LBM_D2Q9 ? D2Q9 : D3Q19;
  c->st = cfg->storage;
  c->Q = c->lat == D3Q19 ? 19 : 9;
  c->s = static_cast<cudaStream_t>(cfg->stream);
  c->v.lat = c->lat;
  c->v.st = c->st;
  if (c->lat == D2Q9) {  // view (nx, 1, ny)
    c->v.NX = cfg->nx;
    c->v.NY = 1;
    c->v.NZ = cfg->ny;
  } else {
    c->v.NX = cfg->nx;
    c->v.NY = cfg->ny;
    c->v.NZ = cfg->nz;
  }
  c->v.px = (c->v.NX + 7) / 8 * 8;
  c->v.rho_ref = cfg->rho_ref;
  view_prepare(c->v);
  c->N = c->v.NX * c->v.NY * c->v.NZ;
  c->kernel = cfg->kernel == LBM_KERNEL_TWO_PASS ? LBM_KERNEL_TWO_PASS : LBM_KERNEL_FUSED;
  c->lat_bytes = (size_t)c->Q * c->v.px * c->v.NY * c->v.NZ * storage_bytes(c->st);
  c->resid = cfg->mass_residual == 1;
  c->st_step = !c->resid ? c->st : (c->st == ST_F16 ? ST_F16R : ST_BF16R);

  auto bail = [&](lbm_status st) {
    lbm_destroy(c);
    return st;
  };
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return fail(LBM_ECUDA, "no CUDA device");
  }
  lbm_status st;
  if ((st = dalloc(c, c->fA, c->lat_bytes)) != LBM_OK) return bail(st);
  if ((st = dalloc(c, c->fB, c->lat_bytes)) != LBM_OK) return bail(st);
  if ((st = dalloc(c, c->d_err, sizeof(int))) != LBM_OK) return bail(st);
  if (c->resid) {
    const size_t rb = sizeof(float) * (size_t)c->v.px * c->v.NY * c->v.NZ;
    if ((st = dalloc(c, c->d_resid, rb)) != LBM_OK) return bail(st);
    if (cudaMemsetAsync(c->d_resid.p, 0, rb, c->s) != cudaSuccess) {
      cudaGetLastError();
      return bail(fail(LBM_ECUDA, "memset failed"));
    }
    c->v.resid = static_cast<const float *>(c->d_resid.p);
  }
  if (cudaMemsetAsync(c->d_err.p, 0, sizeof(int), c->s) != cudaSuccess ||
      cudaMemsetAsync(c->fA.p, 0, c->lat_bytes, c->s) != cudaSuccess ||
      cudaMemsetAsync(c->fB.p, 0, c->lat_bytes, c->s) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(LBM_ECUDA, "memset failed"));
  }
  if (c->kernel == LBM_KERNEL_FUSED) {
    cudaError_t e = fused_make_plan(c->lat, c->st, cfg->tile, c->v.NX, c->v.NY, c->v.NZ, 0, &c->plan);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (cfg->kernel == LBM_KERNEL_FUSED)
        return bail(fail(LBM_EINVAL, "fused kernel: unknown tile, tile too large for this storage, "
                                     "or nx not a multiple of 16 bytes of elements"));
      c->kernel = LBM_KERNEL_TWO_PASS;  // automatic choice falls back to the two-pass path
    }
  }
  if (c->kernel == LBM_KERNEL_FUSED) {
    cudaError_t e = fused_prepare(c->lat, c->st_step, c->plan);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return bail(fail(LBM_ECUDA, std::string("fused kernel set-up: ") + cudaGetErrorString(e)));
    }
    if (fused_encode_maps(c->lat, c->st, c->plan, c->fA.p, c->v.NX, c->v.NY, c->v.NZ, c->v.px,
                          &c->tmA) != CUDA_SUCCESS ||
        fused_encode_maps(c->lat, c->st, c->plan, c->fB.p, c->v.NX, c->v.NY, c->v.NZ, c->v.px,
                          &c->tmB) != CUDA_SUCCESS)
      return bail(fail(LBM_ECUDA, "cuTensorMapEncodeTiled failed"));
  } else {
    const size_t cs = c->st == LBM_F64 ? 8 : 4;
    if ((st = dalloc(c, c->psi_scratch, (size_t)c->N * cs)) != LBM_OK) return bail(st);
  }
  *out = c;
  return LBM_OK;
}

void lbm_destroy(lbm_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->s);
  cudaGetLastError();
  DevBuf *bufs[] = {&c->fA,     &c->fB,     &c->d_resid, &c->d_sx,   &c->d_sy,   &c->d_sz,     &c->d_rate,
                    &c->d_budget, &c->d_goff, &c->d_gsite, &c->d_boff, &c->d_blist, &c->d_cells, &c->d_bub,
                    &c->psi_scratch, &c->d_err, &c->d_rho, &c->d_p, &c->d_tmp, &c->d_j, &c->d_u,
                    &c->d_labels, &c->d_ncomp, &c->d_part, &c->d_tot, &c->d_site_lab,
                    &c->d_count, &c->d_census, &c->d_film_state, &c->d_film_counts,
                    &c->d_film_rec, &c->d_film_save, &c->d_film_mids, &c->d_spread_groups,
                    &c->d_spread_sites, &c->d_spread_count, &c->d_dep};
  for (DevBuf *b : bufs) dfree(c, *b);
  hfree(c->h_err);
  hfree(c->h_site);
  hfree(c->h_mail);
  delete c;
}

lbm_status lbm_sample_sites(int64_t nx, int64_t ny, int64_t nz, int32_t n, double r_min,
                            double r_max, double min_spacing, double min_gap, uint64_t seed,
                            int64_t max_tries, lbm_bubble *out, int32_t *got) {
  if (got) *got = 0;
  if (nx < 1 || ny < 1 || nz < 1 || n < 0 || (n > 0 && !out) || max_tries < 0 ||
      !(r_max >= r_min))
    return fail(LBM_EINVAL, "bad arguments to lbm_sample_sites");
  const uint64_t key = seed ^ 0x7369746573000000ull;
  int32_t k = 0;
  for (int64_t m = 0; m < max_tries && k < n; ++m) {
    lbm_bubble b;
    b.x = std::floor(unit_at(key, 4 * (uint64_t)m + 0) * (double)nx);
    b.y = std::floor(unit_at(key, 4 * (uint64_t)m + 1) * (double)ny);
    b.z = std::floor(unit_at(key, 4 * (uint64_t)m + 2) * (double)nz);
    b.r = r_min + (r_max - r_min) * unit_at(key, 4 * (uint64_t)m + 3);
    bool ok = true;
    for (int32_t a = 0; a < k && ok; ++a) {
      const double dx = min_image(b.x - out[a].x, (double)nx);
      const double dy = min_image(b.y - out[a].y, (double)ny);
      const double dz = min_image(b.z - out[a].z, (double)nz);
      const double need = std::max(min_spacing, b.r + out[a].r + min_gap);
      if (std::sqrt(dx * dx + dy * dy + dz * dz) < need) ok = false;
    }
    if (ok) out[k++] = b;
  }
  if (got) *got = k;
  if (k < n) return fail(LBM_ESTATE, "only " + std::to_string(k) + " of " + std::to_string(n) + " sites fit");
  return LBM_OK;
}

lbm_status lbm_seed_bubbles(lbm_ctx *c, const lbm_bubble *b, int32_t n, double rho_l,
                            double rho_g, double width, double noise_amp, double min_spacing,
                            uint64_t seed) {
  if (!c) return fail(LBM_EINVAL, "ctx is NULL");
  if (n < 0) return fail(LBM_EINVAL, "bad bubble list");
  if (!(width > 0) || !std::isfinite(rho_l) || !std::isfinite(rho_g) || !std::isfinite(noise_amp))
    return fail(LBM_EINVAL, "width must be > 0, densities finite");
  std::vector<lbm_bubble> drawn;
  if (!b && n > 0) {
    // no list: draw n nuclei from the seed with the host sampler
    const double r = c->cfg.nucleus_radius;
    if (!(min_spacing >= 0) || !std::isfinite(min_spacing) || !(r >= 0) || !std::isfinite(r))
      return fail(LBM_EINVAL, "min_spacing and the nucleus radius must be finite and >= 0");
    drawn.resize(n);
    int32_t got = 0;
    CKS(lbm_sample_sites(c->cfg.nx, c->cfg.ny, c->cfg.nz, n, r, r, min_spacing, 0.0, seed,
                         10000000, drawn.data(), &got));
    b = drawn.data();
  }
  for (int32_t k = 0; k < n; ++k)
    if (!std::isfinite(b[k].x) || !std::isfinite(b[k].y) || !std::isfinite(b[k].z) ||
        !std::isfinite(b[k].r))
      return fail(LBM_EINVAL, "non-finite bubble");
  CKS(set_device(c));
  CKS(check_sticky(c));
  c->bubbles.assign(b, b + n);
  c->sx.resize(n);
  c->sy.resize(n);
  c->sz.resize(n);
  std::vector<double> vb(4 * (size_t)std::max(n, 1));
  for (int32_t k = 0; k < n; ++k) {
    double vx = b[k].x, vy = b[k].y, vz = b[k].z;
    if (c->lat == D2Q9) {  // user (x, y) -> view (x, 0, y)
      vz = b[k].y;
      vy = 0.0;
    }
    vb[4 * k + 0] = vx;
    vb[4 * k + 1] = vy;
    vb[4 * k + 2] = vz;
    vb[4 * k + 3] = b[k].r;
    c->sx[k] = (int32_t)wrap64((int64_t)std::floor(vx + 0.5), c->v.NX);
    c->sy[k] = (int32_t)wrap64((int64_t)std::floor(vy + 0.5), c->v.NY);
    c->sz[k] = (int32_t)wrap64((int64_t)std::floor(vz + 0.5), c->v.NZ);
  }
  CKS(ensure_diag(c));
  CKS(upload(c, c->d_bub, vb));
  CK(diag_init_rho(c->v, static_cast<const double *>(c->d_bub.p), n, rho_l, rho_g, width, noise_amp,
                   seed, static_cast<double *>(c->d_rho.p), c->s));
  c->cur = 0;
  CK(diag_store_from_rho(c->v, static_cast<const double *>(c->d_rho.p), lattice_ptr(c, 0), c->s));
  if (c->resid)  // a new state has no rounding residual yet
    CK(cudaMemsetAsync(c->d_resid.p, 0, c->d_resid.bytes, c->s));
  // site cells (view linear index) for label look-ups
  std::vector<int32_t> cells(n);
  for (int32_t k = 0; k < n; ++k)
    cells[k] = (int32_t)(((int64_t)c->sz[k] * c->v.NY + c->sy[k]) * c->v.NX + c->sx[k]);
  CKS(upload(c, c->d_cells, cells));
  CKS(upload(c, c->d_sx, c->sx));
  CKS(upload(c, c->d_sy, c->sy));
  CKS(upload(c, c->d_sz, c->sz));
  c->ninj = 0;
  c->steps = 0;
  c->seeded = true;
  c->have_prev = false;
  c->merge_events = 0;
  c->film_state_clear = false;
  c->p_valid = c->labels_valid = false;
  c->site_pending = false;
  c->site_labels.assign(n, -1);
  CK(cudaStreamSynchronize(c->s));  // host staging buffers go out of scope
  return LBM_OK;
}

lbm_status lbm_read_sites(const lbm_ctx *c, lbm_bubble *out, int32_t n) {
  if (!c) return fail(LBM_EINVAL, "ctx is NULL");
  if (!c->seeded) return fail(LBM_ESTATE, "seed the lattice first");
  if (n != (int32_t)c->bubbles.size() || (n > 0 && !out))
    return fail(LBM_EINVAL, "n must equal the number of seeded bubbles");
  std::copy(c->bubbles.begin(), c->bubbles.end(), out);
  return LBM_OK;
}

lbm_status lbm_inject(lbm_ctx *c, const double *rate, const double *budget, int32_t n) {
  if (!c) return fail(LBM_EINVAL, "ctx is NULL");
  if (!c->seeded) return fail(LBM_ESTATE, "seed the lattice first");
  if (n == 0) {
    c->ninj = 0;
    return LBM_OK;
  }
  if (n != (int32_t)c->sx.size() || !rate || !budget)
    return fail(LBM_EINVAL, "n must be 0 or the number of seeded bubbles");
  for (int32_t k = 0; k < n; ++k)
    if (!(rate[k] >= 0) || !(budget[k] >= 0) || !std::isfinite(rate[k]) || !std::isfinite(budget[k]))
      return fail(LBM_EINVAL, "rates and budgets must be finite and >= 0");
  CKS(set_device(c));
  CKS(check_sticky(c));
  std::vector<double> r(rate, rate + n), bgt(budget, budget + n);
  // groups of sites sharing a cell, in site order (two-pass injection kernel)
  std::map<int64_t, std::vector<int32_t>> by_cell;
  for (int32_t k = 0; k < n; ++k)
    by_cell[((int64_t)c->sz[k] * c->v.NY + c->sy[k]) * c->v.NX + c->sx[k]].push_back(k);
  std::vector<int32_t> goff(1, 0), gsite;
  for (auto &kv : by_cell) {
    gsite.insert(gsite.end(), kv.second.begin(), kv.second.end());
    goff.push_back((int32_t)gsite.size());
  }
  c->ngroups = (int32_t)by_cell.size();
  CKS(upload(c, c->d_rate, r));
  CKS(upload(c, c->d_budget, bgt));
  CKS(upload(c, c->d_goff, goff));
  CKS(upload(c, c->d_gsite, gsite));
  if (c->kernel == LBM_KERNEL_FUSED) CKS(build_buckets(c));
  CK(cudaStreamSynchronize(c->s));
  c->ninj = n;
  return LBM_OK;
}

lbm_status lbm_read_budgets(lbm_ctx *c, double *budget, int32_t n) {
  if (!c || !budget) return fail(LBM_EINVAL, "NULL argument");
  if (n != c->ninj) return fail(LBM_EINVAL, "n must equal the number of injection sites");
  if (n == 0) return LBM_OK;
  CKS(set_device(c));
  CK(cudaMemcpyAsync(budget, c->d_budget.p, sizeof(double) * n, cudaMemcpyDeviceToHost, c->s));
  return sync_and_check(c);
}

static lbm_status ensure_labels(lbm_ctx *c);

lbm_status lbm_step(lbm_ctx *c, int64_t nsteps) {
  if (!c) return fail(LBM_EINVAL, "ctx is NULL");
  if (nsteps < 0) return fail(LBM_EINVAL, "nsteps < 0");
  if (!c->seeded) return fail(LBM_ESTATE, "seed the lattice first");
  CKS(check_sticky(c));
  CKS(set_device(c));
  StepArgs a{};
  a.NX = c->v.NX;
  a.NY = c->v.NY;
  a.NZ = c->v.NZ;
  a.px = c->v.px;
  a.tau = c->cfg.tau;
  a.G = c->cfg.G;
  a.rho0 = c->cfg.rho0;
  a.rho_ref = c->cfg.rho_ref;
  a.nsites = c->ninj;
  a.site_x = static_cast<const int32_t *>(c->d_sx.p);
  a.site_y = static_cast<const int32_t *>(c->d_sy.p);
  a.site_z = static_cast<const int32_t *>(c->d_sz.p);
  a.rate = static_cast<const double *>(c->d_rate.p);
  a.budget = static_cast<double *>(c->d_budget.p);
  a.ngroups = c->ngroups;
  a.group_off = static_cast<const int32_t *>(c->d_goff.p);
  a.group_site = static_cast<const int32_t *>(c->d_gsite.p);
  a.bucket_off = static_cast<const int32_t *>(c->d_boff.p);
  a.bucket_site = static_cast<const int32_t *>(c->d_blist.p);
  a.err = static_cast<int *>(c->d_err.p);
  a.debug_flags = c->cfg.debug_flags;
  a.resid = static_cast<float *>(c->d_resid.p);
  a.tau_f = (float)c->cfg.tau;
  a.omega_f = (float)(1.0 / c->cfg.tau);
  a.G_f = (float)c->cfg.G;
  a.rho0_f = (float)c->cfg.rho0;
  a.inv_rho0_f = (float)(1.0 / c->cfg.rho0);
  a.rho_ref_f = (float)c->cfg.rho_ref;
  const size_t pop_bytes = (size_t)c->v.px * c->v.NY * c->v.NZ * storage_bytes(c->st);
  // spread mode: the bubbles of the sites are those of the state at the
  // start of this call (one synchronisation to read the site labels)
  const bool spread = c->inj_mode == 1 && c->ninj > 0 && nsteps > 0;
  int ngroups = 0;
  bool any_bubble = false;
  if (spread) {
    a.nsites = 0;  // the step kernels deposit nothing
    CKS(ensure_labels(c));
    CKS(dalloc(c, c->d_spread_count, sizeof(int32_t) * c->N));
    CK(inject_component_sizes(c->v, static_cast<const int32_t *>(c->d_labels.p),
                              static_cast<int32_t *>(c->d_spread_count.p), c->s));
    CKS(sync_and_check(c));  // site labels on the host
    // groups: one per bubble holding sites, one per liquid site cell; sites
    // in increasing order within a group
    std::map<int64_t, std::vector<int32_t>> by;
    for (int32_t q = 0; q < c->ninj; ++q) {
      const int32_t lab = c->site_labels[q];
      const int64_t cell = (int64_t)c->sx[q] + c->v.NX * ((int64_t)c->sy[q] + c->v.NY * c->sz[q]);
      by[lab >= 0 ? (int64_t)lab : -1 - cell].push_back(q);
    }
    std::vector<int4> groups;
    std::vector<int32_t> gsites;
    for (auto &kv : by) {
      const int first = (int)gsites.size();
      gsites.insert(gsites.end(), kv.second.begin(), kv.second.end());
      const bool bubble = kv.first >= 0;
      any_bubble |= bubble;
      groups.push_back(make_int4(bubble ? (int)kv.first : -1, first, (int)gsites.size(),
                                 bubble ? 0 : (int)(-1 - kv.first)));
    }
    ngroups = (int)groups.size();
    CKS(upload(c, c->d_spread_groups, groups));
    CKS(upload(c, c->d_spread_sites, gsites));
    CKS(dalloc(c, c->d_dep, sizeof(double) * c->N));
    CK(cudaMemsetAsync(c->d_dep.p, 0, sizeof(double) * c->N, c->s));
    CK(cudaStreamSynchronize(c->s));  // the host vectors go out of scope
  }
  const int32_t *spread_labels = static_cast<const int32_t *>(c->d_labels.p);
  for (int64_t t = 0; t < nsteps; ++t) {
    a.fin = lattice_ptr(c, c->cur);
    a.fout = lattice_ptr(c, 1 - c->cur);
    for (int i = 0; i < c->Q; ++i) a.out_pop[i] = static_cast<char *>(a.fout) + i * pop_bytes;
    cudaError_t e;
    if (c->kernel == LBM_KERNEL_FUSED)
      e = fused_launch(c->lat, c->st_step, c->plan, a, c->cur == 0 ? c->tmA : c->tmB, c->s);
    else
      e = twopass_launch(c->lat, c->st_step, a, c->psi_scratch.p, c->s);
    if (e == cudaSuccess && spread)
      e = inject_spread(c->v, ngroups, static_cast<const int4 *>(c->d_spread_groups.p),
                        static_cast<const int32_t *>(c->d_spread_sites.p),
                        static_cast<const double *>(c->d_rate.p),
                        static_cast<double *>(c->d_budget.p),
                        static_cast<const int32_t *>(c->d_spread_count.p),
                        static_cast<double *>(c->d_dep.p), spread_labels, any_bubble, a.fout,
                        c->s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      c->sticky = LBM_ECUDA;
      return fail(LBM_ECUDA, std::string("step launch: ") + cudaGetErrorString(e));
    }
    c->cur = 1 - c->cur;
    ++c->steps;
    c->p_valid = c->labels_valid = false;
  }
  return LBM_OK;
}

int64_t lbm_step_count(const lbm_ctx *c) { return c ? c->steps : -1; }

lbm_status lbm_set_injection_mode(lbm_ctx *c, int32_t mode) {
  if (!c) return fail(LBM_EINVAL, "ctx is NULL");
  if (mode != 0 && mode != 1) return fail(LBM_EINVAL, "mode must be 0 (site cell) or 1 (bubble)");
  if (mode == 1 && c->st != LBM_F64 && c->st != LBM_F32)
    return fail(LBM_EINVAL, "spread injection needs FP64 or FP32 storage");
  c->inj_mode = mode;
  return LBM_OK;
}

lbm_status lbm_plan_info(const lbm_ctx *c, int32_t out[6]) {
  if (!c || !out) return fail(LBM_EINVAL, "NULL argument");
  const bool fused = c->kernel == LBM_KERNEL_FUSED;
  out[0] = c->kernel;
  out[1] = fused ? c->plan.tile : 0;
  out[2] = fused ? c->plan.bx : 0;
  out[3] = fused ? c->plan.by : 0;
  out[4] = fused ? c->plan.nzc : 0;
  out[5] = fused ? c->plan.items : 0;
  return LBM_OK;
}

// switch the fused kernel to another plan: smem attribute, descriptors and
// the per-CTA injection buckets
static lbm_status use_plan(lbm_ctx *c, const FusedPlan &p) {
  CK(fused_prepare(c->lat, c->st_step, p));
  FusedMaps ma, mb;
  if (fused_encode_maps(c->lat, c->st, p, c->fA.p, c->v.NX, c->v.NY, c->v.NZ, c->v.px, &ma) !=
          CUDA_SUCCESS ||
      fused_encode_maps(c->lat, c->st, p, c->fB.p, c->v.NX, c->v.NY, c->v.NZ, c->v.px, &mb) !=
          CUDA_SUCCESS)
    return fail(LBM_ECUDA, "cuTensorMapEncodeTiled failed");
  c->plan = p;
  c->tmA = ma;
  c->tmB = mb;
  if (c->ninj > 0) CKS(build_buckets(c));
  return LBM_OK;
}

lbm_status lbm_autotune(lbm_ctx *c, int32_t steps, int32_t *best_tile, double *best_ms) {
  if (!c) return fail(LBM_EINVAL, "ctx is NULL");
  if (steps < 1) return fail(LBM_EINVAL, "steps must be >= 1");
  if (c->kernel != LBM_KERNEL_FUSED) return fail(LBM_EINVAL, "autotuning applies to the fused kernel");
  if (!c->seeded) return fail(LBM_ESTATE, "seed the lattice first");
  CKS(set_device(c));
  CKS(check_sticky(c));
  // save the state: current lattice (and rounding residual), budgets, step
  // counter
  DevBuf save_f, save_b;
  lbm_status st = dalloc(c, save_f, c->lat_bytes + c->d_resid.bytes);
  if (st != LBM_OK) return st;
  const size_t bbytes = sizeof(double) * (size_t)std::max(c->ninj, 1);
  if ((st = dalloc(c, save_b, bbytes)) != LBM_OK) {
    dfree(c, save_f);
    return st;
  }
  const int cur0 = c->cur;
  const int64_t steps0 = c->steps;
  auto restore = [&]() -> lbm_status {
    CK(cudaMemcpyAsync(lattice_ptr(c, cur0), save_f.p, c->lat_bytes, cudaMemcpyDeviceToDevice, c->s));
    if (c->resid)
      CK(cudaMemcpyAsync(c->d_resid.p, static_cast<char *>(save_f.p) + c->lat_bytes,
                         c->d_resid.bytes, cudaMemcpyDeviceToDevice, c->s));
    if (c->ninj > 0)
      CK(cudaMemcpyAsync(c->d_budget.p, save_b.p, sizeof(double) * c->ninj,
                         cudaMemcpyDeviceToDevice, c->s));
    c->cur = cur0;
    c->steps = steps0;
    c->p_valid = c->labels_valid = false;
    return LBM_OK;
  };
  auto body = [&]() -> lbm_status {
    CK(cudaMemcpyAsync(save_f.p, lattice_ptr(c, cur0), c->lat_bytes, cudaMemcpyDeviceToDevice, c->s));
    if (c->resid)
      CK(cudaMemcpyAsync(static_cast<char *>(save_f.p) + c->lat_bytes, c->d_resid.p,
                         c->d_resid.bytes, cudaMemcpyDeviceToDevice, c->s));
    if (c->ninj > 0)
      CK(cudaMemcpyAsync(save_b.p, c->d_budget.p, sizeof(double) * c->ninj,
                         cudaMemcpyDeviceToDevice, c->s));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    FusedPlan best{};
    float best_t = 1e30f;
    for (int cand = 0; cand < 64 * 4; ++cand) {
      // every tile, with the modelled number of z chunks, half and double
      // it, and the number that fills the resident slots once
      const int tile = 1 + cand / 4, variant = cand % 4;
      int bx, by, ns;
      if (!fused_tile_shape(c->lat, c->st, tile, &bx, &by, &ns)) continue;
      FusedPlan p, p1;
      if (fused_make_plan(c->lat, c->st, tile, c->v.NX, c->v.NY, c->v.NZ, 0, &p) != cudaSuccess ||
          fused_make_plan(c->lat, c->st, tile, c->v.NX, c->v.NY, c->v.NZ, -1, &p1) !=
              cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      if (variant > 0) {
        const int nzc = variant == 1 ? std::max(1, p.nzc / 2)
                        : variant == 2 ? p.nzc * 2
                                       : p1.nzc;
        if (nzc > c->v.NZ) continue;
        FusedPlan q;
        if (fused_make_plan(c->lat, c->st, tile, c->v.NX, c->v.NY, c->v.NZ, nzc, &q) != cudaSuccess) {
          cudaGetLastError();
          continue;
        }
        // skip chunkings an earlier variant of this tile already timed
        const int n1 = std::max(1, p.nzc / 2), n2 = p.nzc * 2;
        if (q.nzc == p.nzc || (variant >= 2 && q.nzc == n1) || (variant == 3 && q.nzc == n2))
          continue;
        p = q;
      }
      CKS(use_plan(c, p));
      CKS(lbm_step(c, 2));
      // best of two timed rounds (launch-order and clock noise)
      float ms = 1e30f;
      for (int round = 0; round < 2; ++round) {
        CK(cudaEventRecord(e0, c->s));
        CKS(lbm_step(c, steps));
        CK(cudaEventRecord(e1, c->s));
        CK(cudaEventSynchronize(e1));
        float t = 0;
        CK(cudaEventElapsedTime(&t, e0, e1));
        ms = std::min(ms, t / steps);
      }
      CKS(restore());
      if (ms < best_t) {
        best_t = ms;
        best = p;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best.tile == 0) return fail(LBM_ECUDA, "no tile could be timed");
    CKS(use_plan(c, best));
    if (best_tile) *best_tile = best.tile;
    if (best_ms) *best_ms = best_t;
    return LBM_OK;
  };
  st = body();
  if (st != LBM_OK) restore();
  cudaError_t e = cudaStreamSynchronize(c->s);
  dfree(c, save_f);
  dfree(c, save_b);
  if (st == LBM_OK && e != cudaSuccess) return fail(LBM_ECUDA, cudaGetErrorString(e));
  if (st == LBM_OK) st = sync_and_check(c);
  return st;
}

lbm_status lbm_sync(lbm_ctx *c) {
  if (!c) return fail(LBM_EINVAL, "ctx is NULL");
  CKS(set_device(c));
  return sync_and_check(c);
}

static lbm_status compute_pressure(lbm_ctx *c) {
  if (c->p_valid) return LBM_OK;
  CKS(ensure_diag(c));
  CK(diag_moments(c->v, lattice_ptr(c, c->cur), c->cfg.G, c->cfg.rho0,
                  static_cast<double *>(c->d_rho.p), nullptr, nullptr, nullptr, nullptr,
                  static_cast<double *>(c->d_p.p), static_cast<int *>(c->d_err.p), c->s));
  c->p_valid = true;
  return LBM_OK;
}

lbm_status lbm_pressure_laplacian(lbm_ctx *c, double *out, int64_t count, const int64_t *line) {
  if (!c || !out) return fail(LBM_EINVAL, "NULL argument");
  if (!c->seeded) return fail(LBM_ESTATE, "seed the lattice first");
  CKS(set_device(c));
  CKS(check_sticky(c));
  if (!line) {
    if (count != c->N) return fail(LBM_EINVAL, "count must be N for the full Laplacian");
  } else {
    if (line[3] < 0 || line[3] > 2 || line[4] < 0 || count != line[4])
      return fail(LBM_EINVAL, "line = {x, y, z, axis (0..2), len}, count = len");
    if (c->lat == D2Q9 && (line[3] == 2 || line[2] != 0))
      return fail(LBM_EINVAL, "2-D lattice: axis must be 0 or 1 and z 0");
  }
  CKS(compute_pressure(c));
  double *tmp = static_cast<double *>(c->d_tmp.p);
  if (!line) {
    CK(diag_laplacian(c->v, static_cast<const double *>(c->d_p.p), tmp, c->s));
  } else {
    int64_t x0 = line[0], y0 = line[1], z0 = line[2];
    int axis = (int)line[3];
    if (c->lat == D2Q9) {  // user (x, y) -> view (x, 0, y)
      z0 = y0;
      y0 = 0;
      axis = axis == 1 ? 2 : 0;
    }
    if (line[4] > 0)
      CK(diag_line_d2(c->v, static_cast<const double *>(c->d_p.p), wrap64(x0, c->v.NX),
                      wrap64(y0, c->v.NY), wrap64(z0, c->v.NZ), axis, line[4], tmp, c->s));
  }
  if (count > 0)
    CK(cudaMemcpyAsync(out, tmp, sizeof(double) * count, cudaMemcpyDeviceToHost, c->s));
  return sync_and_check(c);
}

// Enqueue the labelling of gas cells (and, for FP32-arithmetic storages, the
// totals in the same pass when want_totals), then the per-site label gather.
static lbm_status enqueue_labels(lbm_ctx *c, bool want_totals) {
  CKS(ensure_diag(c));
  CKS(dalloc(c, c->d_labels, sizeof(int32_t) * c->N));
  int32_t *lab = static_cast<int32_t *>(c->d_labels.p);
  if (c->st != LBM_F64) {
    CK(diag_scan(c->v, lattice_ptr(c, c->cur), c->cfg.gas_threshold, lab,
                 want_totals ? static_cast<double *>(c->d_part.p) : nullptr,
                 want_totals ? static_cast<double *>(c->d_tot.p) : nullptr,
                 static_cast<int *>(c->d_err.p), c->s));
    CK(diag_label_links(c->v, lab, static_cast<unsigned long long *>(c->d_ncomp.p), c->s));
  } else {
    CKS(compute_pressure(c));
    CK(diag_label(c->v, static_cast<const double *>(c->d_rho.p), c->cfg.gas_threshold, lab,
                  static_cast<unsigned long long *>(c->d_ncomp.p), c->s));
    if (want_totals)
      CK(diag_totals(c->v, lattice_ptr(c, c->cur), static_cast<double *>(c->d_part.p),
                     static_cast<double *>(c->d_tot.p), c->s));
  }
  const int32_t ns = (int32_t)c->sx.size();
  if (ns > 0) {
    CKS(dalloc(c, c->d_site_lab, sizeof(int32_t) * ns));
    CK(diag_gather_labels(lab, static_cast<const int32_t *>(c->d_cells.p), ns,
                          static_cast<int32_t *>(c->d_site_lab.p), c->s));
    CKS(halloc(c, c->h_site, sizeof(int32_t) * ns));
    CK(cudaMemcpyAsync(c->h_site.p, c->d_site_lab.p, sizeof(int32_t) * ns,
                       cudaMemcpyDeviceToHost, c->s));
    c->site_pending = true;  // copied to site_labels at the next synchronisation
  }
  c->labels_valid = true;
  return LBM_OK;
}

// labels of the current state, computed at most once per state
static lbm_status ensure_labels(lbm_ctx *c) {
  return c->labels_valid ? LBM_OK : enqueue_labels(c, false);
}

// merge events: pairs of sites with different labels before, equal now
static void count_merges(lbm_ctx *c) {
  const int32_t ns = (int32_t)c->sx.size();
  if (ns == 0) return;
  if (c->have_prev) {
    std::map<int32_t, std::map<int32_t, int64_t>> groups;  // now -> prev -> count
    for (int32_t k = 0; k < ns; ++k)
      if (c->site_labels[k] >= 0) groups[c->site_labels[k]][c->prev_site_labels[k]]++;
    for (auto &g : groups) {
      int64_t tot = 0, same = 0;
      for (auto &p : g.second) {
        tot += p.second;
        same += p.second * (p.second - 1) / 2;
      }
      c->merge_events += tot * (tot - 1) / 2 - same;
    }
  }
  c->prev_site_labels = c->site_labels;
  c->have_prev = true;
}

lbm_status lbm_film_probe(lbm_ctx *c, const int64_t *line, double rho_mid, lbm_film *out) {
  if (!c || !line || !out) return fail(LBM_EINVAL, "NULL argument");
  if (!c->seeded) return fail(LBM_ESTATE, "seed the lattice first");
  const int dims = c->lat == D2Q9 ? 2 : 3;
  if (line[3] < 0 || line[3] >= dims || line[4] < 2)
    return fail(LBM_EINVAL, "line = {x, y, z, axis (< dims), len >= 2}");
  CKS(set_device(c));
  CKS(check_sticky(c));
  CKS(compute_pressure(c));
  // user axes -> view axes (D2Q9: x -> x, y -> z)
  auto vaxis = [&](int a) { return c->lat == D2Q9 ? (a == 0 ? 0 : 2) : a; };
  int e[3] = {0, 0, 0}, ep[3] = {0, 0, 0};
  e[vaxis((int)line[3])] = 1;
  ep[vaxis(((int)line[3] + 1) % dims)] = 1;
  int64_t x0 = line[0], y0 = line[1], z0 = line[2];
  if (c->lat == D2Q9) {
    z0 = y0;
    y0 = 0;
  }
  double *tmp = static_cast<double *>(c->d_tmp.p);
  CK(diag_film_probe(c->v, static_cast<const double *>(c->d_rho.p),
                     static_cast<const double *>(c->d_p.p), wrap64(x0, c->v.NX), wrap64(y0, c->v.NY),
                     wrap64(z0, c->v.NZ), e, ep, line[4], rho_mid, tmp, c->s));
  CKS(halloc(c, c->h_mail, 6 * sizeof(double)));
  const double *h = static_cast<const double *>(c->h_mail.p);
  CK(cudaMemcpyAsync(c->h_mail.p, tmp, 6 * sizeof(double), cudaMemcpyDeviceToHost, c->s));
  CKS(sync_and_check(c));
  out->found = h[0] != 0.0;
  out->x1 = h[1];
  out->x2 = h[2];
  out->h = h[3];
  out->d2p_mid = h[4];
  out->r_d = h[5];
  return LBM_OK;
}

lbm_status lbm_run_until_rupture(lbm_ctx *c, const int64_t *line, double rho_mid,
                                  double eps_arm, double h_max, int64_t diag_every,
                                  int64_t max_steps, lbm_rupture *out) {
  if (!c || !line || !out) return fail(LBM_EINVAL, "NULL argument");
  if (diag_every < 1 || max_steps < 0 || !(eps_arm >= 0) || !(h_max > 0))
    return fail(LBM_EINVAL, "diag_every >= 1, max_steps >= 0, eps_arm >= 0, h_max > 0");
  std::memset(out, 0, sizeof(*out));
  bool armed = false;
  double h_prev = 0.0, d_prev = 0.0;  // previous probe (d_prev < 0 whenever armed)
  int64_t t = 0;
  while (t < max_steps) {
    const int64_t n = std::min(diag_every, max_steps - t);
    CKS(lbm_step(c, n));
    t += n;
    lbm_film pr;
    CKS(lbm_film_probe(c, line, rho_mid, &pr));
    out->steps = t;
    if (!pr.found) {  // the film is gone: merged before the criterion fired
      out->merged = 1;
      return LBM_OK;
    }
    if (pr.h > h_max) {
      armed = false;  // thick film: the criterion does not apply
    } else if (pr.d2p_mid < -eps_arm) {
      armed = true;
    } else if (armed && pr.d2p_mid >= 0.0) {
      out->fired = 1;
      out->h_c = h_prev + (pr.h - h_prev) * (-d_prev / (pr.d2p_mid - d_prev));
      out->h_probe = pr.h;
      out->r_d = pr.r_d;
      return LBM_OK;
    }
    h_prev = pr.h;
    d_prev = pr.d2p_mid;
  }
  return LBM_OK;
}

lbm_status lbm_label_gas(lbm_ctx *c, int32_t *labels, int64_t *ncomp) {
  if (!c) return fail(LBM_EINVAL, "ctx is NULL");
  if (!c->seeded) return fail(LBM_ESTATE, "seed the lattice first");
  CKS(set_device(c));
  CKS(check_sticky(c));
  CKS(enqueue_labels(c, false));
  CKS(halloc(c, c->h_mail, sizeof(unsigned long long)));
  const auto *nc = static_cast<const unsigned long long *>(c->h_mail.p);
  CK(cudaMemcpyAsync(c->h_mail.p, c->d_ncomp.p, sizeof(*nc), cudaMemcpyDeviceToHost, c->s));
  if (labels)
    CK(cudaMemcpyAsync(labels, c->d_labels.p, sizeof(int32_t) * c->N, cudaMemcpyDeviceToHost, c->s));
  CKS(sync_and_check(c));
  if (ncomp) *ncomp = (int64_t)*nc;
  count_merges(c);
  return LBM_OK;
}

lbm_status lbm_diagnose(lbm_ctx *c, double totals[4], int32_t *labels, int64_t *ncomp) {
  if (!c) return fail(LBM_EINVAL, "ctx is NULL");
  if (!c->seeded) return fail(LBM_ESTATE, "seed the lattice first");
  CKS(set_device(c));
  CKS(check_sticky(c));
  CKS(enqueue_labels(c, totals != nullptr));
  // mailbox: [ncomp][totals: 4 doubles]
  CKS(halloc(c, c->h_mail, 5 * sizeof(double)));
  auto *mail = static_cast<unsigned char *>(c->h_mail.p);
  CK(cudaMemcpyAsync(mail, c->d_ncomp.p, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->s));
  if (totals)
    CK(cudaMemcpyAsync(mail + 8, c->d_tot.p, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->s));
  if (labels)
    CK(cudaMemcpyAsync(labels, c->d_labels.p, sizeof(int32_t) * c->N, cudaMemcpyDeviceToHost, c->s));
  CKS(sync_and_check(c));
  if (totals) std::memcpy(totals, mail + 8, 4 * sizeof(double));
  if (ncomp) *ncomp = (int64_t)*reinterpret_cast<const unsigned long long *>(mail);
  count_merges(c);
  return LBM_OK;
}

lbm_status lbm_bubble_sizes(lbm_ctx *c, int64_t *roots, int64_t *sizes, int64_t cap,
                            int64_t *ncomp, int64_t *hist, int32_t nbins) {
  if (!c) return fail(LBM_EINVAL, "ctx is NULL");
  if (cap < 0 || nbins < 0 || nbins > 63 || (hist && nbins < 1))
    return fail(LBM_EINVAL, "cap >= 0 and 1 <= nbins <= 63 when hist is given");
  if (!c->seeded) return fail(LBM_ESTATE, "seed the lattice first");
  CKS(set_device(c));
  CKS(check_sticky(c));
  CKS(ensure_labels(c));
  const int nb = std::max(nbins, 1);
  CKS(dalloc(c, c->d_count, sizeof(int32_t) * c->N));
  // One synchronisation in the common case: the list is written up to the
  // device capacity, which grows (and the list is redone) when a lattice has
  // more components than ever before.
  const unsigned long long *mail = nullptr;
  const int64_t *r = nullptr, *sz = nullptr;
  int64_t n = 0;
  for (int pass = 0; pass < 2; ++pass) {
    const int64_t capdev = c->census_cap;
    // device block and mailbox: [n_dev][hist: 64][roots: capdev][sizes: capdev];
    // the mailbox has the labelling's component count after it
    const size_t block = sizeof(int64_t) * (65 + 2 * (size_t)capdev);
    CKS(dalloc(c, c->d_census, block));
    CKS(halloc(c, c->h_mail, block + sizeof(unsigned long long)));
    auto *base = static_cast<unsigned long long *>(c->d_census.p);
    int64_t *d_roots = reinterpret_cast<int64_t *>(base + 65), *d_sizes = d_roots + capdev;
    CK(diag_bubble_sizes(c->v, static_cast<const int32_t *>(c->d_labels.p),
                         static_cast<int32_t *>(c->d_count.p), base, capdev, d_roots, d_sizes,
                         nb, base + 1, c->s));
    mail = static_cast<const unsigned long long *>(c->h_mail.p);
    CK(cudaMemcpyAsync(c->h_mail.p, base, block, cudaMemcpyDeviceToHost, c->s));
    CK(cudaMemcpyAsync(static_cast<unsigned char *>(c->h_mail.p) + block, c->d_ncomp.p,
                       sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->s));
    CKS(sync_and_check(c));
    n = (int64_t)mail[block / sizeof(unsigned long long)];
    r = reinterpret_cast<const int64_t *>(mail + 65);
    sz = r + capdev;
    if (n <= capdev) break;
    c->census_cap = n;  // more components than the list holds: grow, redo
  }
  count_merges(c);
  if ((int64_t)mail[0] != n) return fail(LBM_ECUDA, "bubble census: component count mismatch");
  if (n > c->census_cap) return fail(LBM_ECUDA, "bubble census: list overflow after regrowth");
  // canonical order: increasing root label
  std::vector<int64_t> order((size_t)n);
  for (int64_t q = 0; q < n; ++q) order[q] = q;
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return r[a] < r[b]; });
  for (int64_t q = 0; q < std::min(n, cap); ++q) {
    if (roots) roots[q] = r[order[q]];
    if (sizes) sizes[q] = sz[order[q]];
  }
  if (ncomp) *ncomp = n;
  if (hist)
    for (int b = 0; b < nbins; ++b) hist[b] = (int64_t)mail[1 + b];
  return LBM_OK;
}

// shared set-up of the film test: labels, arming state, counters
static lbm_status film_prepare(lbm_ctx *c, int32_t h_max, double eps_arm) {
  if (h_max < 1 || h_max > 1024 || !(eps_arm >= 0))
    return fail(LBM_EINVAL, "1 <= h_max <= 1024, eps_arm >= 0");
  if (!c->seeded) return fail(LBM_ESTATE, "seed the lattice first");
  CKS(set_device(c));
  CKS(check_sticky(c));
  CKS(ensure_labels(c));
  CKS(ensure_diag(c));
  // whole 32-bit words: the midpoint pass sets bits with word atomics
  const size_t state_bytes = ((size_t)c->N + 3) & ~(size_t)3;
  CKS(dalloc(c, c->d_film_state, state_bytes));
  if (!c->film_state_clear) {
    CK(cudaMemsetAsync(c->d_film_state.p, 0, state_bytes, c->s));
    c->film_state_clear = true;
  }
  CKS(dalloc(c, c->d_film_counts, FILM_COUNT_SLOTS * sizeof(unsigned long long)));
  // queue of the line walks' midpoints: up to 2^20 (one per cell and axis at
  // most); midpoints beyond it are taken inside the walks
  c->film_mid_queue = (c->cfg.debug_flags & 4)  // LBM_DEBUG_SMALL_FILM_QUEUE
                           ? 16
                           : std::min<int64_t>(int64_t(1) << 20, c->N * (c->lat == D2Q9 ? 2 : 3));
  CKS(dalloc(c, c->d_film_mids, sizeof(FilmMid) * (size_t)c->film_mid_queue));
  return LBM_OK;
}

lbm_status lbm_film_cells(lbm_ctx *c, int32_t h_max, double eps_arm, lbm_film_census *out,
                          lbm_film_cell *fired, int64_t cap) {
  if (!c || !out) return fail(LBM_EINVAL, "NULL argument");
  if (cap < 0) return fail(LBM_EINVAL, "cap >= 0");
  CKS(film_prepare(c, h_max, eps_arm));
  CKS(dalloc(c, c->d_film_rec, film_record_bytes() * (size_t)std::max<int64_t>(cap, 1)));
  CK(diag_film_cells(c->v, static_cast<const int32_t *>(c->d_labels.p), lattice_ptr(c, c->cur),
                     c->cfg.G, c->cfg.rho0, h_max, eps_arm,
                     static_cast<uint8_t *>(c->d_film_state.p),
                     static_cast<unsigned long long *>(c->d_film_counts.p), cap, c->d_film_rec.p,
                     false, static_cast<FilmMid *>(c->d_film_mids.p), c->film_mid_queue, c->s));
  // mailbox: [counts: 4][up to cap records], one synchronisation
  const size_t rec_bytes = fired ? sizeof(lbm_film_cell) * (size_t)cap : 0;
  CKS(halloc(c, c->h_mail, 4 * sizeof(unsigned long long) + rec_bytes));
  auto *mail = static_cast<unsigned char *>(c->h_mail.p);
  CK(cudaMemcpyAsync(mail, c->d_film_counts.p, 4 * sizeof(unsigned long long),
                     cudaMemcpyDeviceToHost, c->s));
  if (rec_bytes)
    CK(cudaMemcpyAsync(mail + 32, c->d_film_rec.p, rec_bytes, cudaMemcpyDeviceToHost, c->s));
  CKS(sync_and_check(c));
  count_merges(c);
  const auto *cnt = reinterpret_cast<const unsigned long long *>(mail);
  out->film = (int64_t)cnt[0];
  out->midpoints = (int64_t)cnt[1];
  out->armed = (int64_t)cnt[2];
  out->fired = (int64_t)cnt[3];
  const int64_t nrec = std::min<int64_t>(out->fired, cap);
  if (fired && nrec > 0) {
    std::memcpy(fired, mail + 32, sizeof(lbm_film_cell) * (size_t)nrec);
    std::sort(fired, fired + nrec, [](const lbm_film_cell &a, const lbm_film_cell &b) {
      return a.cell != b.cell ? a.cell < b.cell : a.axis < b.axis;
    });
  }
  return LBM_OK;
}

lbm_status lbm_film_pairs(lbm_ctx *c, int32_t h_max, double eps_arm, lbm_film_census *census,
                          lbm_film_pair *pairs, int64_t cap, int64_t *npairs) {
  if (!c || !census) return fail(LBM_EINVAL, "NULL argument");
  if (cap < 0 || (cap > 0 && !pairs)) return fail(LBM_EINVAL, "cap >= 0, pairs given when cap > 0");
  CKS(film_prepare(c, h_max, eps_arm));
  // every midpoint is recorded; when they outnumber the record buffer the
  // arming state is put back and the pass redone with a larger buffer, so
  // that one call advances the state once
  CKS(dalloc(c, c->d_film_save, (size_t)c->N));
  CK(cudaMemcpyAsync(c->d_film_save.p, c->d_film_state.p, (size_t)c->N,
                     cudaMemcpyDeviceToDevice, c->s));
  const auto *mail = static_cast<const unsigned long long *>(nullptr);
  int64_t nmid = 0, capdev = 0;
  for (int pass = 0; pass < 2; ++pass) {
    capdev = c->film_mid_cap;
    const size_t rec_bytes = film_record_bytes() * (size_t)capdev;
    CKS(dalloc(c, c->d_film_rec, rec_bytes));
    CK(diag_film_cells(c->v, static_cast<const int32_t *>(c->d_labels.p), lattice_ptr(c, c->cur),
                       c->cfg.G, c->cfg.rho0, h_max, eps_arm,
                       static_cast<uint8_t *>(c->d_film_state.p),
                       static_cast<unsigned long long *>(c->d_film_counts.p), capdev,
                       c->d_film_rec.p, true,
                       static_cast<FilmMid *>(c->d_film_mids.p), c->film_mid_queue, c->s));
    // mailbox: [counts: 5, one padding word][records]
    CKS(halloc(c, c->h_mail, 6 * sizeof(unsigned long long) + rec_bytes));
    auto *m = static_cast<unsigned char *>(c->h_mail.p);
    CK(cudaMemcpyAsync(m, c->d_film_counts.p, 5 * sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, c->s));
    CK(cudaMemcpyAsync(m + 48, c->d_film_rec.p, rec_bytes, cudaMemcpyDeviceToHost, c->s));
    CKS(sync_and_check(c));
    mail = reinterpret_cast<const unsigned long long *>(m);
    nmid = (int64_t)mail[4];
    if (nmid <= capdev) break;
    c->film_mid_cap = nmid + nmid / 4;  // grow, restore the state, redo
    CK(cudaMemcpyAsync(c->d_film_state.p, c->d_film_save.p, (size_t)c->N,
                       cudaMemcpyDeviceToDevice, c->s));
  }
  // the redo sees the same state, so its midpoints fit; a count that still
  // exceeds the records read back is an error, never an over-read
  if (nmid > capdev) return fail(LBM_ECUDA, "film pairs: midpoint records overflow after regrowth");
  census->film = (int64_t)mail[0];
  census->midpoints = (int64_t)mail[1];
  census->armed = (int64_t)mail[2];
  census->fired = (int64_t)mail[3];
  // per pair and axis: lines holding a midpoint, midpoints, thinnest run;
  // per pair: fired midpoints and their summed thickness
  const auto *rec = reinterpret_cast<const lbm_film_cell *>(reinterpret_cast<const unsigned char *>(mail) + 48);
  const int dims = c->lat == D2Q9 ? 2 : 3;
  const int64_t nx = c->cfg.nx, ny = c->cfg.ny;
  struct Acc {
    std::vector<int64_t> lines[3];
    int64_t mid[3] = {0, 0, 0};
    int32_t hmin[3] = {INT32_MAX, INT32_MAX, INT32_MAX};
    int64_t fired = 0;
    double tsum = 0.0;
  };
  std::map<std::pair<int32_t, int32_t>, Acc> acc;
  for (int64_t q = 0; q < nmid; ++q) {
    const lbm_film_cell &r = rec[q];
    const int a = r.axis & 0xff;
    const bool fired = (r.axis >> 8) & 1;
    Acc &g = acc[{std::min(r.label_minus, r.label_plus), std::max(r.label_minus, r.label_plus)}];
    // the lattice line through the cell along axis a, as the cell's index
    // with its a-coordinate removed (user coordinates x + nx (y + ny z))
    const int64_t x = r.cell % nx, yz = r.cell / nx, y = yz % ny, z = yz / ny;
    const int64_t line = a == 0 ? yz : (a == 1 ? x + nx * z : x + nx * y);
    g.lines[a].push_back(line);
    g.mid[a] += 1;
    g.hmin[a] = std::min(g.hmin[a], r.thickness);
    if (fired) {
      g.fired += 1;
      g.tsum += r.thickness;
    }
  }
  int64_t n = 0;
  for (auto &kv : acc) {
    Acc &g = kv.second;
    int best = 0;
    int64_t best_lines = -1;
    for (int a = 0; a < dims; ++a) {
      std::sort(g.lines[a].begin(), g.lines[a].end());
      const int64_t nl = std::unique(g.lines[a].begin(), g.lines[a].end()) - g.lines[a].begin();
      if (nl > best_lines) {  // the lower axis on a tie
        best_lines = nl;
        best = a;
      }
    }
    if (n < cap) {
      lbm_film_pair &o = pairs[n];
      o.label_a = kv.first.first;
      o.label_b = kv.first.second;
      o.axis = best;
      o.h_min = g.hmin[best];
      o.lines = best_lines;
      o.midpoints = g.mid[best];
      o.fired = g.fired;
      constexpr double kPi = 3.14159265358979323846;
      o.r_d = dims == 3 ? std::sqrt((double)best_lines / kPi) : 0.5 * (double)best_lines;
      o.h_c = g.fired ? g.tsum / (double)g.fired : 0.0;
    }
    ++n;
  }
  if (npairs) *npairs = n;
  return LBM_OK;
}

lbm_status lbm_diagnostic_interval(lbm_ctx *c, int32_t h_max, double eps_arm, int32_t *labels,
                                   lbm_film_cell *fired, int64_t fired_cap, int64_t *roots,
                                   int64_t *sizes, int64_t sizes_cap, int64_t *hist,
                                   int32_t nbins, lbm_interval_report *out) {
  if (!c || !out) return fail(LBM_EINVAL, "NULL argument");
  if (fired_cap < 0 || sizes_cap < 0 || nbins < 0 || nbins > 63 || (hist && nbins < 1))
    return fail(LBM_EINVAL, "caps >= 0 and 1 <= nbins <= 63 when hist is given");
  if (!c->seeded) return fail(LBM_ESTATE, "seed the lattice first");
  CKS(set_device(c));
  CKS(check_sticky(c));
  const int nb = std::max(nbins, 1);
  // everything of the interval on the stream: FP64 totals and labels (one
  // pass), site labels, the film test, the census
  CKS(enqueue_labels(c, true));
  CKS(film_prepare(c, h_max, eps_arm));  // arming state and counters (labels are current)
  CKS(dalloc(c, c->d_film_rec, film_record_bytes() * (size_t)std::max<int64_t>(fired_cap, 1)));
  CK(diag_film_cells(c->v, static_cast<const int32_t *>(c->d_labels.p), lattice_ptr(c, c->cur),
                     c->cfg.G, c->cfg.rho0, h_max, eps_arm,
                     static_cast<uint8_t *>(c->d_film_state.p),
                     static_cast<unsigned long long *>(c->d_film_counts.p), fired_cap,
                     c->d_film_rec.p, false,
                     static_cast<FilmMid *>(c->d_film_mids.p), c->film_mid_queue, c->s));
  CKS(dalloc(c, c->d_count, sizeof(int32_t) * c->N));
  // mailbox: [ncomp][totals 4][film counts 5][census block][fired records]
  const size_t rec_bytes = fired ? sizeof(lbm_film_cell) * (size_t)fired_cap : 0;
  const unsigned long long *census = nullptr;
  unsigned char *mail = nullptr;
  int64_t n = 0;
  for (int pass = 0; pass < 2; ++pass) {
    const int64_t capdev = c->census_cap;
    const size_t block = sizeof(int64_t) * (65 + 2 * (size_t)capdev);
    CKS(dalloc(c, c->d_census, block));
    auto *base = static_cast<unsigned long long *>(c->d_census.p);
    int64_t *d_roots = reinterpret_cast<int64_t *>(base + 65), *d_sizes = d_roots + capdev;
    CK(diag_bubble_sizes(c->v, static_cast<const int32_t *>(c->d_labels.p),
                         static_cast<int32_t *>(c->d_count.p), base, capdev, d_roots, d_sizes,
                         nb, base + 1, c->s));
    CKS(halloc(c, c->h_mail, 80 + block + rec_bytes));
    mail = static_cast<unsigned char *>(c->h_mail.p);
    if (pass == 0) {
      CK(cudaMemcpyAsync(mail, c->d_ncomp.p, 8, cudaMemcpyDeviceToHost, c->s));
      CK(cudaMemcpyAsync(mail + 8, c->d_tot.p, 32, cudaMemcpyDeviceToHost, c->s));
      CK(cudaMemcpyAsync(mail + 40, c->d_film_counts.p, 40, cudaMemcpyDeviceToHost, c->s));
      if (labels)
        CK(cudaMemcpyAsync(labels, c->d_labels.p, sizeof(int32_t) * c->N, cudaMemcpyDeviceToHost,
                           c->s));
      if (rec_bytes)
        CK(cudaMemcpyAsync(mail + 80 + block, c->d_film_rec.p, rec_bytes, cudaMemcpyDeviceToHost,
                           c->s));
    }
    CK(cudaMemcpyAsync(mail + 80, base, block, cudaMemcpyDeviceToHost, c->s));
    CKS(sync_and_check(c));
    census = reinterpret_cast<const unsigned long long *>(mail + 80);
    n = (int64_t)census[0];
    if (n <= capdev) break;
    // more components than the census list holds: grow and redo the census
    // only; the other results stay where they are in the mailbox
    std::vector<unsigned char> keep(80);
    std::memcpy(keep.data(), mail, 80);
    std::vector<unsigned char> keep_rec(rec_bytes);
    if (rec_bytes) std::memcpy(keep_rec.data(), mail + 80 + block, rec_bytes);
    c->census_cap = n;
    const size_t block2 = sizeof(int64_t) * (65 + 2 * (size_t)n);
    CKS(halloc(c, c->h_mail, 80 + block2 + rec_bytes));
    mail = static_cast<unsigned char *>(c->h_mail.p);
    std::memcpy(mail, keep.data(), 80);
    if (rec_bytes) std::memcpy(mail + 80 + block2, keep_rec.data(), rec_bytes);
  }
  count_merges(c);
  const auto *w64 = reinterpret_cast<const unsigned long long *>(mail);
  out->ncomp = (int64_t)w64[0];
  std::memcpy(out->totals, mail + 8, 32);
  out->film.film = (int64_t)w64[5];
  out->film.midpoints = (int64_t)w64[6];
  out->film.armed = (int64_t)w64[7];
  out->film.fired = (int64_t)w64[8];
  out->merge_events = c->merge_events;
  if (n != out->ncomp) return fail(LBM_ECUDA, "interval: component count mismatch");
  // census entries in increasing root order
  const int64_t capdev = c->census_cap;
  if (n > capdev) return fail(LBM_ECUDA, "interval: census list overflow after regrowth");
  const auto *r = reinterpret_cast<const int64_t *>(census + 65);
  const int64_t *sz = r + capdev;
  std::vector<int64_t> order((size_t)n);
  for (int64_t q = 0; q < n; ++q) order[q] = q;
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return r[a] < r[b]; });
  out->nsizes = std::min(n, sizes_cap);
  for (int64_t q = 0; q < out->nsizes; ++q) {
    if (roots) roots[q] = r[order[q]];
    if (sizes) sizes[q] = sz[order[q]];
  }
  if (hist)
    for (int b = 0; b < nbins; ++b) hist[b] = (int64_t)census[1 + b];
  // fired film records in (cell, axis) order
  const size_t block = sizeof(int64_t) * (65 + 2 * (size_t)capdev);
  out->nfired = fired ? std::min<int64_t>(out->film.fired, fired_cap) : 0;
  if (out->nfired > 0) {
    std::memcpy(fired, mail + 80 + block, sizeof(lbm_film_cell) * (size_t)out->nfired);
    std::sort(fired, fired + out->nfired, [](const lbm_film_cell &a, const lbm_film_cell &b) {
      return a.cell != b.cell ? a.cell < b.cell : a.axis < b.axis;
    });
  }
  return LBM_OK;
}

lbm_status lbm_site_labels(lbm_ctx *c, int32_t *site_labels, int32_t n, int64_t *merge_events) {
  if (!c) return fail(LBM_EINVAL, "ctx is NULL");
  if (site_labels) {
    if (n != (int32_t)c->site_labels.size()) return fail(LBM_EINVAL, "n must equal the number of sites");
    std::copy(c->site_labels.begin(), c->site_labels.end(), site_labels);
  }
  if (merge_events) *merge_events = c->merge_events;
  return LBM_OK;
}

lbm_status lbm_totals(lbm_ctx *c, double out[4]) {
  if (!c || !out) return fail(LBM_EINVAL, "NULL argument");
  if (!c->seeded) return fail(LBM_ESTATE, "seed the lattice first");
  CKS(set_device(c));
  CKS(check_sticky(c));
  CKS(ensure_diag(c));
  if (c->st != LBM_F64)
    CK(diag_scan(c->v, lattice_ptr(c, c->cur), c->cfg.gas_threshold, nullptr,
                 static_cast<double *>(c->d_part.p), static_cast<double *>(c->d_tot.p),
                 static_cast<int *>(c->d_err.p), c->s));
  else
    CK(diag_totals(c->v, lattice_ptr(c, c->cur), static_cast<double *>(c->d_part.p),
                   static_cast<double *>(c->d_tot.p), c->s));
  CKS(halloc(c, c->h_mail, 4 * sizeof(double)));
  CK(cudaMemcpyAsync(c->h_mail.p, c->d_tot.p, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->s));
  CKS(sync_and_check(c));
  std::memcpy(out, c->h_mail.p, 4 * sizeof(double));
  return LBM_OK;
}

lbm_status lbm_read(lbm_ctx *c, int32_t field, double *dst, size_t bytes) {
  if (!c || !dst) return fail(LBM_EINVAL, "NULL argument");
  if (!c->seeded) return fail(LBM_ESTATE, "seed the lattice first");
  const size_t nd = (size_t)c->N * sizeof(double);
  size_t need;
  switch (field) {
    case LBM_RHO: case LBM_PSI: case LBM_P: case LBM_LAPP: need = nd; break;
    case LBM_U: need = 3 * nd; break;
    case LBM_F: need = (size_t)c->Q * nd; break;
    default: return fail(LBM_EINVAL, "unknown field");
  }
  if (bytes != need) return fail(LBM_EINVAL, "bytes must be " + std::to_string(need));
  CKS(set_device(c));
  CKS(check_sticky(c));
  CKS(ensure_diag(c));
  double *rho = static_cast<double *>(c->d_rho.p), *p = static_cast<double *>(c->d_p.p),
         *tmp = static_cast<double *>(c->d_tmp.p);
  int *err = static_cast<int *>(c->d_err.p);
  const void *cur = lattice_ptr(c, c->cur);
  switch (field) {
    case LBM_RHO:
      CK(diag_moments(c->v, cur, c->cfg.G, c->cfg.rho0, rho, nullptr, nullptr, nullptr, nullptr,
                      nullptr, err, c->s));
      CK(cudaMemcpyAsync(dst, rho, nd, cudaMemcpyDeviceToHost, c->s));
      break;
    case LBM_PSI:
      CK(diag_moments(c->v, cur, c->cfg.G, c->cfg.rho0, nullptr, nullptr, nullptr, nullptr, tmp,
                      nullptr, err, c->s));
      CK(cudaMemcpyAsync(dst, tmp, nd, cudaMemcpyDeviceToHost, c->s));
      break;
    case LBM_P:
      CKS(compute_pressure(c));
      CK(cudaMemcpyAsync(dst, p, nd, cudaMemcpyDeviceToHost, c->s));
      break;
    case LBM_LAPP:
      CKS(compute_pressure(c));
      CK(diag_laplacian(c->v, p, tmp, c->s));
      CK(cudaMemcpyAsync(dst, tmp, nd, cudaMemcpyDeviceToHost, c->s));
      break;
    case LBM_U: {
      c->p_valid = false;  // d_p holds psi below
      CKS(dalloc(c, c->d_j, 3 * nd));
      double *j = static_cast<double *>(c->d_j.p);
      CK(diag_moments(c->v, cur, c->cfg.G, c->cfg.rho0, rho, j, j + c->N, j + 2 * c->N, p, nullptr,
                      err, c->s));
      CKS(dalloc(c, c->d_u, 3 * nd));  // p holds psi here
      CK(diag_velocity(c->v, c->cfg.G, rho, j, j + c->N, j + 2 * c->N, p,
                       static_cast<double *>(c->d_u.p), c->s));
      CK(cudaMemcpyAsync(dst, c->d_u.p, 3 * nd, cudaMemcpyDeviceToHost, c->s));
      break;
    }
    case LBM_F:
      for (int i = 0; i < c->Q; ++i) {
        CK(diag_gather_pop(c->v, cur, i, tmp, c->s));
        CK(cudaMemcpyAsync(dst + (size_t)i * c->N, tmp, nd, cudaMemcpyDeviceToHost, c->s));
      }
      break;
  }
  return sync_and_check(c);
}

lbm_status lbm_write_f(lbm_ctx *c, const double *src, size_t bytes) {
  if (!c || !src) return fail(LBM_EINVAL, "NULL argument");
  const size_t nd = (size_t)c->N * sizeof(double);
  if (bytes != (size_t)c->Q * nd) return fail(LBM_EINVAL, "bytes must be Q*N*8");
  CKS(set_device(c));
  CKS(check_sticky(c));
  CKS(ensure_diag(c));
  double *tmp = static_cast<double *>(c->d_tmp.p);
  for (int i = 0; i < c->Q; ++i) {
    CK(cudaMemcpyAsync(tmp, src + (size_t)i * c->N, nd, cudaMemcpyHostToDevice, c->s));
    CK(diag_store_pop(c->v, tmp, i, lattice_ptr(c, c->cur), c->s));
  }
  if (c->resid)  // the written populations are the whole state
    CK(cudaMemsetAsync(c->d_resid.p, 0, c->d_resid.bytes, c->s));
  CK(cudaStreamSynchronize(c->s));
  c->seeded = true;
  c->film_state_clear = false;
  c->p_valid = c->labels_valid = false;
  return LBM_OK;
}

}  // extern "C"
