// Batched ensemble of independent two-bubble D2Q9 domains: the bubble-size
// sweep of Sec. 4 (Fig. 3: critical film thickness h_c against the film-disc
// radius R_d), run as many uneven lattices at once.
//
// All domains live in one arena (two FP32 offset-storage lattices each).
// One launch per tile class per time step covers every active domain: each
// CTA reads a work item (domain, x tile, chunk of rows) and runs the same
// column march as the single-lattice fused kernel, with the domain's TMA
// descriptors read from global memory.  After diag_every steps a probe
// kernel measures each active domain's film (FP64) and advances its rupture
// state machine.  The diag_every steps plus the probe (ten such intervals
// when few domains remain) are captured once into a CUDA graph and
// replayed; domains whose criterion fired (or whose film is gone) drop out
// of the work lists between replays, and within a replay their steps return
// at once.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "film.cuh"
#include "internal.h"
#include "lattice.cuh"
#include "step_fused.cuh"

namespace sclbm {
namespace {

struct EnsDomain {
  int NX, NZ;  // view extents (nx, 1, ny)
  int64_t px, popstride;
  float tau_f, omega_f, G_f, rho0_f, inv_rho0_f, rho_ref_f;
  double tau, G, rho0, rho_ref;
  float *latA, *latB;
  int64_t x0, z0, len;  // probe line start (view x, z) and length
  int e[3], ep[3];      // probe direction and perpendicular (view axes)
  double rho_mid;
};

struct EnsState {
  int32_t active, armed, fired, merged;
  int64_t step;
  double h_c, h_probe, r_d, last_d2p, last_h;
};

// D2Q9 tile classes of the ensemble (the fused tile table's D2Q9 ids)
constexpr int NCLASS = 3;
constexpr int CLASS_BX[NCLASS] = {256, 128, 64};

template <int BX, int NS>
__global__ void __launch_bounds__(BX)
    ens_step_kernel(const EnsDomain *doms, const FusedMaps *mapsA, const FusedMaps *mapsB,
                    const int4 *items, const int *count, const EnsState *st, int parity) {
  if ((int)blockIdx.x >= *count) return;
  const int4 it = items[blockIdx.x];
  const EnsDomain &D = doms[it.x];
  MarchArgs m;
  m.NX = D.NX;
  m.NY = 1;
  m.NZ = D.NZ;
  m.px = D.px;
  m.tau = D.tau;
  m.G = D.G;
  m.rho0 = D.rho0;
  m.tau_f = D.tau_f;
  m.omega_f = D.omega_f;
  m.G_f = D.G_f;
  m.rho0_f = D.rho0_f;
  m.inv_rho0_f = D.inv_rho0_f;
  m.rho_ref_f = D.rho_ref_f;
  m.tm = parity ? &mapsB[it.x] : &mapsA[it.x];
  m.x0 = it.y;
  m.y0 = 0;
  m.zs = it.z;
  m.ze = it.w;
  m.nsites = 0;
  m.sp = m.send = 0;
  m.site_x = m.site_y = m.site_z = m.bucket_site = nullptr;
  m.rate = nullptr;
  m.budget = nullptr;
  m.resid = nullptr;
  m.err = nullptr;
  m.debug_flags = 0;
  float *out = parity ? D.latA : D.latB;
  const int64_t ps = D.popstride;
  fused_barriers_init<D2Q9, ST_F32, BX, 1, NS>(m);
  // programmatic dependent launch within a class chain: the work item and
  // the domain record are never written by a step, the lattices are read
  // and written only after the previous step has completed
  asm volatile("griddepcontrol.wait;" ::: "memory");
  // a domain whose criterion was settled by a probe earlier in the same
  // launch of intervals keeps the state it had there (uniform over the CTA)
  if (!st[it.x].active) return;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  uint32_t kb = 0;
  fused_march<D2Q9, ST_F32, BX, 1, NS>(m, [&](int i) { return out + i * ps; }, kb);
}

// FP64 density / EOS pressure straight from a domain's populations
struct PopAcc {
  const EnsDomain *D;
  const float *lat;
  __device__ int64_t off(int64_t x, int64_t z) const {
    // periodic wrap without a 64-bit division (probe coordinates stay
    // within a few extents of the domain)
    int64_t xx = x, zz = z;
    while (xx >= D->NX) xx -= D->NX;
    while (xx < 0) xx += D->NX;
    while (zz >= D->NZ) zz -= D->NZ;
    while (zz < 0) zz += D->NZ;
    return zz * D->px + xx;
  }
  __device__ double rho(int64_t x, int64_t, int64_t z) const {
    const int64_t o = off(x, z);
    double r = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i)
      r += __dadd_rn(__dmul_rn(Lattice<D2Q9>::w(i), D->rho_ref), (double)lat[i * D->popstride + o]);
    return r;
  }
  // rho < mid as the FP64 sum above decides it.  The FP32 sum of the same
  // eighteen terms (w_i rho_ref and g_i) is within 20 u sum|terms| of the
  // exact value (u = 2^-24, Higham's bound for recursive summation with the
  // rounded products), so a value outside a band of 4e-6 sum|terms| around
  // mid is decided in FP32 and only the rest is summed again in FP64.
  __device__ bool below(int64_t x, int64_t y, int64_t z, double mid) const {
    const int64_t o = off(x, z);
    float r = 0.0f, s = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const float t = (float)Lattice<D2Q9>::w(i) * D->rho_ref_f, g = lat[i * D->popstride + o];
      r += t + g;
      s += fabsf(t) + fabsf(g);
    }
    const double d = (double)r - mid, band = 4e-6 * (double)s;
    if (d < -band) return true;
    if (d > band) return false;
    return rho(x, y, z) < mid;
  }
  __device__ double p(int64_t x, int64_t y, int64_t z) const {
    const double r = rho(x, y, z);
    const double s = D->rho0 * (1.0 - exp(-r / D->rho0));
    return r / 3.0 + D->G / 6.0 * s * s;
  }
};

// one CTA per domain: the film probe in parallel, then thread 0 advances the
// domain's rupture state machine
__global__ void k_ens_probe(const EnsDomain *doms, EnsState *st, int n, int parity,
                            const int64_t *step_now, double eps_arm, double h_max) {
  const int d = blockIdx.x;
  if (d >= n || !st[d].active) return;  // uniform over the CTA
  const EnsDomain &D = doms[d];
  const PopAcc acc{&D, parity ? D.latB : D.latA};
  __shared__ double out[6];
  film_probe_block(acc, D.x0, 0, D.z0, D.e, D.ep, D.len, D.rho_mid, out);
  __syncthreads();
  if (threadIdx.x != 0) return;
  EnsState s = st[d];
  s.step = *step_now;
  if (out[0] == 0.0) {  // no film: merged before the criterion
    s.merged = 1;
    s.active = 0;
  } else {
    if (out[3] > h_max) {
      s.armed = 0;  // thick film: the criterion does not apply
    } else if (out[4] < -eps_arm) {
      s.armed = 1;
    } else if (s.armed && out[4] >= 0.0) {
      // zero crossing of d2p between the previous probe (d2p < 0) and this one
      s.fired = 1;
      s.active = 0;
      s.h_c = s.last_h + (out[3] - s.last_h) * (-s.last_d2p / (out[4] - s.last_d2p));
      s.h_probe = out[3];
      s.r_d = out[5];
    }
    s.last_h = out[3];
    s.last_d2p = out[4];
  }
  st[d] = s;
}

template <int BX, int NS>
cudaError_t ens_prepare_t() {
  return cudaFuncSetAttribute(ens_step_kernel<BX, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              FusedK<D2Q9, ST_F32, BX, 1, NS>::SMEM);
}
template <int BX, int NS>
cudaError_t ens_launch_t(int grid, const EnsDomain *doms, const FusedMaps *a, const FusedMaps *b,
                  const int4 *items, const int *count, const EnsState *st, int parity,
                  cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)BX);
  cfg.dynamicSmemBytes = (size_t)FusedK<D2Q9, ST_F32, BX, 1, NS>::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, ens_step_kernel<BX, NS>, doms, a, b, items, count, st, parity);
}
// class -> (BX, NS) of the D2Q9 fused tile table
cudaError_t ens_prepare(int cls) {
  switch (cls) {
    case 0: return ens_prepare_t<256, 4>();
    case 1: return ens_prepare_t<128, 4>();
    default: return ens_prepare_t<64, 6>();
  }
}
cudaError_t ens_launch(int cls, int grid, const EnsDomain *doms, const FusedMaps *a,
                       const FusedMaps *b, const int4 *items, const int *count,
                       const EnsState *st, int parity, cudaStream_t s) {
  switch (cls) {
    case 0: return ens_launch_t<256, 4>(grid, doms, a, b, items, count, st, parity, s);
    case 1: return ens_launch_t<128, 4>(grid, doms, a, b, items, count, st, parity, s);
    default: return ens_launch_t<64, 6>(grid, doms, a, b, items, count, st, parity, s);
  }
}
int class_tile_id(int cls) { return cls == 0 ? 1 : (cls == 1 ? 2 : 3); }

}  // namespace
}  // namespace sclbm

using namespace sclbm;

struct lbm_ensemble {
  int n = 0;
  std::vector<lbm_domain> spec;
  std::vector<EnsDomain> hdom;
  std::vector<EnsState> hstate;
  std::vector<int> cls;  // tile class per domain
  cudaStream_t s = nullptr;
  // side streams of the captured interval: the tile classes hold disjoint
  // domains, so their chains of steps run concurrently
  cudaStream_t side[NCLASS] = {};
  cudaEvent_t fork = nullptr, join[NCLASS] = {};
  lbm_alloc_fn alloc = nullptr;
  lbm_free_fn free = nullptr;
  void *user = nullptr;
  std::vector<std::pair<void *, size_t>> bufs;
  char *arena = nullptr;
  size_t arena_bytes = 0;
  EnsDomain *d_dom = nullptr;
  FusedMaps *d_mapsA = nullptr, *d_mapsB = nullptr;
  EnsState *d_state = nullptr;
  int64_t *d_step = nullptr;
  int4 *d_items[NCLASS] = {};
  int *d_count[NCLASS] = {};
  int max_items[NCLASS] = {};
  int zlen = 16;  // rows per work item (chosen at every regrid)
  int nsm = 152;
  double eps_arm = 0, h_max = 8;
  int diag_every = 100;
  int64_t steps = 0;
  double updates = 0;  // lattice updates performed
  int64_t launches = 0;
  // captured launches of one interval and of ENS_BATCH intervals
  cudaGraph_t graph = nullptr, graph_b = nullptr;
  cudaGraphExec_t exec = nullptr, exec_b = nullptr;
  // pinned host copies of the step counters (one per interval of a launch)
  // and the domain states, so that a launch's two transfers are plain
  // asynchronous copies
  int64_t *h_step = nullptr;
  EnsState *h_state = nullptr;
};

namespace {

lbm_status efail(lbm_status st, const std::string &m) { return set_error(st, m.c_str()); }

#define ECK(call)                                                                   \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      cudaGetLastError();                                                           \
      return efail(LBM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
    }                                                                               \
  } while (0)
#define ECKS(expr)               \
  do {                           \
    lbm_status s_ = (expr);      \
    if (s_ != LBM_OK) return s_; \
  } while (0)

lbm_status ealloc(lbm_ensemble *E, size_t bytes, void **out) {
  if (bytes == 0) bytes = 16;
  void *p = nullptr;
  if (E->alloc) {
    p = E->alloc(bytes, E->s, E->user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (!p) return efail(LBM_ENOMEM, "ensemble: device allocation of " + std::to_string(bytes) + " bytes failed");
  E->bufs.push_back({p, bytes});
  *out = p;
  return LBM_OK;
}

void efree_all(lbm_ensemble *E) {
  for (auto &b : E->bufs) {
    if (E->alloc && E->free)
      E->free(b.first, b.second, E->s, E->user);
    else if (!E->alloc)
      cudaFree(b.first);
  }
  E->bufs.clear();
}

// Work items of the active domains of each class.  Rows are cut into chunks
// of at most zmax rows: a CTA marches its chunk row by row, so the chunk
// length sets the latency of a step, and short chunks give many independent
// items.  Every chunk also stages the two rows around it, so long chunks
// are cheaper while there are enough of them to fill the GPU.
constexpr int ENS_ZLEN_MAX = 16, ENS_ZLEN_MIN = 2;
// With few domains left, a launch covers ENS_BATCH intervals: the host's
// per-interval round trip (graph launch, state copy, synchronisation) then
// comes once per ENS_BATCH probes.  A domain settled by one of the probes
// is skipped by the later steps of the launch, so it keeps the state of its
// settling probe, as with one interval per launch.
constexpr int ENS_BATCH = 10, ENS_BATCH_ACTIVE = 32;

int chunk_len(int ny, int zmax) {
  int zlen = std::min(ny, zmax);
  const int nzc = (ny + zlen - 1) / zlen;
  return (ny + nzc - 1) / nzc;
}

lbm_status build_items(lbm_ensemble *E, int counts[NCLASS]) {
  for (int c = 0; c < NCLASS; ++c) {
    std::vector<int4> it;
    for (int d = 0; d < E->n; ++d) {
      if (E->cls[d] != c || !E->hstate[d].active) continue;
      const int bx = CLASS_BX[c];
      const int nx = E->hdom[d].NX, ny = E->hdom[d].NZ;
      const int tiles_x = (nx + bx - 1) / bx;
      const int zlen = chunk_len(ny, E->zlen);
      const int nzc = (ny + zlen - 1) / zlen;
      for (int zc = 0; zc < nzc; ++zc)
        for (int tx = 0; tx < tiles_x; ++tx)
          it.push_back(make_int4(d, tx * bx, zc * zlen, std::min(ny, (zc + 1) * zlen)));
    }
    const int cnt = (int)it.size();
    counts[c] = cnt;
    if (cnt > 0)
      ECK(cudaMemcpyAsync(E->d_items[c], it.data(), sizeof(int4) * cnt, cudaMemcpyHostToDevice, E->s));
    ECK(cudaMemcpyAsync(E->d_count[c], &cnt, sizeof(int), cudaMemcpyHostToDevice, E->s));
    ECK(cudaStreamSynchronize(E->s));  // host staging vectors go out of scope
  }
  return LBM_OK;
}

int count_items(const lbm_ensemble *E, int d, int c, int zmax) {
  const int bx = CLASS_BX[c];
  const int nx = E->hdom[d].NX, ny = E->hdom[d].NZ;
  const int zlen = chunk_len(ny, zmax);
  return ((nx + bx - 1) / bx) * ((ny + zlen - 1) / zlen);
}

// the longest chunk (16, 8, 4, 2 rows) that still gives the active domains
// at least four CTAs per SM
int choose_zlen(const lbm_ensemble *E) {
  int z = ENS_ZLEN_MAX;
  for (; z > ENS_ZLEN_MIN; z /= 2) {
    int64_t items = 0;
    for (int d = 0; d < E->n; ++d)
      if (E->hstate[d].active) items += count_items(E, d, E->cls[d], z);
    if (items >= 4LL * E->nsm) break;
  }
  return z;
}

void drop_graph(lbm_ensemble *E) {
  if (E->exec) cudaGraphExecDestroy(E->exec);
  if (E->graph) cudaGraphDestroy(E->graph);
  if (E->exec_b) cudaGraphExecDestroy(E->exec_b);
  if (E->graph_b) cudaGraphDestroy(E->graph_b);
  E->exec = E->exec_b = nullptr;
  E->graph = E->graph_b = nullptr;
}

// one diagnostic interval (the k-th of a launch): diag_every steps of every
// class, then the probe, which stamps settled domains with step counter k
lbm_status enqueue_interval(lbm_ensemble *E, int k) {
  // fork: one chain of diag_every steps per tile class, joined before the probe
  ECK(cudaEventRecord(E->fork, E->s));
  for (int c = 0; c < NCLASS; ++c) {
    if (E->max_items[c] == 0) continue;
    ECK(cudaStreamWaitEvent(E->side[c], E->fork, 0));
    for (int t = 0; t < E->diag_every; ++t)
      ECK(ens_launch(c, E->max_items[c], E->d_dom, E->d_mapsA, E->d_mapsB, E->d_items[c],
                     E->d_count[c], E->d_state, t & 1, E->side[c]));
    ECK(cudaEventRecord(E->join[c], E->side[c]));
    ECK(cudaStreamWaitEvent(E->s, E->join[c], 0));
  }
  k_ens_probe<<<E->n, 256, 0, E->s>>>(E->d_dom, E->d_state, E->n, 0, E->d_step + k, E->eps_arm,
                                       E->h_max);
  ECK(cudaGetLastError());
  return LBM_OK;
}

lbm_status ensure_graph(lbm_ensemble *E, int K) {
  cudaGraph_t &graph = K == 1 ? E->graph : E->graph_b;
  cudaGraphExec_t &exec = K == 1 ? E->exec : E->exec_b;
  if (exec) return LBM_OK;
  ECK(cudaStreamBeginCapture(E->s, cudaStreamCaptureModeThreadLocal));
  lbm_status st = LBM_OK;
  for (int k = 0; k < K && st == LBM_OK; ++k) st = enqueue_interval(E, k);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(E->s, &g);
  if (st != LBM_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  ECK(e);
  graph = g;
  ECK(cudaGraphInstantiate(&exec, g, 0));
  return LBM_OK;
}

// K intervals in one launch (K = 1 or ENS_BATCH), then the domain states
// on the host.  A domain that a probe of this launch settled was stepped up
// to that probe's step counter, which its state records.
lbm_status ens_interval(lbm_ensemble *E, int K) {
  std::vector<char> was(E->n);
  for (int d = 0; d < E->n; ++d) was[d] = E->hstate[d].active != 0;
  for (int k = 0; k < K; ++k) E->h_step[k] = E->steps + (int64_t)(k + 1) * E->diag_every;
  ECK(cudaMemcpyAsync(E->d_step, E->h_step, sizeof(int64_t) * K, cudaMemcpyHostToDevice, E->s));
  ECKS(ensure_graph(E, K));
  ECK(cudaGraphLaunch(K == 1 ? E->exec : E->exec_b, E->s));
  ECK(cudaMemcpyAsync(E->h_state, E->d_state, sizeof(EnsState) * E->n, cudaMemcpyDeviceToHost,
                      E->s));
  ECK(cudaStreamSynchronize(E->s));
  std::copy(E->h_state, E->h_state + E->n, E->hstate.begin());
  const int64_t end = E->steps + (int64_t)K * E->diag_every;
  for (int d = 0; d < E->n; ++d) {
    if (!was[d]) continue;
    const EnsState &st = E->hstate[d];
    const int64_t ran = (st.active ? end : st.step) - E->steps;
    E->updates += (double)E->hdom[d].NX * E->hdom[d].NZ * (double)ran;
  }
  E->steps = end;
  int ncls = 0;
  for (int c = 0; c < NCLASS; ++c) ncls += E->max_items[c] > 0;
  E->launches += (int64_t)K * ((int64_t)E->diag_every * ncls + 1);
  return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_ensemble_create(const lbm_domain *dom, int32_t n, double eps_arm,
                               double h_max, int32_t diag_every, lbm_alloc_fn alloc,
                               lbm_free_fn free_fn, void *alloc_user, lbm_ensemble **out) {
  if (!out) return efail(LBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!dom || n < 1) return efail(LBM_EINVAL, "need at least one domain");
  if (diag_every < 2 || diag_every % 2) return efail(LBM_EINVAL, "diag_every must be even and >= 2");
  if (!(eps_arm >= 0) || !(h_max > 0)) return efail(LBM_EINVAL, "eps_arm >= 0 and h_max > 0");
  if ((alloc == nullptr) != (free_fn == nullptr))
    return efail(LBM_EINVAL, "alloc and free callbacks must be given together");
  for (int d = 0; d < n; ++d) {
    const lbm_domain &s = dom[d];
    if (s.nx < 8 || s.ny < 8 || s.nx % 4 || s.nx > 4096 || s.ny > 4096)
      return efail(LBM_EINVAL, "domain " + std::to_string(d) + ": nx, ny in [8, 4096], nx % 4 == 0");
    if (!(s.tau > 0.5) || !(s.rho0 > 0) || s.nbubbles < 0 || s.nbubbles > 4 || !(s.width > 0))
      return efail(LBM_EINVAL, "domain " + std::to_string(d) + ": bad parameters");
    if (s.line[3] < 0 || s.line[3] > 1 || s.line[4] < 2)
      return efail(LBM_EINVAL, "domain " + std::to_string(d) + ": probe line axis 0/1, len >= 2");
  }
  lbm_ensemble *E = new lbm_ensemble();
  E->n = n;
  E->spec.assign(dom, dom + n);
  E->alloc = alloc;
  E->free = free_fn;
  E->user = alloc_user;
  E->eps_arm = eps_arm;
  E->h_max = h_max;
  E->diag_every = diag_every;
  auto bail = [&](lbm_status st) {
    lbm_ensemble_destroy(E);
    return st;
  };
  bool streams_ok = cudaStreamCreateWithFlags(&E->s, cudaStreamNonBlocking) == cudaSuccess &&
                    cudaEventCreateWithFlags(&E->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int c = 0; c < NCLASS && streams_ok; ++c)
    streams_ok = cudaStreamCreateWithFlags(&E->side[c], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&E->join[c], cudaEventDisableTiming) == cudaSuccess;
  if (!streams_ok) {
    cudaGetLastError();
    lbm_ensemble_destroy(E);
    return efail(LBM_ECUDA, "ensemble: stream creation failed");
  }
  if (cudaMallocHost(reinterpret_cast<void **>(&E->h_step), sizeof(int64_t) * ENS_BATCH) !=
          cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void **>(&E->h_state), sizeof(EnsState) * (size_t)n) !=
          cudaSuccess) {
    cudaGetLastError();
    lbm_ensemble_destroy(E);
    return efail(LBM_ENOMEM, "ensemble: pinned host allocation failed");
  }
  // arena layout
  std::vector<size_t> off(n);
  size_t total = 0;
  int64_t max_cells = 0;
  for (int d = 0; d < n; ++d) {
    const int64_t px = (dom[d].nx + 7) / 8 * 8;
    const size_t lat = (size_t)9 * px * dom[d].ny * sizeof(float);
    off[d] = total;
    total += 2 * ((lat + 255) / 256 * 256);
    max_cells = std::max<int64_t>(max_cells, dom[d].nx * dom[d].ny);
  }
  void *p;
  lbm_status st;
  if ((st = ealloc(E, total, &p)) != LBM_OK) return bail(st);
  E->arena = static_cast<char *>(p);
  E->arena_bytes = total;
  E->hdom.resize(n);
  E->hstate.assign(n, EnsState{});
  E->cls.resize(n);
  for (int d = 0; d < n; ++d) {
    const lbm_domain &s = dom[d];
    EnsDomain &D = E->hdom[d];
    D.NX = (int)s.nx;
    D.NZ = (int)s.ny;
    D.px = (s.nx + 7) / 8 * 8;
    D.popstride = D.px * s.ny;
    D.tau = s.tau;
    D.G = s.G;
    D.rho0 = s.rho0;
    D.rho_ref = s.rho_ref;
    D.tau_f = (float)s.tau;
    D.omega_f = (float)(1.0 / s.tau);
    D.G_f = (float)s.G;
    D.rho0_f = (float)s.rho0;
    D.inv_rho0_f = (float)(1.0 / s.rho0);
    D.rho_ref_f = (float)s.rho_ref;
    const size_t lat = (size_t)9 * D.px * s.ny * sizeof(float);
    D.latA = reinterpret_cast<float *>(E->arena + off[d]);
    D.latB = reinterpret_cast<float *>(E->arena + off[d] + (lat + 255) / 256 * 256);
    // probe line, user (x, y) -> view (x, 0, y)
    D.x0 = ((s.line[0] % s.nx) + s.nx) % s.nx;
    D.z0 = ((s.line[1] % s.ny) + s.ny) % s.ny;
    D.len = s.line[4];
    D.e[0] = D.e[1] = D.e[2] = D.ep[0] = D.ep[1] = D.ep[2] = 0;
    if (s.line[3] == 0) {
      D.e[0] = 1;
      D.ep[2] = 1;
    } else {
      D.e[2] = 1;
      D.ep[0] = 1;
    }
    D.rho_mid = s.rho_mid;
    E->cls[d] = s.nx >= 256 ? 0 : (s.nx >= 128 ? 1 : 2);
    E->hstate[d].active = 1;
  }
  if ((st = ealloc(E, sizeof(EnsDomain) * n, &p)) != LBM_OK) return bail(st);
  E->d_dom = static_cast<EnsDomain *>(p);
  if ((st = ealloc(E, sizeof(FusedMaps) * n, &p)) != LBM_OK) return bail(st);
  E->d_mapsA = static_cast<FusedMaps *>(p);
  if ((st = ealloc(E, sizeof(FusedMaps) * n, &p)) != LBM_OK) return bail(st);
  E->d_mapsB = static_cast<FusedMaps *>(p);
  if ((st = ealloc(E, sizeof(EnsState) * n, &p)) != LBM_OK) return bail(st);
  E->d_state = static_cast<EnsState *>(p);
  if ((st = ealloc(E, sizeof(int64_t) * ENS_BATCH, &p)) != LBM_OK) return bail(st);
  E->d_step = static_cast<int64_t *>(p);
  // work-list capacity per class: every domain could be moved to any class
  for (int c = 0; c < NCLASS; ++c) {
    int cap = 0;
    for (int d = 0; d < n; ++d) cap += count_items(E, d, c, ENS_ZLEN_MIN);
    E->max_items[c] = 0;
    if ((st = ealloc(E, sizeof(int4) * cap, &p)) != LBM_OK) return bail(st);
    E->d_items[c] = static_cast<int4 *>(p);
    if ((st = ealloc(E, sizeof(int), &p)) != LBM_OK) return bail(st);
    E->d_count[c] = static_cast<int *>(p);
    if (ens_prepare(c) != cudaSuccess) {
      cudaGetLastError();
      return bail(efail(LBM_ECUDA, "ensemble kernel set-up failed"));
    }
  }
  // TMA descriptors per domain and lattice
  std::vector<FusedMaps> ma(n), mb(n);
  for (int d = 0; d < n; ++d) {
    const EnsDomain &D = E->hdom[d];
    const int c = E->cls[d];
    FusedPlan pl;
    if (fused_make_plan(D2Q9, ST_F32, class_tile_id(c), D.NX, 1, D.NZ, 1, &pl) != cudaSuccess) {
      cudaGetLastError();
      return bail(efail(LBM_EINVAL, "ensemble: no tile plan for domain " + std::to_string(d)));
    }
    // the descriptors depend only on the tile width through the box
    // extents; encode with every class's box is unnecessary: boxes are
    // (BX, 1, 1, 9) and (HX, 1, 1, 9), re-encoded when a class changes
    if (fused_encode_maps(D2Q9, ST_F32, pl, D.latA, D.NX, 1, D.NZ, D.px, &ma[d]) != CUDA_SUCCESS ||
        fused_encode_maps(D2Q9, ST_F32, pl, D.latB, D.NX, 1, D.NZ, D.px, &mb[d]) != CUDA_SUCCESS)
      return bail(efail(LBM_ECUDA, "ensemble: cuTensorMapEncodeTiled failed"));
  }
  if (cudaMemcpyAsync(E->d_mapsA, ma.data(), sizeof(FusedMaps) * n, cudaMemcpyHostToDevice, E->s) != cudaSuccess ||
      cudaMemcpyAsync(E->d_mapsB, mb.data(), sizeof(FusedMaps) * n, cudaMemcpyHostToDevice, E->s) != cudaSuccess ||
      cudaMemcpyAsync(E->d_dom, E->hdom.data(), sizeof(EnsDomain) * n, cudaMemcpyHostToDevice, E->s) != cudaSuccess ||
      cudaMemcpyAsync(E->d_state, E->hstate.data(), sizeof(EnsState) * n, cudaMemcpyHostToDevice, E->s) != cudaSuccess) {
    cudaGetLastError();
    return bail(efail(LBM_ECUDA, "ensemble: upload failed"));
  }
  // initial state of every domain (FP64 density field, then populations)
  double *rho = nullptr, *bub = nullptr;
  if ((st = ealloc(E, sizeof(double) * max_cells, &p)) != LBM_OK) return bail(st);
  rho = static_cast<double *>(p);
  if ((st = ealloc(E, sizeof(double) * 16, &p)) != LBM_OK) return bail(st);
  bub = static_cast<double *>(p);
  for (int d = 0; d < n; ++d) {
    const lbm_domain &s = dom[d];
    const EnsDomain &D = E->hdom[d];
    View v{D2Q9, ST_F32, D.NX, 1, D.NZ, D.px, s.rho_ref};
    view_prepare(v);
    double hb[16];
    for (int b = 0; b < s.nbubbles; ++b) {
      hb[4 * b + 0] = s.bubbles[b].x;
      hb[4 * b + 1] = 0.0;
      hb[4 * b + 2] = s.bubbles[b].y;
      hb[4 * b + 3] = s.bubbles[b].r;
    }
    if (cudaMemcpyAsync(bub, hb, sizeof(hb), cudaMemcpyHostToDevice, E->s) != cudaSuccess ||
        diag_init_rho(v, bub, s.nbubbles, s.rho_l, s.rho_g, s.width, s.noise_amp, s.seed, rho,
                      E->s) != cudaSuccess ||
        diag_store_from_rho(v, rho, D.latA, E->s) != cudaSuccess ||
        cudaStreamSynchronize(E->s) != cudaSuccess) {
      cudaGetLastError();
      return bail(efail(LBM_ECUDA, "ensemble: initial state failed"));
    }
  }
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&E->nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  E->zlen = choose_zlen(E);
  int counts[NCLASS];
  if ((st = build_items(E, counts)) != LBM_OK) return bail(st);
  for (int c = 0; c < NCLASS; ++c) E->max_items[c] = counts[c];
  *out = E;
  return LBM_OK;
}

void lbm_ensemble_destroy(lbm_ensemble *E) {
  if (!E) return;
  if (E->s) cudaStreamSynchronize(E->s);
  drop_graph(E);
  efree_all(E);
  for (int c = 0; c < NCLASS; ++c) {
    if (E->side[c]) cudaStreamDestroy(E->side[c]);
    if (E->join[c]) cudaEventDestroy(E->join[c]);
  }
  if (E->fork) cudaEventDestroy(E->fork);
  if (E->s) cudaStreamDestroy(E->s);
  if (E->h_step) cudaFreeHost(E->h_step);
  if (E->h_state) cudaFreeHost(E->h_state);
  cudaGetLastError();
  delete E;
}

// After the active set changed: new work lists; the captured grids (one
// CTA per item) are re-captured when a class emptied or shrank by half, so
// that finished domains stop costing launches.
static lbm_status refresh_work(lbm_ensemble *E) {
  const int z = choose_zlen(E);
  bool regrid = z != E->zlen;
  E->zlen = z;
  int counts[NCLASS];
  ECKS(build_items(E, counts));
  for (int c = 0; c < NCLASS; ++c)
    regrid |= (counts[c] == 0) != (E->max_items[c] == 0) || 2 * counts[c] < E->max_items[c];
  for (int c = 0; c < NCLASS; ++c) regrid |= counts[c] > E->max_items[c];
  if (regrid) {
    drop_graph(E);
    for (int c = 0; c < NCLASS; ++c) E->max_items[c] = counts[c];
  }
  return LBM_OK;
}

lbm_status lbm_ensemble_run(lbm_ensemble *E, int64_t max_steps, int64_t *steps_done) {
  if (!E) return efail(LBM_EINVAL, "ensemble is NULL");
  if (max_steps < 0) return efail(LBM_EINVAL, "max_steps < 0");
  const int64_t start = E->steps;
  while (E->steps - start < max_steps) {
    int active = 0;
    for (int d = 0; d < E->n; ++d) active += E->hstate[d].active;
    if (!active) break;
    std::vector<int32_t> before(E->n);
    for (int d = 0; d < E->n; ++d) before[d] = E->hstate[d].active;
    const int64_t left = max_steps - (E->steps - start);
    const int K = active <= ENS_BATCH_ACTIVE && left >= (int64_t)ENS_BATCH * E->diag_every
                      ? ENS_BATCH : 1;
    ECKS(ens_interval(E, K));
    bool changed = false;
    for (int d = 0; d < E->n; ++d) changed |= before[d] != E->hstate[d].active;
    if (changed) ECKS(refresh_work(E));
  }
  if (steps_done) *steps_done = E->steps - start;
  return LBM_OK;
}

lbm_status lbm_ensemble_results(const lbm_ensemble *E, lbm_rupture *out, int32_t n) {
  if (!E || !out) return efail(LBM_EINVAL, "NULL argument");
  if (n != E->n) return efail(LBM_EINVAL, "n must equal the number of domains");
  for (int d = 0; d < n; ++d) {
    const EnsState &s = E->hstate[d];
    out[d].fired = s.fired;
    out[d].merged = s.merged;
    out[d].steps = s.active ? E->steps : s.step;
    out[d].h_c = s.h_c;
    out[d].h_probe = s.h_probe;
    out[d].r_d = s.r_d;
  }
  return LBM_OK;
}

lbm_status lbm_ensemble_stats(const lbm_ensemble *E, double out[4]) {
  if (!E || !out) return efail(LBM_EINVAL, "NULL argument");
  int active = 0;
  for (int d = 0; d < E->n; ++d) active += E->hstate[d].active;
  out[0] = (double)E->steps;
  out[1] = E->updates;
  out[2] = (double)active;
  out[3] = (double)E->launches;
  return LBM_OK;
}

lbm_status lbm_ensemble_read_f(lbm_ensemble *E, int32_t d, double *host, size_t bytes) {
  if (!E || !host || d < 0 || d >= E->n) return efail(LBM_EINVAL, "bad arguments");
  const EnsDomain &D = E->hdom[d];
  const size_t N = (size_t)D.NX * D.NZ;
  if (bytes != 9 * N * sizeof(double)) return efail(LBM_EINVAL, "bytes must be 9*nx*ny*8");
  // the current lattice of a domain: A after an even number of its steps
  const EnsState &s = E->hstate[d];
  const int64_t its = s.active ? E->steps : s.step;
  const float *lat = (its & 1) ? D.latB : D.latA;
  View v{D2Q9, ST_F32, D.NX, 1, D.NZ, D.px, D.rho_ref};
  view_prepare(v);
  void *p;
  ECKS(ealloc(E, N * sizeof(double), &p));
  double *tmp = static_cast<double *>(p);
  lbm_status st = LBM_OK;
  for (int i = 0; i < 9 && st == LBM_OK; ++i) {
    if (diag_gather_pop(v, lat, i, tmp, E->s) != cudaSuccess ||
        cudaMemcpyAsync(host + i * N, tmp, N * sizeof(double), cudaMemcpyDeviceToHost, E->s) !=
            cudaSuccess) {
      cudaGetLastError();
      st = efail(LBM_ECUDA, "ensemble: read failed");
    }
  }
  cudaStreamSynchronize(E->s);
  // release the temporary
  for (size_t k = 0; k < E->bufs.size(); ++k)
    if (E->bufs[k].first == p) {
      if (E->alloc && E->free)
        E->free(p, E->bufs[k].second, E->s, E->user);
      else if (!E->alloc)
        cudaFree(p);
      E->bufs.erase(E->bufs.begin() + k);
      break;
    }
  return st;
}

}  // extern "C"
