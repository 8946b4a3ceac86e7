// Batched ensemble of independent two-bubble D2Q9 domains: the bubble-size
// sweep of Sec. 4 (Fig. 3: critical film thickness h_c against the film-disc
// radius R_d), run as many uneven lattices at once.
//
// All domains live in one arena (two FP32 offset-storage lattices each).
// An interval is diag_every steps of every active domain followed by a
// probe kernel that measures each active domain's film (FP64), advances its
// step counter and its rupture state machine.  The interval's launches are
// captured once per launch form into a CUDA graph and replayed (ten times
// per host round trip when few domains remain); domains whose criterion
// fired (or whose film is gone) drop out of the work lists between
// replays, and within a replay their launches return at once.  Launch
// forms:
//   - per-step launches, one per tile class: each CTA reads a work item
//     (domain, x tile, chunk of rows) and runs the single-lattice x-pair
//     column march (two cells per thread) with the domain's TMA descriptors;
//   - temporally blocked launches (ensemble_tb.cuh): a CTA advances a tile
//     with a 2 S-cell halo S steps in shared memory;
//   - persistent cooperative launches, in which each CTA keeps its work item
//     for ten intervals and waits only on its neighbours' step flags.
// All forms give bit-identical populations.  By default the form is chosen
// by measured time as the active set shrinks (see auto_form).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "ensemble_tb.cuh"
#include "film.cuh"
#include "internal.h"
#include "lattice.cuh"
#include "step_fused.cuh"
#include "step_fused_x2.cuh"

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

// The march arguments of work item it (domain, x0, zs, ze) of domain D
// with the TMA descriptors tm of its input lattice.
__device__ __forceinline__ MarchArgs ens_march_args(const EnsDomain &D, const int4 it,
                                                    const FusedMaps *tm) {
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
  m.tm = tm;
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
  return m;
}

template <int BX, int NS>
__global__ void __launch_bounds__(BX / 2)
    ens_step_kernel(const EnsDomain *doms, const FusedMaps *mapsA, const FusedMaps *mapsB,
                    const int4 *items, const int *count, const EnsState *st, int parity) {
  if ((int)blockIdx.x >= *count) return;
  const int4 it = items[blockIdx.x];
  const EnsDomain &D = doms[it.x];
  MarchArgs m = ens_march_args(D, it, parity ? &mapsB[it.x] : &mapsA[it.x]);
  float *out = parity ? D.latA : D.latB;
  const int64_t ps = D.popstride;
  fused_barriers_init_k<FusedK2<D2Q9, ST_F32, BX, 1, NS>>(m);
  // programmatic dependent launch within a class chain: the work item and
  // the domain record are never written by a step, the lattices are read
  // and written only after the previous step has completed
  asm volatile("griddepcontrol.wait;" ::: "memory");
  // a domain whose criterion was settled by a probe earlier in the same
  // launch of intervals keeps the state it had there (uniform over the CTA)
  if (!st[it.x].active) return;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  uint32_t kb = 0;
  fused_march_x2<D2Q9, ST_F32, BX, 1, NS>(m, [&](int i) { return out + i * ps; }, kb);
}

// ---- temporally blocked steps (S steps per launch) ---------------------------
template <int TX, int TZ, int S, int NT>
__global__ void __launch_bounds__(NT)
    ens_tb_kernel(const EnsDomain *doms, const int4 *items, const int *count, const EnsState *st,
                  int parity) {
  if ((int)blockIdx.x >= *count) return;
  const int4 it = items[blockIdx.x];  // (domain, x0, z0, -)
  const EnsDomain &E = doms[it.x];
  TbDomain D;
  D.NX = E.NX;
  D.NZ = E.NZ;
  D.px = E.px;
  D.popstride = E.popstride;
  D.tau = E.tau_f;
  D.omega = E.omega_f;
  D.G = E.G_f;
  D.rho0 = E.rho0_f;
  D.inv_rho0 = E.inv_rho0_f;
  D.rho_ref = E.rho_ref_f;
  D.in = parity ? E.latB : E.latA;
  D.out = parity ? E.latA : E.latB;
  // programmatic dependent launch: the lattices are read and written only
  // after the previous launch has completed
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (!st[it.x].active) return;  // settled earlier in the same launch of intervals
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  ens_tb_tile<EnsTB<TX, TZ, S>, NT>(D, it.y, it.z);
}

// Tile configurations of the temporally blocked launch: (TX, TZ, S, threads).
constexpr int NTB = 8;
constexpr int TB_TX[NTB] = {32, 32, 24, 16, 64, 32, 16, 32},
              TB_TZ[NTB] = {32, 16, 24, 16, 16, 16, 16, 8},
              TB_S[NTB] = {5, 5, 2, 2, 2, 5, 5, 5},
              TB_NT[NTB] = {1024, 512, 512, 256, 512, 1024, 512, 512};
template <int C>
using TbCfg = EnsTB<TB_TX[C], TB_TZ[C], TB_S[C]>;
template <int C>
constexpr auto tb_kernel_of() {
  return ens_tb_kernel<TB_TX[C], TB_TZ[C], TB_S[C], TB_NT[C]>;
}
template <int C>
cudaError_t tb_launch_t(int grid, const EnsDomain *doms, const int4 *items, const int *count,
                        const EnsState *st, int parity, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)TB_NT[C]);
  cfg.dynamicSmemBytes = (size_t)TbCfg<C>::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, tb_kernel_of<C>(), doms, items, count, st, parity);
}
template <int C>
cudaError_t tb_prepare_t() {
  return cudaFuncSetAttribute(tb_kernel_of<C>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                              TbCfg<C>::SMEM);
}
cudaError_t tb_prepare(int c) {
  switch (c) {
    case 5: return tb_prepare_t<5>();
    case 6: return tb_prepare_t<6>();
    case 7: return tb_prepare_t<7>();
    case 0: return cudaFuncSetAttribute(tb_kernel_of<0>(), cudaFuncAttributeMaxDynamicSharedMemorySize, TbCfg<0>::SMEM);
    case 1: return cudaFuncSetAttribute(tb_kernel_of<1>(), cudaFuncAttributeMaxDynamicSharedMemorySize, TbCfg<1>::SMEM);
    case 2: return cudaFuncSetAttribute(tb_kernel_of<2>(), cudaFuncAttributeMaxDynamicSharedMemorySize, TbCfg<2>::SMEM);
    case 3: return cudaFuncSetAttribute(tb_kernel_of<3>(), cudaFuncAttributeMaxDynamicSharedMemorySize, TbCfg<3>::SMEM);
    default: return cudaFuncSetAttribute(tb_kernel_of<4>(), cudaFuncAttributeMaxDynamicSharedMemorySize, TbCfg<4>::SMEM);
  }
}
cudaError_t tb_launch(int c, int grid, const EnsDomain *doms, const int4 *items, const int *count,
                      const EnsState *st, int parity, cudaStream_t s) {
  switch (c) {
    case 0: return tb_launch_t<0>(grid, doms, items, count, st, parity, s);
    case 1: return tb_launch_t<1>(grid, doms, items, count, st, parity, s);
    case 2: return tb_launch_t<2>(grid, doms, items, count, st, parity, s);
    case 3: return tb_launch_t<3>(grid, doms, items, count, st, parity, s);
    case 4: return tb_launch_t<4>(grid, doms, items, count, st, parity, s);
    case 5: return tb_launch_t<5>(grid, doms, items, count, st, parity, s);
    case 6: return tb_launch_t<6>(grid, doms, items, count, st, parity, s);
    default: return tb_launch_t<7>(grid, doms, items, count, st, parity, s);
  }
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

// The film probe of domain D on lattice `parity` (A = 0) at the end of an
// interval of diag_every steps, run by a whole CTA; then thread 0 advances
// the domain's step counter and its rupture state machine in *sp (a settled
// domain keeps the step it settled at).  Returns, to every thread, whether
// the domain is still active.
__device__ __noinline__ bool ens_probe_domain(const EnsDomain &D, EnsState *sp, int parity,
                                              int diag_every, double eps_arm, double h_max) {
  const PopAcc acc{&D, parity ? D.latB : D.latA};
  __shared__ double out[6];
  __shared__ int s_active;
  // R_d is recorded only by a probe that fires: the disc rows are scanned
  // only under the firing branch of the state machine below
  const bool armed = sp->armed;
  film_probe_block(acc, D.x0, 0, D.z0, D.e, D.ep, D.len, D.rho_mid, out,
                   [&](double h, double d2p) {
                     return !(h > h_max) && !(d2p < -eps_arm) && armed && d2p >= 0.0;
                   });
  __syncthreads();
  if (threadIdx.x == 0) {
    EnsState s = *sp;
    s.step += diag_every;
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
    *sp = s;
    s_active = s.active;
  }
  __syncthreads();
  return s_active != 0;
}

// one CTA per active domain
__global__ void k_ens_probe(const EnsDomain *doms, EnsState *st, int n, int parity, int diag_every,
                            double eps_arm, double h_max) {
  const int d = blockIdx.x;
  if (d >= n || !st[d].active) return;  // uniform over the CTA
  ens_probe_domain(doms[d], &st[d], parity, diag_every, eps_arm, h_max);
}

// ---- persistent launch -----------------------------------------------------
// Once the active domains' work items fit in one wave, one cooperative
// launch runs nint intervals: each CTA keeps its work item for the whole
// launch and marches it once per step.  The rows a step stages were written
// in the previous step by items at most two chunks and two tiles away (push
// streaming moves populations by one cell and a chunk stages one row on
// each side of its own; only the last tile of a row is narrower than a
// tile), and the rows it writes were staged one step before by those same
// items.  So a CTA starts step j + 1 once those items (up to 25, periodic)
// have released their flag for step j: no grid-wide barrier.  At the end
// of an interval the domain's first CTA waits for the whole domain, probes
// it and releases its verdict, which the other CTAs read before their next
// step.  Every wait has a time limit, after which the CTA sets
// ERR_SYNC_TIMEOUT and returns; waits give up at once when another CTA has
// set an error bit.
struct EnsRunArgs {
  const EnsDomain *doms;
  const FusedMaps *mapsA, *mapsB;
  const int4 *items;        // (domain, x0, zs, ze) per CTA
  const int4 *layout;       // (first item, tiles, chunks, items) per active domain
  EnsState *st;
  uint32_t *flags;          // steps completed in this launch, per item (zero at launch)
  uint32_t *pflag;          // intervals probed in this launch, per domain (zero at launch)
  int *err;
  int nint, diag_every;
  int withhold;  // test hook: CTA 0 never releases its step flag
  double eps_arm, h_max;
};

constexpr uint64_t ENS_WAIT_NS = 1000000000ull;  // 1 s

// Wait until *p >= target, then an acquire fence (the flag's release store
// and everything before it happen before what follows); false after the
// time limit or when another CTA has reported an error.  The flag is polled
// with relaxed loads and a short back-off, so that many waiting CTAs do not
// crowd the lines of the flags they wait for.
__device__ bool ens_wait_at_least(const uint32_t *p, uint32_t target, int *err) {
  if (ld_relaxed_u32(p) < target) {
    const uint64_t t0 = globaltimer_ns();
    do {
      __nanosleep(32);
      if (ld_relaxed_u32(reinterpret_cast<const uint32_t *>(err)) != 0) return false;
      if (globaltimer_ns() - t0 > ENS_WAIT_NS) {
        atomicOr(err, ERR_SYNC_TIMEOUT);
        return false;
      }
    } while (ld_relaxed_u32(p) < target);
  }
  fence_acq_rel_gpu();
  return true;
}

template <int BX, int NS>
__global__ void __launch_bounds__(BX, 8) ens_run_kernel(const EnsRunArgs a) {
  const int tid = threadIdx.x;
  const int4 it = a.items[blockIdx.x];
  const int d = it.x;
  const EnsDomain &D = a.doms[d];
  const int4 lay = a.layout[d];
  const int rel = (int)blockIdx.x - lay.x;
  const int tx = rel % lay.y, zc = rel / lay.y;
  MarchArgs m = ens_march_args(D, it, &a.mapsA[d]);
  m.err = a.err;
  fused_barriers_init<D2Q9, ST_F32, BX, 1, NS>(m);
  if (tid == 0) {
    prefetch_tmap(&a.mapsB[d].main);
    prefetch_tmap(&a.mapsB[d].col);
  }
  // the item this thread watches between steps: chunk zc + dz, tile tx + dx,
  // dz and dx in -2..2 (periodic; repeats when a domain has few items)
  const uint32_t *watch = nullptr;
  if (tid < 25) {
    const int z2 = ((zc + tid / 5 - 2) % lay.z + lay.z) % lay.z;
    const int x2 = ((tx + tid % 5 - 2) % lay.y + lay.y) % lay.y;
    watch = a.flags + lay.x + z2 * lay.y + x2;
  }
  const int64_t ps = D.popstride;
  uint32_t kb = 0, done = 0;
  __shared__ int s_go;
  for (int k = 0; k < a.nint; ++k) {
    for (int t = 0; t < a.diag_every; ++t) {
      if (done > 0) {
        const bool ok = watch == nullptr || ens_wait_at_least(watch, done, a.err);
        if (!__syncthreads_and(ok)) return;
        // the neighbours' stores (generic proxy) before this CTA's bulk copies
        if (tid == 0) fence_proxy_async_global();
      }
      const int parity = t & 1;  // intervals have even length: A is the input at t = 0
      m.tm = parity ? &a.mapsB[d] : &a.mapsA[d];
      float *out = parity ? D.latA : D.latB;
      if (!fused_march<D2Q9, ST_F32, BX, 1, NS>(m, [&](int i) { return out + i * ps; }, kb))
        return;  // a copy timed out (reported in err; none is left in flight)
      ++done;
      __syncthreads();  // every thread's stores of this step precede the release
      if (tid == 0 && !(a.withhold && blockIdx.x == 0)) st_release_u32(a.flags + blockIdx.x, done);
    }
    if (rel == 0) {
      // the probe reads lattice A once the whole domain finished the step
      bool ok = true;
      for (int i = tid; i < lay.w && ok; i += BX)
        ok = ens_wait_at_least(a.flags + lay.x + i, done, a.err);
      if (!__syncthreads_and(ok)) return;
      const bool act = ens_probe_domain(D, &a.st[d], 0, a.diag_every, a.eps_arm, a.h_max);
      if (tid == 0) st_release_u32(a.pflag + d, (uint32_t)(k + 1));
      if (!act) return;
    } else {
      if (tid == 0)
        s_go = ens_wait_at_least(a.pflag + d, (uint32_t)(k + 1), a.err) ? __ldcg(&a.st[d].active)
                                                                        : 0;
      __syncthreads();
      if (!s_go) return;
    }
  }
}

// the persistent launch's tile (BX cells, NS stages)
constexpr int ENS_RUN_BX = 128, ENS_RUN_NS = 4;
using EnsRunK = FusedK<D2Q9, ST_F32, ENS_RUN_BX, 1, ENS_RUN_NS>;

template <int BX, int NS>
cudaError_t ens_prepare_t() {
  return cudaFuncSetAttribute(ens_step_kernel<BX, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              FusedK2<D2Q9, ST_F32, BX, 1, NS>::SMEM);
}
template <int BX, int NS>
cudaError_t ens_launch_t(int grid, const EnsDomain *doms, const FusedMaps *a, const FusedMaps *b,
                  const int4 *items, const int *count, const EnsState *st, int parity,
                  cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)(BX / 2));
  cfg.dynamicSmemBytes = (size_t)FusedK2<D2Q9, ST_F32, BX, 1, NS>::SMEM;
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
  int4 *d_items[NCLASS] = {};
  int *d_count[NCLASS] = {};
  int zlen = 16;  // rows per work item of the per-step launches' lists
  // current work-list sizes: the tile classes' and the temporally blocked one
  int cnt[NCLASS + 1] = {};
  int nsm = 152;
  double eps_arm = 0, h_max = 8;
  int diag_every = 100;
  int64_t steps = 0;
  double updates = 0;  // lattice updates performed
  int64_t launches = 0;
  // the captured interval of each launch form (key: rows per chunk of the
  // per-step launches, or 100 + the temporally blocked configuration),
  // replayed K times per launch; its grids cover the work lists it runs
  struct Captured {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    int grid[NCLASS + 1] = {};
  };
  std::map<int, Captured> graphs;
  // pinned staging of the work lists (asynchronous uploads; `staged` while
  // an upload from it may still be pending)
  int4 *h_stage = nullptr;
  int *h_cnt = nullptr;
  size_t stage_cap = 0;
  bool staged = false;
  size_t cap_items = 0, cap_tb = 0;  // work-list capacities (classes together, blocked)
  // pinned host copy of the domain states (a plain asynchronous read-back)
  EnsState *h_state = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;  // device time of a launch
  // persistent launch: CTAs that fit in one wave (0: unavailable), the
  // rows per item of the current work list (0: to be rebuilt), its items
  int pcap = 0, pz = 0, pitems = 0;
  bool persistent = false;  // the sweep moved to persistent launches
  int mode = LBM_ENS_AUTO;
  // temporally blocked intervals: the tile configuration (-1: one launch
  // per step and tile class), the work list and its captured grid
  int tb = -1;
  int tb_pref = 0;  // the configuration LBM_ENS_TEMPORAL runs
  // measured choice of the launch form (LBM_ENS_AUTO): the candidates of the
  // current measurement (x: temporally blocked configuration or -1, y: rows
  // per chunk of the per-step launches), their device time per lattice
  // update, the next one to time, and the active cells when it began
  int zforce = 0;  // rows per chunk of the per-step launches (0: the rule)
  std::vector<int2> trials;
  std::vector<double> trial_ns;
  size_t trial = 0;
  double tuned_cells = 0;
  int4 *d_tbitems = nullptr;
  int *d_tbcount = nullptr;
  bool failed = false;  // a bounded wait gave up: the domain states are invalid
  int4 *d_pitems = nullptr, *d_layout = nullptr;
  // TMA descriptors of every domain with the persistent tile's boxes (the
  // per-step launches' descriptors carry their tile class's box width)
  FusedMaps *d_pmapsA = nullptr, *d_pmapsB = nullptr;
  uint32_t *d_flags = nullptr, *d_pflag = nullptr;
  int *d_err = nullptr, *h_err = nullptr;
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
constexpr int ENS_ZLEN_MAX = 16, ENS_ZLEN_MIN = 1;
// With few domains left, a launch covers ENS_BATCH intervals: the host's
// per-interval round trip (graph launch, state copy, synchronisation) then
// comes once per ENS_BATCH probes.  A domain settled by one of the probes
// is skipped by the later steps of the launch, so it keeps the state of its
// settling probe, as with one interval per launch.
constexpr int ENS_BATCH = 10, ENS_BATCH_ACTIVE = 32;
// intervals of one persistent launch: domains settled by a probe of a
// launch leave their CTAs idle until the next launch rebuilds the work list
constexpr int ENS_PBATCH_RUN = 10;

int chunk_len(int ny, int zmax) {
  int zlen = std::min(ny, zmax);
  const int nzc = (ny + zlen - 1) / zlen;
  return (ny + nzc - 1) / nzc;
}

// Before the host writes the staging area: wait for the uploads from it.
lbm_status stage_ready(lbm_ensemble *E) {
  if (E->staged) ECK(cudaStreamSynchronize(E->s));
  E->staged = false;
  return LBM_OK;
}

// Work lists of the per-step launches (chunks of at most E->zlen rows) into
// d_items / d_count per class; sizes into E->cnt.
lbm_status build_items(lbm_ensemble *E) {
  ECKS(stage_ready(E));
  size_t off = 0;
  for (int c = 0; c < NCLASS; ++c) {
    int4 *it = E->h_stage + off;
    int k = 0;
    for (int d = 0; d < E->n; ++d) {
      if (E->cls[d] != c || !E->hstate[d].active) continue;
      const int bx = CLASS_BX[c];
      const int nx = E->hdom[d].NX, ny = E->hdom[d].NZ;
      const int tiles_x = (nx + bx - 1) / bx;
      const int zlen = chunk_len(ny, E->zlen);
      const int nzc = (ny + zlen - 1) / zlen;
      for (int zc = 0; zc < nzc; ++zc)
        for (int tx = 0; tx < tiles_x; ++tx)
          it[k++] = make_int4(d, tx * bx, zc * zlen, std::min(ny, (zc + 1) * zlen));
    }
    E->cnt[c] = E->h_cnt[c] = k;
    if (k > 0)
      ECK(cudaMemcpyAsync(E->d_items[c], it, sizeof(int4) * k, cudaMemcpyHostToDevice, E->s));
    ECK(cudaMemcpyAsync(E->d_count[c], E->h_cnt + c, sizeof(int), cudaMemcpyHostToDevice, E->s));
    off += (size_t)k;
  }
  E->staged = true;
  return LBM_OK;
}

// Work list of the temporally blocked launches: tiles of configuration cfg
// over the active domains, (domain, x0, z0, 0); size into E->cnt[NCLASS].
lbm_status build_tb_items(lbm_ensemble *E, int cfg) {
  ECKS(stage_ready(E));
  int k = 0;
  for (int d = 0; d < E->n; ++d) {
    if (!E->hstate[d].active) continue;
    const int nx = E->hdom[d].NX, ny = E->hdom[d].NZ;
    for (int z0 = 0; z0 < ny; z0 += TB_TZ[cfg])
      for (int x0 = 0; x0 < nx; x0 += TB_TX[cfg]) E->h_stage[k++] = make_int4(d, x0, z0, 0);
  }
  E->cnt[NCLASS] = E->h_cnt[NCLASS] = k;
  if (k > 0)
    ECK(cudaMemcpyAsync(E->d_tbitems, E->h_stage, sizeof(int4) * k, cudaMemcpyHostToDevice, E->s));
  ECK(cudaMemcpyAsync(E->d_tbcount, E->h_cnt + NCLASS, sizeof(int), cudaMemcpyHostToDevice, E->s));
  E->staged = true;
  return LBM_OK;
}

int count_items(const lbm_ensemble *E, int d, int c, int zmax) {
  const int bx = CLASS_BX[c];
  const int nx = E->hdom[d].NX, ny = E->hdom[d].NZ;
  const int zlen = chunk_len(ny, zmax);
  return ((nx + bx - 1) / bx) * ((ny + zlen - 1) / zlen);
}

// the longest chunk (16, 8, 4, 2, 1 rows) that still gives the active
// domains at least four CTAs per SM
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

void drop_graphs(lbm_ensemble *E) {
  for (auto &kv : E->graphs) {
    if (kv.second.x) cudaGraphExecDestroy(kv.second.x);
    if (kv.second.g) cudaGraphDestroy(kv.second.g);
  }
  E->graphs.clear();
}

// one diagnostic interval: diag_every steps of every active domain, then
// the probe, which advances each active domain's step counter
// grid: CTAs per tile class and of the temporally blocked launches (at
// least the work lists' sizes; the CTAs beyond a list return at once)
lbm_status enqueue_interval(lbm_ensemble *E, const int grid[NCLASS + 1]) {
  if (E->tb >= 0) {
    // diag_every / S temporally blocked launches, each reading one lattice
    // and writing the other (an even number: lattice A is current after it)
    const int L = E->diag_every / TB_S[E->tb];
    for (int j = 0; j < L; ++j)
      ECK(tb_launch(E->tb, grid[NCLASS], E->d_dom, E->d_tbitems, E->d_tbcount, E->d_state,
                    j & 1, E->s));
  } else {
    // fork: one chain of diag_every steps per tile class, joined before the probe
    ECK(cudaEventRecord(E->fork, E->s));
    for (int c = 0; c < NCLASS; ++c) {
      if (grid[c] == 0) continue;
      ECK(cudaStreamWaitEvent(E->side[c], E->fork, 0));
      for (int t = 0; t < E->diag_every; ++t)
        ECK(ens_launch(c, grid[c], E->d_dom, E->d_mapsA, E->d_mapsB, E->d_items[c],
                       E->d_count[c], E->d_state, t & 1, E->side[c]));
      ECK(cudaEventRecord(E->join[c], E->side[c]));
      ECK(cudaStreamWaitEvent(E->s, E->join[c], 0));
    }
  }
  k_ens_probe<<<E->n, 256, 0, E->s>>>(E->d_dom, E->d_state, E->n, 0, E->diag_every, E->eps_arm,
                                       E->h_max);
  ECK(cudaGetLastError());
  return LBM_OK;
}

// The captured interval of the current launch form, captured again when
// its grids no longer fit the work lists: a list larger than its grid, or
// smaller than half of it (stopped domains then stop costing CTAs), or a
// tile class that emptied or filled.  Returns the executable graph.
lbm_status ensure_graph(lbm_ensemble *E, cudaGraphExec_t *exec) {
  const int key = E->tb >= 0 ? 100 + E->tb : E->zlen;
  lbm_ensemble::Captured &c = E->graphs[key];
  bool fit = c.x != nullptr;
  for (int k = 0; k <= NCLASS && fit; ++k) {
    const bool used = E->tb >= 0 ? k == NCLASS : k < NCLASS;
    const int n = used ? E->cnt[k] : 0;
    fit = (n == 0) == (c.grid[k] == 0) && n <= c.grid[k] && 2 * n >= c.grid[k];
  }
  if (!fit) {
    if (c.x) cudaGraphExecDestroy(c.x);
    if (c.g) cudaGraphDestroy(c.g);
    c = lbm_ensemble::Captured();
    for (int k = 0; k <= NCLASS; ++k)
      c.grid[k] = (E->tb >= 0 ? k == NCLASS : k < NCLASS) ? E->cnt[k] : 0;
    ECK(cudaStreamBeginCapture(E->s, cudaStreamCaptureModeThreadLocal));
    const lbm_status st = enqueue_interval(E, c.grid);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(E->s, &g);
    if (st != LBM_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    ECK(e);
    c.g = g;
    ECK(cudaGraphInstantiate(&c.x, g, 0));
    ECK(cudaGraphUpload(c.x, E->s));  // not on the first launch's (timed) path
  }
  *exec = c.x;
  return LBM_OK;
}

// K intervals (the captured interval replayed K times, K = 1 or
// ENS_BATCH), then the domain states on the host.  A domain that a probe of
// this launch settled keeps the step counter it had there.  *ms (may be
// NULL) receives the device time of the K intervals.
lbm_status ens_interval(lbm_ensemble *E, int K, float *ms) {
  std::vector<char> was(E->n);
  for (int d = 0; d < E->n; ++d) was[d] = E->hstate[d].active != 0;
  cudaGraphExec_t x = nullptr;
  ECKS(ensure_graph(E, &x));
  if (ms) ECK(cudaEventRecord(E->t0, E->s));
  for (int k = 0; k < K; ++k) ECK(cudaGraphLaunch(x, E->s));
  if (ms) ECK(cudaEventRecord(E->t1, E->s));
  ECK(cudaMemcpyAsync(E->h_state, E->d_state, sizeof(EnsState) * E->n, cudaMemcpyDeviceToHost,
                      E->s));
  ECK(cudaStreamSynchronize(E->s));
  E->staged = false;
  if (ms) ECK(cudaEventElapsedTime(ms, E->t0, E->t1));
  std::copy(E->h_state, E->h_state + E->n, E->hstate.begin());
  const int64_t end = E->steps + (int64_t)K * E->diag_every;
  for (int d = 0; d < E->n; ++d) {
    if (!was[d]) continue;
    const EnsState &st = E->hstate[d];
    const int64_t ran = (st.active ? end : st.step) - E->steps;
    E->updates += (double)E->hdom[d].NX * E->hdom[d].NZ * (double)ran;
  }
  E->steps = end;
  int per = 0;  // launches of one interval before its probe
  if (E->tb >= 0) {
    per = E->diag_every / TB_S[E->tb];
  } else {
    for (int c = 0; c < NCLASS; ++c) per += E->cnt[c] > 0 ? E->diag_every : 0;
  }
  E->launches += (int64_t)K * (per + 1);
  return LBM_OK;
}

// Work list of the persistent launch: the active domains cut into tiles of
// ENS_RUN_BX columns and chunks of at most z rows, for the shortest z (most
// CTAs, shortest march per step) whose items fit in one wave.  Sets
// *fits = false when even 16-row chunks do not fit.
lbm_status build_pitems(lbm_ensemble *E, bool *fits) {
  *fits = false;
  if (E->pcap <= 0) return LBM_OK;
  int z = 1;
  for (;; ++z) {
    if (z > ENS_ZLEN_MAX) return LBM_OK;
    int64_t items = 0;
    for (int d = 0; d < E->n; ++d) {
      if (!E->hstate[d].active) continue;
      const int nx = E->hdom[d].NX, ny = E->hdom[d].NZ, zl = chunk_len(ny, z);
      items += (int64_t)((nx + ENS_RUN_BX - 1) / ENS_RUN_BX) * ((ny + zl - 1) / zl);
    }
    if (items <= E->pcap) break;
  }
  ECKS(stage_ready(E));
  int4 *it = E->h_stage, *lay = E->h_stage + E->pcap;  // items, then the layout
  int k = 0;
  for (int d = 0; d < E->n; ++d) {
    lay[d] = make_int4(0, 1, 1, 0);
    if (!E->hstate[d].active) continue;
    const int nx = E->hdom[d].NX, ny = E->hdom[d].NZ;
    const int tiles = (nx + ENS_RUN_BX - 1) / ENS_RUN_BX;
    const int zl = chunk_len(ny, z), nzc = (ny + zl - 1) / zl;
    lay[d] = make_int4(k, tiles, nzc, tiles * nzc);
    for (int zc = 0; zc < nzc; ++zc)
      for (int tx = 0; tx < tiles; ++tx)
        it[k++] = make_int4(d, tx * ENS_RUN_BX, zc * zl, std::min(ny, (zc + 1) * zl));
  }
  E->pitems = k;
  E->pz = z;
  if (k > 0)
    ECK(cudaMemcpyAsync(E->d_pitems, it, sizeof(int4) * k, cudaMemcpyHostToDevice, E->s));
  ECK(cudaMemcpyAsync(E->d_layout, lay, sizeof(int4) * E->n, cudaMemcpyHostToDevice, E->s));
  E->staged = true;
  *fits = true;
  return LBM_OK;
}

// K intervals in one persistent launch, then the domain states on the host
// (the same bookkeeping as ens_interval).
lbm_status ens_persistent(lbm_ensemble *E, int K) {
  std::vector<char> was(E->n);
  for (int d = 0; d < E->n; ++d) was[d] = E->hstate[d].active != 0;
  ECK(cudaMemsetAsync(E->d_flags, 0, sizeof(uint32_t) * E->pitems, E->s));
  ECK(cudaMemsetAsync(E->d_pflag, 0, sizeof(uint32_t) * E->n, E->s));
  ECK(cudaMemsetAsync(E->d_err, 0, sizeof(int), E->s));
  EnsRunArgs a;
  a.doms = E->d_dom;
  a.mapsA = E->d_pmapsA;
  a.mapsB = E->d_pmapsB;
  a.items = E->d_pitems;
  a.layout = E->d_layout;
  a.st = E->d_state;
  a.flags = E->d_flags;
  a.pflag = E->d_pflag;
  a.err = E->d_err;
  a.nint = K;
  a.diag_every = E->diag_every;
  a.eps_arm = E->eps_arm;
  a.h_max = E->h_max;
  a.withhold = E->mode == LBM_ENS_DEBUG_WITHHOLD_FLAG;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)E->pitems);
  cfg.blockDim = dim3((unsigned)ENS_RUN_BX);
  cfg.dynamicSmemBytes = (size_t)EnsRunK::SMEM;
  cfg.stream = E->s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident at once
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ECK(cudaLaunchKernelEx(&cfg, ens_run_kernel<ENS_RUN_BX, ENS_RUN_NS>, a));
  ECK(cudaMemcpyAsync(E->h_state, E->d_state, sizeof(EnsState) * E->n, cudaMemcpyDeviceToHost,
                      E->s));
  ECK(cudaMemcpyAsync(E->h_err, E->d_err, sizeof(int), cudaMemcpyDeviceToHost, E->s));
  ECK(cudaStreamSynchronize(E->s));
  E->staged = false;
  E->launches += 1;
  if (*E->h_err) {
    E->failed = true;
    return efail(LBM_ETIMEOUT, std::string("ensemble: persistent launch stopped (") +
                                (*E->h_err & ERR_SYNC_TIMEOUT ? "a wait for a neighbour timed out"
                                                               : "a bulk copy timed out") +
                                ")");
  }
  std::copy(E->h_state, E->h_state + E->n, E->hstate.begin());
  const int64_t end = E->steps + (int64_t)K * E->diag_every;
  for (int d = 0; d < E->n; ++d) {
    if (!was[d]) continue;
    const EnsState &st = E->hstate[d];
    const int64_t ran = (st.active ? end : st.step) - E->steps;
    E->updates += (double)E->hdom[d].NX * E->hdom[d].NZ * (double)ran;
  }
  E->steps = end;
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
  if (cudaEventCreate(&E->t0) != cudaSuccess || cudaEventCreate(&E->t1) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void **>(&E->h_state), sizeof(EnsState) * (size_t)n) !=
          cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void **>(&E->h_err), sizeof(int)) != cudaSuccess) {
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
  // work-list capacity per class: every domain could be moved to any class
  for (int c = 0; c < NCLASS; ++c) {
    int cap = 0;
    for (int d = 0; d < n; ++d) cap += count_items(E, d, c, ENS_ZLEN_MIN);
    E->cap_items += (size_t)cap;
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
  // temporally blocked launches: work-list capacity for the smallest tile
  {
    int64_t cap = 0;
    for (int c = 0; c < NTB; ++c) {
      int64_t t = 0;
      for (int d = 0; d < n; ++d)
        t += (int64_t)((E->hdom[d].NX + TB_TX[c] - 1) / TB_TX[c]) *
             ((E->hdom[d].NZ + TB_TZ[c] - 1) / TB_TZ[c]);
      cap = std::max(cap, t);
      if (tb_prepare(c) != cudaSuccess) {
        cudaGetLastError();
        return bail(efail(LBM_ECUDA, "ensemble: temporally blocked kernel set-up failed"));
      }
    }
    E->cap_tb = (size_t)cap;
    if ((st = ealloc(E, sizeof(int4) * cap, &p)) != LBM_OK) return bail(st);
    E->d_tbitems = static_cast<int4 *>(p);
    if ((st = ealloc(E, sizeof(int), &p)) != LBM_OK) return bail(st);
    E->d_tbcount = static_cast<int *>(p);
  }
  // the persistent launch: one wave of CTAs of its tile, where the device
  // supports cooperative launches (otherwise every interval is a graph)
  {
    int coop = 0, occ = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop &&
        cudaFuncSetAttribute(ens_run_kernel<ENS_RUN_BX, ENS_RUN_NS>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, EnsRunK::SMEM) ==
            cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &occ, ens_run_kernel<ENS_RUN_BX, ENS_RUN_NS>, ENS_RUN_BX, EnsRunK::SMEM) ==
            cudaSuccess)
      E->pcap = occ * E->nsm;
    cudaGetLastError();
  }
  if (E->pcap > 0) {
    if ((st = ealloc(E, sizeof(int4) * E->pcap, &p)) != LBM_OK) return bail(st);
    E->d_pitems = static_cast<int4 *>(p);
    if ((st = ealloc(E, sizeof(uint32_t) * E->pcap, &p)) != LBM_OK) return bail(st);
    E->d_flags = static_cast<uint32_t *>(p);
    if ((st = ealloc(E, sizeof(int4) * n, &p)) != LBM_OK) return bail(st);
    E->d_layout = static_cast<int4 *>(p);
    if ((st = ealloc(E, sizeof(uint32_t) * n, &p)) != LBM_OK) return bail(st);
    E->d_pflag = static_cast<uint32_t *>(p);
    if ((st = ealloc(E, sizeof(int), &p)) != LBM_OK) return bail(st);
    E->d_err = static_cast<int *>(p);
    if ((st = ealloc(E, sizeof(FusedMaps) * n, &p)) != LBM_OK) return bail(st);
    E->d_pmapsA = static_cast<FusedMaps *>(p);
    if ((st = ealloc(E, sizeof(FusedMaps) * n, &p)) != LBM_OK) return bail(st);
    E->d_pmapsB = static_cast<FusedMaps *>(p);
    std::vector<FusedMaps> pa(n), pb(n);
    bool enc_ok = true;
    for (int d = 0; d < n && enc_ok; ++d) {
      const EnsDomain &D = E->hdom[d];
      FusedPlan pl;
      enc_ok = fused_make_plan(D2Q9, ST_F32, class_tile_id(1), D.NX, 1, D.NZ, 1, &pl) ==
                   cudaSuccess &&
               pl.bx == ENS_RUN_BX && pl.by == 1 && pl.xc == 1 && pl.nstage == ENS_RUN_NS &&
               fused_encode_maps(D2Q9, ST_F32, pl, D.latA, D.NX, 1, D.NZ, D.px, &pa[d]) ==
                   CUDA_SUCCESS &&
               fused_encode_maps(D2Q9, ST_F32, pl, D.latB, D.NX, 1, D.NZ, D.px, &pb[d]) ==
                   CUDA_SUCCESS;
    }
    cudaGetLastError();
    if (!enc_ok) {
      E->pcap = 0;  // no persistent launches: every interval is a graph
    } else if (cudaMemcpyAsync(E->d_pmapsA, pa.data(), sizeof(FusedMaps) * n,
                               cudaMemcpyHostToDevice, E->s) != cudaSuccess ||
               cudaMemcpyAsync(E->d_pmapsB, pb.data(), sizeof(FusedMaps) * n,
                               cudaMemcpyHostToDevice, E->s) != cudaSuccess ||
               cudaStreamSynchronize(E->s) != cudaSuccess) {
      cudaGetLastError();
      return bail(efail(LBM_ECUDA, "ensemble: upload failed"));
    }
  }
  // pinned staging of the work lists: the largest of the classes' lists
  // together, the temporally blocked list and the persistent one with its
  // layout
  E->stage_cap = std::max(E->cap_items, std::max(E->cap_tb, (size_t)E->pcap + (size_t)n));
  if (cudaMallocHost(reinterpret_cast<void **>(&E->h_stage), sizeof(int4) * E->stage_cap) !=
          cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void **>(&E->h_cnt), sizeof(int) * (NCLASS + 1)) !=
          cudaSuccess) {
    cudaGetLastError();
    return bail(efail(LBM_ENOMEM, "ensemble: pinned host allocation failed"));
  }
  E->zlen = choose_zlen(E);
  if ((st = build_items(E)) != LBM_OK) return bail(st);
  *out = E;
  return LBM_OK;
}

void lbm_ensemble_destroy(lbm_ensemble *E) {
  if (!E) return;
  if (E->s) cudaStreamSynchronize(E->s);
  drop_graphs(E);
  efree_all(E);
  for (int c = 0; c < NCLASS; ++c) {
    if (E->side[c]) cudaStreamDestroy(E->side[c]);
    if (E->join[c]) cudaEventDestroy(E->join[c]);
  }
  if (E->fork) cudaEventDestroy(E->fork);
  if (E->s) cudaStreamDestroy(E->s);
  if (E->t0) cudaEventDestroy(E->t0);
  if (E->t1) cudaEventDestroy(E->t1);
  if (E->h_state) cudaFreeHost(E->h_state);
  if (E->h_err) cudaFreeHost(E->h_err);
  if (E->h_stage) cudaFreeHost(E->h_stage);
  if (E->h_cnt) cudaFreeHost(E->h_cnt);
  cudaGetLastError();
  delete E;
}

// After the active set or the launch form changed: the current form's work
// lists (the captured intervals are checked against them before a launch).
static lbm_status refresh_work(lbm_ensemble *E) {
  if (E->tb >= 0) return build_tb_items(E, E->tb);
  E->zlen = E->zforce > 0 ? E->zforce : choose_zlen(E);
  return build_items(E);
}

// Switch the interval's steps to temporally blocked launches of
// configuration cfg (-1: back to one launch per step and tile class).
static lbm_status set_tb(lbm_ensemble *E, int cfg) {
  if (cfg == E->tb) return LBM_OK;
  E->tb = cfg;
  return refresh_work(E);
}

// ---- measured choice of the launch form (LBM_ENS_AUTO) ----------------------
// With many active cells the steps are bound by memory bandwidth and the
// per-step launches with the rule's long chunks are the fastest form.  Below
// ENS_TUNE_CELLS they become latency-bound and the fastest form depends on
// the active set (measured on the 256-domain sweep: 6-row chunks at 10
// domains, 16 x 16 temporally blocked tiles at 6, 32 x 16 tiles for one
// domain).  There the candidates are timed on the sweep itself, one
// interval each, whenever the active cells fell below ENS_RETUNE of those
// of the last measurement; the fastest per lattice update is kept.  Every
// form gives the same populations, so a trial is ordinary work.
constexpr double ENS_TUNE_CELLS = 3.0e6, ENS_RETUNE = 0.75, ENS_TB_CELLS = 4.0e5;

static double active_cells(const lbm_ensemble *E) {
  double c = 0;
  for (int d = 0; d < E->n; ++d)
    if (E->hstate[d].active) c += (double)E->hdom[d].NX * E->hdom[d].NZ;
  return c;
}

// tb >= 0: temporally blocked configuration tb; else per-step launches with
// chunks of z rows (0: the rule)
static lbm_status apply_form(lbm_ensemble *E, int tb, int z) {
  if (tb >= 0) return set_tb(E, tb);
  if (E->tb < 0 && E->zforce == z) return LBM_OK;
  E->tb = -1;
  E->zforce = z;
  return refresh_work(E);
}

// The next interval's launch form; *measure when that interval is a trial.
static lbm_status auto_form(lbm_ensemble *E, bool *measure) {
  *measure = false;
  if (E->trial < E->trials.size()) {
    *measure = true;
    return apply_form(E, E->trials[E->trial].x, E->trials[E->trial].y);
  }
  const double cells = active_cells(E);
  if (cells > ENS_TUNE_CELLS) return apply_form(E, -1, 0);
  if (E->tuned_cells > 0 && cells > ENS_RETUNE * E->tuned_cells) return LBM_OK;
  // a new measurement: chunk lengths around the rule's, and the
  // temporally blocked tiles once few cells are active
  E->tuned_cells = cells;
  E->trials.clear();
  E->trial_ns.clear();
  E->trial = 0;
  const int zr = choose_zlen(E);
  for (int z : {1, 2, 3, 4, 6, 8, 12, 16})
    if (2 * z >= zr && z <= 2 * zr) E->trials.push_back(make_int2(-1, z));
  if (cells <= ENS_TB_CELLS)
    for (int c : {0, 1, 3})
      if (E->diag_every % (2 * TB_S[c]) == 0) E->trials.push_back(make_int2(c, 0));
  *measure = true;
  return apply_form(E, E->trials[0].x, E->trials[0].y);
}

static lbm_status auto_record(lbm_ensemble *E, float ms, double updates) {
  E->trial_ns.push_back(updates > 0 ? 1e6 * (double)ms / updates : 1e300);
  if (++E->trial < E->trials.size()) return LBM_OK;
  size_t b = 0;
  for (size_t i = 1; i < E->trial_ns.size(); ++i)
    if (E->trial_ns[i] < E->trial_ns[b]) b = i;
  return apply_form(E, E->trials[b].x, E->trials[b].y);
}

lbm_status lbm_ensemble_run(lbm_ensemble *E, int64_t max_steps, int64_t *steps_done) {
  if (!E) return efail(LBM_EINVAL, "ensemble is NULL");
  if (max_steps < 0) return efail(LBM_EINVAL, "max_steps < 0");
  if (E->failed) return efail(LBM_ETIMEOUT, "ensemble: an earlier launch timed out");
  const int64_t start = E->steps;
  while (E->steps - start < max_steps) {
    int active = 0;
    for (int d = 0; d < E->n; ++d) active += E->hstate[d].active;
    if (!active) break;
    std::vector<int32_t> before(E->n);
    for (int d = 0; d < E->n; ++d) before[d] = E->hstate[d].active;
    const int64_t left = max_steps - (E->steps - start);
    // persistent launches once the active work fits in one wave (the
    // active set only shrinks, so the sweep stays there)
    bool fits = false;
    if (E->mode == LBM_ENS_PERSISTENT || E->mode == LBM_ENS_DEBUG_WITHHOLD_FLAG) {
      fits = E->persistent && E->pz > 0;
      if (!fits && E->pcap > 0) ECKS(build_pitems(E, &fits));
    }
    if (!fits && E->mode == LBM_ENS_TEMPORAL && E->tb != E->tb_pref &&
        E->diag_every % (2 * TB_S[E->tb_pref]) == 0)
      ECKS(set_tb(E, E->tb_pref));
    if (fits) {
      E->persistent = true;
      const int64_t ki = left / E->diag_every;
      ECKS(ens_persistent(E, (int)std::max<int64_t>(1, std::min<int64_t>(ENS_PBATCH_RUN, ki))));
    } else {
      bool measure = false;
      if (E->mode == LBM_ENS_AUTO) ECKS(auto_form(E, &measure));
      const int K = !measure && active <= ENS_BATCH_ACTIVE &&
                            left >= (int64_t)ENS_BATCH * E->diag_every
                        ? ENS_BATCH
                        : 1;
      float ms = 0;
      const double u0 = E->updates;
      ECKS(ens_interval(E, K, measure ? &ms : nullptr));
      if (measure) ECKS(auto_record(E, ms, E->updates - u0));
    }
    bool changed = false;
    for (int d = 0; d < E->n; ++d) changed |= before[d] != E->hstate[d].active;
    if (changed) {
      E->pz = 0;
      if (!E->persistent) ECKS(refresh_work(E));
    }
  }
  if (steps_done) *steps_done = E->steps - start;
  return LBM_OK;
}

lbm_status lbm_ensemble_set_launch(lbm_ensemble *E, int32_t mode) {
  if (!E) return efail(LBM_EINVAL, "ensemble is NULL");
  if (mode < LBM_ENS_AUTO || mode > LBM_ENS_TEMPORAL)
    return efail(LBM_EINVAL, "unknown launch mode");
  if (E->failed) return efail(LBM_ETIMEOUT, "ensemble: an earlier launch timed out");
  E->mode = mode;
  if (E->persistent && mode != LBM_ENS_PERSISTENT && mode != LBM_ENS_DEBUG_WITHHOLD_FLAG) {
    // back to per-step launches: their work lists follow the active set again
    E->persistent = false;
    E->pz = 0;
    ECKS(refresh_work(E));
  }
  if (mode != LBM_ENS_AUTO) {
    // a fixed form: no measurement, the rule's chunks or the blocked tiles
    E->trials.clear();
    E->trial_ns.clear();
    E->trial = 0;
    E->tuned_cells = 0;
    if (mode != LBM_ENS_TEMPORAL && !E->persistent) ECKS(apply_form(E, -1, 0));
  }
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
