// Internal interfaces between the translation units of the library.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm.h"

namespace sclbm {

// store a message for lbm_last_error() and return st
lbm_status set_error(lbm_status st, const char *msg);

// Everything a step kernel needs.  Cells are addressed in the kernels'
// three-dimensional view (D2Q9 on (nx, 1, ny)); the population arrays are
// f[i][z][y][x] with a row pitch px >= NX (elements), planes of px*NY and
// population blocks of px*NY*NZ.  fin holds f_i(x, t) at x (push form: the
// populations that have arrived), fout receives f_i(x, t+1).
struct StepArgs {
  const void *fin;
  void *fout;
  int64_t NX, NY, NZ, px;
  double tau, G, rho0, rho_ref;
  // the same constants in FP32 (the FP32-arithmetic kernels use no FP64)
  float tau_f, omega_f, G_f, rho0_f, inv_rho0_f, rho_ref_f;
  // base of every population block of fout (push destinations)
  void *out_pop[19];
  // injection (virtual blowing agent); nsites == 0 disables it
  int32_t nsites;
  const int32_t *site_x, *site_y, *site_z;  // view coordinates per site
  const double *rate;
  double *budget;
  // sites grouped by cell (site order inside a group) for the two-pass
  // injection kernel: group g holds group_site[group_off[g] .. group_off[g+1])
  int32_t ngroups;
  const int32_t *group_off;
  const int32_t *group_site;
  // per work item lists of sites, sorted by (z, site), for the fused kernel
  const int32_t *bucket_off;
  const int32_t *bucket_site;
  int *err;  // device status word (ERR_* bits)
  int debug_flags;  // LBM_DEBUG_* bits of the configuration
  // 16-bit storage with the rounding residual (kernel forms ST_F16R /
  // ST_BF16R): one FP32 per cell, indexed like population 0 (row pitch px);
  // NULL otherwise
  float *resid;
};

// TMA descriptors of one population lattice for the fused kernel: the
// column box, the left/right halo-column box, the top/bottom halo-row box and
// the corner box (all over the 4-D tensor x, y, z, population)
struct FusedMaps {
  CUtensorMap main, col, row, crn;
};

// fused-kernel launch plan
struct FusedPlan {
  int tile;      // tile id (see fused_tile_shape)
  int bx, by;    // interior tile of one CTA
  int nstage;    // TMA pipeline depth
  int tiles_x, tiles_y, nzc, zlen;
  int items;     // tiles_x * tiles_y * nzc CTAs
  int threads;
  int smem;      // dynamic shared memory bytes
  int hx;        // halo columns per box (16 bytes of elements)
  int xc;        // cells per thread along x: 1, or 2 for the x-pair kernel
};

// Tile shapes: returns false when the id is unknown for the lattice and
// storage.  *xc (may be NULL) receives the cells per thread along x.
bool fused_tile_shape(int lat, int st, int tile, int *bx, int *by, int *nstage,
                      int *xc = nullptr);
// Fill *plan for a lattice.  nzc > 0: that many z chunks; 0: the number
// with the fewest staged planes per resident CTA slot when the CTAs run in
// waves of SMs x CTAs per SM; -1: as many as fill those slots once.  Returns
// cudaErrorInvalidValue when the tile does not fit or nx is not a multiple
// of the 16-byte halo width.
cudaError_t fused_make_plan(int lat, int st, int tile, int64_t NX, int64_t NY, int64_t NZ,
                            int nzc, FusedPlan *plan);
// Encode the TMA descriptors of one population lattice for a plan.
CUresult fused_encode_maps(int lat, int st, const FusedPlan &plan, const void *base,
                           int64_t NX, int64_t NY, int64_t NZ, int64_t px, FusedMaps *tm);
cudaError_t fused_launch(int lat, int st, const FusedPlan &plan, const StepArgs &a,
                         const FusedMaps &tm_in, cudaStream_t s);
// work item (CTA) owning a view cell, for the injection buckets
int fused_item_of(const FusedPlan &plan, int64_t x, int64_t y, int64_t z);

// per-storage entry points (one translation unit each)
cudaError_t fused_launch_f64(int lat, const FusedPlan &, const StepArgs &, const FusedMaps &,
                             cudaStream_t);
cudaError_t fused_launch_f32(int lat, const FusedPlan &, const StepArgs &, const FusedMaps &,
                             cudaStream_t);
cudaError_t fused_launch_h16(int lat, int st, const FusedPlan &, const StepArgs &,
                             const FusedMaps &, cudaStream_t);
int fused_smem_f64(int lat, int tile);
int fused_smem_f32(int lat, int tile);
int fused_smem_h16(int lat, int st, int tile);
// set the kernel's shared-memory attribute; blocks_per_sm (may be NULL)
// receives the number of CTAs of the plan's kernel resident per SM
cudaError_t fused_prepare(int lat, int st, const FusedPlan &plan, int *blocks_per_sm = nullptr);
cudaError_t fused_prepare_f64(int lat, const FusedPlan &, int *blocks_per_sm);
cudaError_t fused_prepare_f32(int lat, const FusedPlan &, int *blocks_per_sm);
cudaError_t fused_prepare_h16(int lat, int st, const FusedPlan &, int *blocks_per_sm);
// x-pair kernels (FP32, FP16, BF16 storage; one translation unit each)
cudaError_t fused_x2_launch_f32(int lat, const FusedPlan &, const StepArgs &, const FusedMaps &,
                                cudaStream_t);
cudaError_t fused_x2_launch_f16(int lat, const FusedPlan &, const StepArgs &, const FusedMaps &,
                                cudaStream_t);
cudaError_t fused_x2_launch_bf16(int lat, const FusedPlan &, const StepArgs &,
                                 const FusedMaps &, cudaStream_t);
cudaError_t fused_x2_prepare_f32(int lat, const FusedPlan &, int *blocks_per_sm);
// the same kernels for the residual forms ST_F16R / ST_BF16R
cudaError_t fused_launch_h16r(int lat, int st, const FusedPlan &, const StepArgs &,
                              const FusedMaps &, cudaStream_t);
cudaError_t fused_prepare_h16r(int lat, int st, const FusedPlan &, int *blocks_per_sm);
cudaError_t fused_x2_launch_h16r(int lat, int st, const FusedPlan &, const StepArgs &,
                                 const FusedMaps &, cudaStream_t);
cudaError_t fused_x2_prepare_h16r(int lat, int st, const FusedPlan &, int *blocks_per_sm);
cudaError_t fused_x2_prepare_f16(int lat, const FusedPlan &, int *blocks_per_sm);
cudaError_t fused_x2_prepare_bf16(int lat, const FusedPlan &, int *blocks_per_sm);
int fused_x2_smem_f32(int lat, int tile);
int fused_x2_smem_f16(int lat, int tile);
int fused_x2_smem_bf16(int lat, int tile);

// two-pass path: psi field pass, then collide/stream (+ injection kernel)
cudaError_t twopass_launch(int lat, int st, const StepArgs &a, void *psi_scratch, cudaStream_t s);

// ---- diagnostics / state kernels (diag.cu) --------------------------------
// n / d for every 32-bit n with one multiply-high and two shifts: division
// by an invariant integer (Granlund and Montgomery, PLDI 1994, Fig. 4.1).
// The kernels' runtime 32-bit divisions otherwise run as a sequence on the
// FP64 pipe, which is narrow on this part.  m = 0: not prepared.
struct FastDiv {
  uint32_t m = 0;
  int s1 = 0, s2 = 0;
};
inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  int l = 0;
  while ((uint64_t(1) << l) < d) ++l;
  // d < 2^31, so 2^32 (2^l - d) < 2^63 and m < 2^32
  f.m = (uint32_t)(((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1);
  f.s1 = l < 1 ? l : 1;
  f.s2 = l - f.s1;
  return f;
}

struct View {
  int lat, st;
  int64_t NX, NY, NZ, px;
  double rho_ref;
  FastDiv fx, fy;  // division by NX and by NY (view_prepare)
  // per-cell FP32 rounding residual of the 16-bit storages (NULL: none):
  // part of population 0's value, indexed like it
  const float *resid = nullptr;
};
inline void view_prepare(View &v) {
  v.fx = make_fastdiv((uint32_t)v.NX);
  v.fy = make_fastdiv((uint32_t)v.NY);
}
#ifdef __CUDACC__
__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv &f, uint32_t d) {
  if (f.m == 0) return n / d;  // a view that was not prepared
  const uint32_t t = __umulhi(f.m, n);
  return (t + ((n - t) >> f.s1)) >> f.s2;
}
// A grid-stride pass over the N cells of an int32 array A, four cells per
// iteration from one 16-byte load: f(k, A[k]) for every cell, in increasing
// k within a thread.  Four times the bytes in flight of a one-cell loop.  A
// may be written during the pass only where f's decision does not depend on
// the timing (the sign of a label).  An A not on a 16-byte boundary (a
// caller's allocator) takes one cell per iteration.
template <class F>
__device__ __forceinline__ void quad_pass(int64_t N, const int32_t *A, F f) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (reinterpret_cast<uintptr_t>(A) & 15) {
    for (int64_t k = t; k < N; k += stride) f(k, A[k]);
    return;
  }
  const int64_t nq = N >> 2;
  const int4 *A4 = reinterpret_cast<const int4 *>(A);
  for (int64_t q = t; q < nq; q += stride) {
    const int4 a = A4[q];
    f(4 * q, a.x);
    f(4 * q + 1, a.y);
    f(4 * q + 2, a.z);
    f(4 * q + 3, a.w);
  }
  const int64_t k = 4 * nq + t;  // the last N mod 4 cells
  if (k < N) f(k, A[k]);
}
#endif
// initial density field (doubles, N) from bubbles (view coordinates, x y z r)
cudaError_t diag_init_rho(const View &v, const double *bub, int32_t nb, double rho_l,
                          double rho_g, double width, double noise_amp, uint64_t seed,
                          double *rho, cudaStream_t s);
// stored populations from canonical f_i(x) (doubles, Q*N), or from rho at rest
cudaError_t diag_store_from_f(const View &v, const double *f, void *stored, cudaStream_t s);
cudaError_t diag_store_from_rho(const View &v, const double *rho, void *stored, cudaStream_t s);
// one population f_i (N doubles) from / into stored populations
cudaError_t diag_gather_pop(const View &v, const void *stored, int i, double *out, cudaStream_t s);
cudaError_t diag_store_pop(const View &v, const double *f, int i, void *stored, cudaStream_t s);
// canonical f_i(x) (doubles, Q*N) from stored populations
cudaError_t diag_gather_f(const View &v, const void *stored, double *f, cudaStream_t s);
// FP64 moments: any output may be null; sets ERR_NONFINITE in err
cudaError_t diag_moments(const View &v, const void *stored, double G, double rho0, double *rho,
                         double *jx, double *jy, double *jz, double *psi, double *p, int *err,
                         cudaStream_t s);
// physical velocity (j + F/2)/rho from rho, j and psi fields
cudaError_t diag_velocity(const View &v, double G, const double *rho, const double *jx,
                          const double *jy, const double *jz, const double *psi, double *u,
                          cudaStream_t s);
cudaError_t diag_laplacian(const View &v, const double *p, double *lap, cudaStream_t s);
cudaError_t diag_line_d2(const View &v, const double *p, int64_t x0, int64_t y0, int64_t z0,
                         int axis, int64_t len, double *out, cudaStream_t s);
// FP64 totals (M, Jx, Jy, Jz) in user axes; partials must hold 4*diag_totals_blocks() doubles
int diag_totals_blocks();
cudaError_t diag_totals(const View &v, const void *stored, double *partials, double *out4,
                        cudaStream_t s);
// One pass over the populations of an FP32-arithmetic storage: gas labels
// initialised from rho < thr (labels may be null) and the totals (partials:
// 4*diag_scan_blocks() doubles; out4 may be null).  Not for LBM_F64.
int diag_scan_blocks();
cudaError_t diag_scan(const View &v, const void *stored, double thr, int32_t *labels,
                      double *partials, double *out4, int *err, cudaStream_t s);
// union-find linking and compression of initialised labels
cudaError_t diag_label_links(const View &v, int32_t *labels, unsigned long long *ncomp_dev,
                             cudaStream_t s);
// connected components of rho < thr; labels N int32; count -> *ncomp_dev (int64)
cudaError_t diag_label(const View &v, const double *rho, double thr, int32_t *labels,
                       unsigned long long *ncomp_dev, cudaStream_t s);
// film probe along a line (view coordinates, directions e and ep); out: 6 doubles
cudaError_t diag_film_probe(const View &v, const double *rho, const double *p, int64_t x0,
                            int64_t y0, int64_t z0, const int e[3], const int ep[3], int64_t len,
                            double mid, double *out, cudaStream_t s);
cudaError_t diag_gather_labels(const int32_t *labels, const int32_t *cells, int32_t n,
                               int32_t *out, cudaStream_t s);
// bubble census (census.cu): component sizes from labels (count_scratch: N
// int32), unordered (root, size) entries up to cap, *n_dev = components,
// hist[nbins] = log2 size histogram
cudaError_t diag_bubble_sizes(const View &v, const int32_t *labels, int32_t *count_scratch,
                              unsigned long long *n_dev, int64_t cap, int64_t *roots,
                              int64_t *sizes, int nbins, unsigned long long *hist,
                              cudaStream_t s);
// film test at every lattice point on the stored populations (FP64 pressure
// of the midpoints computed on demand): counts[5] = {film, midpoints, armed,
// fired, midpoint records}; records (film_record_bytes() each, unordered)
// up to cap: the fired (cell, axis) pairs, or with all_mid every midpoint
// (axis | fired << 8)
// blowing agent spread over each site's bubble (inject.cu): cells per gas
// root; then, after a step, take dm from the grouped sites (groups[g] =
// {bubble label or -1, first, end into gsites, cell of a liquid group}) and
// add w_i dm / n to the bubble's cells (dep: N doubles, per label)
cudaError_t inject_component_sizes(const View &v, const int32_t *labels, int32_t *count,
                                   cudaStream_t s);
cudaError_t inject_spread(const View &v, int ngroups, const int4 *groups, const int32_t *gsites,
                          const double *rate, double *budget, const int32_t *count, double *dep,
                          const int32_t *labels, bool any_bubble, void *lattice, cudaStream_t s);
size_t film_record_bytes();
// A queued film midpoint: cell, the labels on its two sides, and
// meta = user axis | old arming bit << 2 | run length << 3.
struct FilmMid {
  int64_t cell;
  int32_t label_minus, label_plus;
  int32_t meta, pad;
};
// counters of a film pass: film, midpoints, armed, fired, midpoint record
// slots, queued midpoints
constexpr int FILM_COUNT_SLOTS = 6;
// The film test at every lattice point, arming state updated in place.
// mids (capacity mid_cap) queues midpoints for the line walks (h_max <= 63);
// NULL selects the per-cell kernel.
cudaError_t diag_film_cells(const View &v, const int32_t *labels, const void *stored, double G,
                            double rho0, int h_max, double eps_arm, uint8_t *state,
                            unsigned long long *counts, int64_t cap, void *records,
                            bool all_mid, FilmMid *mids, int64_t mid_cap, cudaStream_t s);

}  // namespace sclbm
