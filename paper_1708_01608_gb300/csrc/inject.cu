// Blowing agent spread over each site's bubble (Sec. 3: gas is added to each
// bubble every step until the agent is used up), the alternative to the
// deposit at the site cell that the step kernels make.  The sites are
// grouped on the host: all sites whose cell lies in one bubble (gas label L
// at the start of the lbm_step call) form one group, and a site whose cell
// is liquid forms a group of that cell.  After each step:
//   k_spread_take   one thread per group: its sites, in increasing order,
//                   take dm = min(rate, budget) from their FP64 budgets; a
//                   bubble group's total divided by the bubble's cells is
//                   its deposit per cell, a cell group's total goes to its
//                   cell;
//   k_spread_apply  one thread per cell: a gas cell of a bubble with a
//                   deposit d gets w_i d on every population.
// Deposits land on the post-streaming populations (zero momentum).  FP64 and
// FP32 storage only: a deposit per cell is far below a 16-bit offset's
// resolution.
#include "internal.h"
#include "lattice.cuh"

namespace sclbm {
namespace {

constexpr int TPB = 256;

template <int ST>
__device__ __forceinline__ void add_w(void *lat, int64_t pop, int64_t o, double w, double d) {
  if constexpr (ST == ST_F64) {
    static_cast<double *>(lat)[o] += w * d;
  } else {
    static_cast<float *>(lat)[o] += (float)(w * d);
  }
  (void)pop;
}

template <int LAT, int ST>
__global__ void k_spread_take(View v, int ngroups, const int4 *groups, const int32_t *gsites,
                              const double *rate, double *budget, const int32_t *count,
                              double *dep, void *lat) {
  using L = Lattice<LAT>;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ngroups) return;
  const int4 G = groups[g];  // {label or -1, first site, end, cell of a liquid group}
  double sum = 0.0;
  for (int q = G.y; q < G.z; ++q) {
    const int s = gsites[q];
    const double d = fmin(rate[s], budget[s]);
    budget[s] -= d;
    sum += d;
  }
  if (G.x >= 0) {
    dep[G.x] = sum / (double)count[G.x];
  } else {
    const int64_t k = G.w;
    const int64_t x = k % v.NX, yz = k / v.NX, y = yz % v.NY, z = yz / v.NY;
    const int64_t pop = v.px * v.NY * v.NZ, o = (z * v.NY + y) * v.px + x;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) add_w<ST>(lat, pop, i * pop + o, L::w(i), sum);
  }
}

template <int LAT, int ST>
__global__ void __launch_bounds__(TPB)
    k_spread_apply(View v, const int32_t *labels, const double *dep, void *lat) {
  using L = Lattice<LAT>;
  const int64_t N = v.NX * v.NY * v.NZ, pop = v.px * v.NY * v.NZ;
  for (int64_t k = blockIdx.x * (int64_t)TPB + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * TPB) {
    const int32_t lab = labels[k];
    if (lab < 0) continue;
    const double d = dep[lab];
    if (d == 0.0) continue;
    // cell coordinates with the view's invariant-integer divisors
    const uint32_t kk = (uint32_t)k, nx = (uint32_t)v.NX, ny = (uint32_t)v.NY;
    const uint32_t yz = fdiv(kk, v.fx, nx), z = fdiv(yz, v.fy, ny);
    const int64_t x = kk - yz * nx, y = yz - z * ny;
    const int64_t o = ((int64_t)z * v.NY + y) * v.px + x;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) add_w<ST>(lat, pop, i * pop + o, L::w(i), d);
  }
}

__global__ void k_component_count(int64_t N, const int32_t *labels, int32_t *count) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t l = labels[k];
    const unsigned peers = __match_any_sync(__activemask(), l);
    if (l >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&count[l], __popc(peers));
  }
}

inline int grid_for(int64_t n) {
  const int64_t b = (n + TPB - 1) / TPB;
  return (int)(b < 1 ? 1 : (b > 65536 ? 65536 : b));
}

template <class Fn>
cudaError_t dispatch_spread(const View &v, Fn &&fn) {
  using D3 = std::integral_constant<int, D3Q19>;
  using D2 = std::integral_constant<int, D2Q9>;
  using F64 = std::integral_constant<int, ST_F64>;
  using F32 = std::integral_constant<int, ST_F32>;
  if (v.st != ST_F64 && v.st != ST_F32) return cudaErrorInvalidValue;
  if (v.lat == D3Q19) {
    if (v.st == ST_F64) fn(D3{}, F64{}); else fn(D3{}, F32{});
  } else {
    if (v.st == ST_F64) fn(D2{}, F64{}); else fn(D2{}, F32{});
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t inject_component_sizes(const View &v, const int32_t *labels, int32_t *count,
                                   cudaStream_t s) {
  const int64_t N = v.NX * v.NY * v.NZ;
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int32_t) * N, s);
  if (e != cudaSuccess) return e;
  k_component_count<<<grid_for(N), TPB, 0, s>>>(N, labels, count);
  return cudaGetLastError();
}

cudaError_t inject_spread(const View &v, int ngroups, const int4 *groups, const int32_t *gsites,
                          const double *rate, double *budget, const int32_t *count, double *dep,
                          const int32_t *labels, bool any_bubble, void *lattice, cudaStream_t s) {
  return dispatch_spread(v, [&](auto L, auto S) {
    constexpr int LAT = decltype(L)::value, ST = decltype(S)::value;
    if (ngroups > 0)
      k_spread_take<LAT, ST><<<(ngroups + 127) / 128, 128, 0, s>>>(v, ngroups, groups, gsites,
                                                                  rate, budget, count, dep, lattice);
    // the pass over the cells only when a site lies in a bubble
    if (any_bubble)
      k_spread_apply<LAT, ST><<<grid_for(v.NX * v.NY * v.NZ), TPB, 0, s>>>(v, labels, dep,
                                                                            lattice);
  });
}

}  // namespace sclbm
