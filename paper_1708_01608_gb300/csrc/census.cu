// Bubble census (Sec. 4): component sizes from the gas labels of the
// labelling kernels (label = smallest linear index of the component, -1 for
// liquid), listed per component, with a log2 size histogram.
#include "internal.h"

namespace sclbm {

namespace {

constexpr int TPB = 256;
inline int grid_of(int64_t n) {
  const int64_t b = (n + TPB - 1) / TPB;
  return (int)(b < 1 ? 1 : (b > 262144 ? 262144 : b));
}

// ---- bubble sizes -----------------------------------------------------------
// Cells per root.  A warp reads 128 consecutive cells of a row, four per
// lane; in each of four rounds its lanes hold cells four apart, which inside
// a bubble share one label: the lanes of equal labels add their number once,
// so that a large bubble does not serialise on one counter.
__global__ void k_size_count(int64_t N, const int32_t *labels, int32_t *count) {
  quad_pass(N, labels, [&](int64_t, int32_t l) {
    const unsigned peers = __match_any_sync(__activemask(), l);
    if (l >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&count[l], __popc(peers));
  });
}

// one entry per component (its root has a non-zero count); unordered
__global__ void k_size_list(int64_t N, const int32_t *count, unsigned long long *n,
                            int64_t cap, int64_t *roots, int64_t *sizes, int nbins,
                            unsigned long long *hist) {
  quad_pass(N, count, [&](int64_t k, int32_t c) {
    if (c == 0) return;
    const unsigned long long q = atomicAdd(n, 1ull);
    if ((int64_t)q < cap) {
      roots[q] = k;
      sizes[q] = c;
    }
    // 2^b <= c < 2^(b+1), the last bin open-ended
    int b = 31 - __clz(c);
    if (b > nbins - 1) b = nbins - 1;
    atomicAdd(&hist[b], 1ull);
  });
}

}  // namespace

cudaError_t diag_bubble_sizes(const View &v, const int32_t *labels, int32_t *count_scratch,
                              unsigned long long *n_dev, int64_t cap, int64_t *roots,
                              int64_t *sizes, int nbins, unsigned long long *hist,
                              cudaStream_t s) {
  const int64_t N = v.NX * v.NY * v.NZ;
  cudaError_t e = cudaMemsetAsync(count_scratch, 0, sizeof(int32_t) * N, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(n_dev, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * nbins, s);
  if (e != cudaSuccess) return e;
  k_size_count<<<grid_of((N + 3) / 4), TPB, 0, s>>>(N, labels, count_scratch);
  k_size_list<<<grid_of((N + 3) / 4), TPB, 0, s>>>(N, count_scratch, n_dev, cap, roots, sizes, nbins, hist);
  return cudaGetLastError();
}

}  // namespace sclbm
