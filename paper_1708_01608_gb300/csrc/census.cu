// Bubble census and the per-lattice-point film test (Sec. 4).
//
// Both work on the gas labels of the labelling kernels (label = smallest
// linear index of the component, -1 for liquid) and, for the film test, on
// the FP64 EOS pressure field of diag_moments.  Cells are linear view
// indices x + NX (y + NY z); D2Q9 runs on the view (nx, 1, ny), so its two
// axes are view axes 0 and 2.
#include "internal.h"
#include "lattice.cuh"

namespace sclbm {

namespace {

constexpr int TPB = 256;
inline int grid_of(int64_t n) {
  const int64_t b = (n + TPB - 1) / TPB;
  return (int)(b < 1 ? 1 : (b > 262144 ? 262144 : b));
}
#define CENSUS_LOOP(k, n) \
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < (n); \
       k += (int64_t)gridDim.x * blockDim.x)

// ---- bubble sizes -----------------------------------------------------------
__global__ void k_size_count(int64_t N, const int32_t *labels, int32_t *count) {
  CENSUS_LOOP(k, N) {
    const int32_t l = labels[k];
    if (l >= 0) atomicAdd(&count[l], 1);
  }
}

// one entry per component (its root has a non-zero count); unordered
__global__ void k_size_list(int64_t N, const int32_t *count, unsigned long long *n,
                            int64_t cap, int64_t *roots, int64_t *sizes, int nbins,
                            unsigned long long *hist) {
  CENSUS_LOOP(k, N) {
    const int32_t c = count[k];
    if (c == 0) continue;
    const unsigned long long q = atomicAdd(n, 1ull);
    if ((int64_t)q < cap) {
      roots[q] = k;
      sizes[q] = c;
    }
    // 2^b <= c < 2^(b+1), the last bin open-ended
    int b = 31 - __clz(c);
    if (b > nbins - 1) b = nbins - 1;
    atomicAdd(&hist[b], 1ull);
  }
}

// ---- film test at every lattice point ---------------------------------------
using FilmRec = lbm_film_cell;  // written as the C ABI hands it out

__device__ __forceinline__ int wrap(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

// One thread per cell.  For each lattice axis: walk to the first gas cell on
// each side (at most h_max cells), classify film / midpoint, and update the
// arming bit of (cell, axis) as the two-bubble criterion does.
__global__ void __launch_bounds__(TPB)
    k_film_cells(const View v, const int32_t *labels, const double *p, int h_max, double eps_arm,
                 uint8_t *state, unsigned long long *counts, int64_t cap, FilmRec *rec) {
  __shared__ unsigned long long sh[4];
  if (threadIdx.x < 4) sh[threadIdx.x] = 0;
  __syncthreads();
  const int64_t N = v.NX * v.NY * v.NZ;
  const int naxes = v.lat == D2Q9 ? 2 : 3;
  unsigned long long nfilm = 0, nmid = 0, narmed = 0;
  CENSUS_LOOP(k, N) {
    const int x = (int)(k % v.NX);
    const int y = (int)((k / v.NX) % v.NY);
    const int z = (int)(k / (v.NX * v.NY));
    uint8_t st = state[k];
    const bool liquid = labels[k] < 0;
    for (int ua = 0; ua < naxes; ++ua) {
      // user axis ua -> view axis (D2Q9: x, z)
      const int va = v.lat == D2Q9 && ua == 1 ? 2 : ua;
      const int n_a = va == 0 ? (int)v.NX : (va == 1 ? (int)v.NY : (int)v.NZ);
      const int c_a = va == 0 ? x : (va == 1 ? y : z);
      auto cell_at = [&](int s) -> int64_t {
        const int q = wrap(c_a + s, n_a);
        const int xx = va == 0 ? q : x, yy = va == 1 ? q : y, zz = va == 2 ? q : z;
        return ((int64_t)zz * v.NY + yy) * v.NX + xx;
      };
      const uint8_t bit = (uint8_t)(1u << ua);
      bool mid = false;
      int32_t Lp = -1, Lm = -1;
      int dp = 0, dm = 0;
      if (liquid) {
        for (int s = 1; s <= h_max; ++s) {
          const int32_t l = labels[cell_at(s)];
          if (l >= 0) {
            Lp = l;
            dp = s;
            break;
          }
        }
        if (Lp >= 0) {
          for (int s = 1; s <= h_max; ++s) {
            const int32_t l = labels[cell_at(-s)];
            if (l >= 0) {
              Lm = l;
              dm = s;
              break;
            }
          }
        }
        const bool film = Lp >= 0 && Lm >= 0 && Lp != Lm && dp + dm - 1 <= h_max;
        nfilm += film;
        mid = film && dp - dm <= 1 && dm - dp <= 1;
      }
      if (!mid) {
        st = (uint8_t)(st & ~bit);
        continue;
      }
      ++nmid;
      const double d2 = p[cell_at(1)] - 2.0 * p[k] + p[cell_at(-1)];
      if (d2 < -eps_arm) {
        st = (uint8_t)(st | bit);
      } else if ((st & bit) && d2 >= 0.0) {
        st = (uint8_t)(st & ~bit);
        const unsigned long long q = atomicAdd(&counts[3], 1ull);
        if ((int64_t)q < cap) {
          FilmRec r;
          r.cell = k;
          r.axis = ua;
          r.label_minus = Lm;
          r.label_plus = Lp;
          r.thickness = dp + dm - 1;
          r.d2p = d2;
          rec[q] = r;
        }
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
  k_size_count<<<grid_of(N), TPB, 0, s>>>(N, labels, count_scratch);
  k_size_list<<<grid_of(N), TPB, 0, s>>>(N, count_scratch, n_dev, cap, roots, sizes, nbins, hist);
  return cudaGetLastError();
}

size_t film_record_bytes() { return sizeof(FilmRec); }

cudaError_t diag_film_cells(const View &v, const int32_t *labels, const double *p, int h_max,
                            double eps_arm, uint8_t *state, unsigned long long *counts,
                            int64_t cap, void *records, cudaStream_t s) {
  const int64_t N = v.NX * v.NY * v.NZ;
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * 4, s);
  if (e != cudaSuccess) return e;
  k_film_cells<<<grid_of(N), TPB, 0, s>>>(v, labels, p, h_max, eps_arm, state, counts, cap,
                                         static_cast<FilmRec *>(records));
  return cudaGetLastError();
}

}  // namespace sclbm
