// Lattice tables, storage codecs and small PTX helpers of the GB300 library.
//
// Kernels see every lattice as three-dimensional: D3Q19 on (nx, ny, nz) and
// D2Q9 on the view (nx, 1, ny), whose velocity (cx, cy) becomes
// (cx, 0, cy).  The memory layout f[i][z][y][x] of the two is identical, so
// the user-facing order of cells and populations does not change.  All
// kernels march along the view's z axis.
//
// Velocity order (user axes) follows the public header: D2Q9
// rest, +x, +y, -x, -y, (1,1), (-1,1), (-1,-1), (1,-1); D3Q19 rest, the six
// axis directions (+x,-x,+y,-y,+z,-z) and the twelve edge directions.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace sclbm {

enum { D2Q9 = 0, D3Q19 = 1 };
enum { ST_F64 = 0, ST_F32 = 1, ST_F16 = 2, ST_BF16 = 3 };
// Step-kernel forms of the 16-bit storages that also keep a per-cell FP32
// rounding residual (the mass the stores' rounding took off the cell in the
// last step, returned into its next collision): the same populations and
// codec as ST_F16 / ST_BF16.  Diagnostics use the base form and read the
// residual field through their View.
enum { ST_F16R = 4, ST_BF16R = 5 };

template <int LAT>
struct Lattice;

// D2Q9 in the 3-D view (x, 1, y): cy of the 2-D set goes to the z slot.
template <>
struct Lattice<D2Q9> {
  static constexpr int Q = 9;
  static constexpr bool HAS_Y = false;  // no velocity moves along the view's y
  __host__ __device__ static constexpr int cx(int i) {
    return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
  }
  __host__ __device__ static constexpr int cy(int) { return 0; }
  __host__ __device__ static constexpr int cz(int i) {
    return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
  // pairs of opposite velocities: (1,3) (2,4) (5,7) (6,8)
  static constexpr int NP = 4;
  __host__ __device__ static constexpr int rep(int k) { return k < 2 ? 1 + k : 3 + k; }
  __host__ __device__ static constexpr int opp(int i) { return i + 2; }
};

template <>
struct Lattice<D3Q19> {
  static constexpr int Q = 19;
  static constexpr bool HAS_Y = true;
  // rest, +x, -x, +y, -y, +z, -z,
  // (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0) (1,0,1) (-1,0,-1) (1,0,-1) (-1,0,1)
  // (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1)
  __host__ __device__ static constexpr int cx(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13)
               ? 1
               : ((i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0);
  }
  __host__ __device__ static constexpr int cy(int i) {
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17)
               ? 1
               : ((i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0);
  }
  __host__ __device__ static constexpr int cz(int i) {
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18)
               ? 1
               : ((i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0);
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
  // pairs of opposite velocities: (1,2) (3,4) ... (17,18)
  static constexpr int NP = 9;
  __host__ __device__ static constexpr int rep(int k) { return 2 * k + 1; }
  __host__ __device__ static constexpr int opp(int i) { return i + 1; }
};

// ---- storage codecs -------------------------------------------------------
// T = stored type, C = arithmetic type.  FP64 stores f_i itself.  The FP32
// and 16-bit forms store the offset g_i = f_i - w_i*rho_ref and the FP32
// kernels do their arithmetic on offsets: round-off then scales with |g|,
// which is small wherever rho is near rho_ref (the bulk liquid), instead of
// with |f| (the shifted-distribution technique of Skordos, Phys. Rev. E 48,
// 4823 (1993)).  load/store convert between T and C without the offset.
template <int ST>
struct Storage;

template <>
struct Storage<ST_F64> {
  using T = double;
  using C = double;
  static constexpr bool OFFSET = false, RESID = false;
  __device__ static C load(T v) { return v; }
  __device__ static T store(C v) { return v; }
};
template <>
struct Storage<ST_F32> {
  using T = float;
  using C = float;
  static constexpr bool OFFSET = true, RESID = false;
  __device__ static C load(T v) { return v; }
  __device__ static T store(C v) { return v; }
};
template <>
struct Storage<ST_F16> {
  using T = __half;
  using C = float;
  static constexpr bool OFFSET = true, RESID = false;
  __device__ static C load(T v) { return __half2float(v); }
  __device__ static T store(C v) { return __float2half_rn(v); }
};
template <>
struct Storage<ST_BF16> {
  using T = __nv_bfloat16;
  using C = float;
  static constexpr bool OFFSET = true, RESID = false;
  __device__ static C load(T v) { return __bfloat162float(v); }
  __device__ static T store(C v) { return __float2bfloat16_rn(v); }
};
template <>
struct Storage<ST_F16R> : Storage<ST_F16> {
  static constexpr bool RESID = true;
};
template <>
struct Storage<ST_BF16R> : Storage<ST_BF16> {
  static constexpr bool RESID = true;
};

// f_i from a stored value and back, in double (diagnostics, state I/O)
// (no FMA contraction: every path that decodes a stored value gets the same
// double, which the host-side checks rely on)
template <int ST>
__device__ __forceinline__ double decode_f(typename Storage<ST>::T v, double wref) {
  return Storage<ST>::OFFSET ? __dadd_rn(wref, (double)Storage<ST>::load(v))
                             : (double)Storage<ST>::load(v);
}
template <int ST>
__device__ __forceinline__ typename Storage<ST>::T encode_f(double f, double wref) {
  using C = typename Storage<ST>::C;
  return Storage<ST>::store(Storage<ST>::OFFSET ? (C)(f - wref) : (C)f);
}

inline size_t storage_bytes(int st) { return st == ST_F64 ? 8 : (st == ST_F32 ? 4 : 2); }

// psi(rho) = rho0 (1 - exp(-rho/rho0))
__device__ __forceinline__ double psi_of(double rho, double rho0, double inv_rho0) {
  return rho0 * (1.0 - exp(-rho * inv_rho0));
}
// (FP32: the hardware exponential, a few ulp, far below FP32 storage noise;
// evaluated as rho0 - rho0 e in one FMA, the form every FP32 kernel uses)
__device__ __forceinline__ float psi_of(float rho, float rho0, float inv_rho0) {
  return fmaf(-rho0, __expf(rho * -inv_rho0), rho0);
}

// ---- compile-time helpers of the FP32 collision ----------------------------
// f(integral_constant<int, 0>), ..., f(integral_constant<int, N-1>)
template <class F, int... K>
__device__ __forceinline__ void static_for_impl(F &f, std::integer_sequence<int, K...>) {
  (f(std::integral_constant<int, K>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F &&f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}
// acc + c v and acc + c w v for a velocity component c in {-1, 0, 1}: terms
// with c = 0 vanish at compile time (a product with 0.0 is not removable
// under IEEE rules, so c v must not be written out for c = 0)
template <int CC>
__device__ __forceinline__ float cacc(float acc, float v) {
  if constexpr (CC > 0) return acc + v;
  else if constexpr (CC < 0) return acc - v;
  else return acc;
}
template <int CC>
__device__ __forceinline__ float cfma(float acc, float w, float v) {
  if constexpr (CC > 0) return fmaf(w, v, acc);
  else if constexpr (CC < 0) return fmaf(-w, v, acc);
  else return acc;
}
// c.u for a moving velocity c with components in {-1, 0, 1}: nonzero terms only
template <int A, int B, int Z>
__device__ __forceinline__ float cdot(float x, float y, float z) {
  static_assert(A != 0 || B != 0 || Z != 0, "moving velocities only");
  float r;
  if constexpr (A != 0) r = A > 0 ? x : -x;
  else if constexpr (B != 0) r = B > 0 ? y : -y;
  else r = Z > 0 ? z : -z;
  if constexpr (A != 0 && B != 0) r = B > 0 ? r + y : r - y;
  if constexpr ((A != 0 || B != 0) && Z != 0) r = Z > 0 ? r + z : r - z;
  return r;
}

// ---- small PTX helpers ----------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for a phase with a time limit; false when the limit passed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
  return true;
}
// 4-D tiled TMA load (coordinates x, y, z, population) completing on bar.
__device__ __forceinline__ void tma_load_4d(void *dst, const void *tmap, int c0, int c1, int c2,
                                            int c3, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void prefetch_tmap(const void *tmap) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(tmap) : "memory");
}

// GPU-scope acquire load and release store of a 32-bit flag
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void fence_acq_rel_gpu() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}
// orders this thread's view of global memory (generic proxy) before its
// later bulk-tensor copies (async proxy)
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// error bits reported through the context's device status word
enum { ERR_TMA_TIMEOUT = 1, ERR_NONFINITE = 2, ERR_SYNC_TIMEOUT = 4 };

}  // namespace sclbm
