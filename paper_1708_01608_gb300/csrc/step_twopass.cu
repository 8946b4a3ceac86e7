// Two-pass Shan-Chen step (push form, stored_i(x) = f_i(x, t)): pass 1
// computes psi(x) for every cell; pass 2 reads the populations again, takes
// psi of the neighbours from that field, collides and pushes f*_i to x + c_i.  The blowing-agent
// injection runs as a third, one-thread-per-site kernel.  This path moves
// 3*Q*S + 2*sizeof(psi) bytes per update instead of the fused kernel's
// 2*Q*S; it is kept as a simple, independently written comparison path.
#include <cmath>
#include <mutex>

#include "internal.h"
#include "lattice.cuh"

namespace sclbm {

struct Cell {
  int x, y, z;
};

__device__ __forceinline__ Cell cell_of(int64_t k, int64_t NX, int64_t NY) {
  Cell c;
  c.x = (int)(k % NX);
  const int64_t r = k / NX;
  c.y = (int)(r % NY);
  c.z = (int)(r / NY);
  return c;
}
__device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// f_i in the arithmetic type from a stored value and back (offset storage
// adds / removes w_i rho_ref)
template <int ST>
__device__ __forceinline__ typename Storage<ST>::C dec(typename Storage<ST>::T v,
                                                       typename Storage<ST>::C wref) {
  return Storage<ST>::OFFSET ? wref + Storage<ST>::load(v) : Storage<ST>::load(v);
}
template <int ST>
__device__ __forceinline__ typename Storage<ST>::T enc(typename Storage<ST>::C f,
                                                       typename Storage<ST>::C wref) {
  return Storage<ST>::store(Storage<ST>::OFFSET ? f - wref : f);
}

template <int LAT, int ST>
__global__ void tp_psi_kernel(const StepArgs a, typename Storage<ST>::C *psi) {
  using L = Lattice<LAT>;
  using S = Storage<ST>;
  using T = typename S::T;
  using C = typename S::C;
  const int64_t N = a.NX * a.NY * a.NZ;
  const int64_t plane = a.px * a.NY, pop = plane * a.NZ;
  const T *f = static_cast<const T *>(a.fin);
  const C rho0 = (C)a.rho0, inv_rho0 = (C)(1.0 / a.rho0);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x) {
    const Cell c = cell_of(k, a.NX, a.NY);
    const int64_t o = (int64_t)c.z * plane + (int64_t)c.y * a.px + c.x;
    C rho = 0;
    if constexpr (S::OFFSET) {  // rho_ref + the sum of the offsets, as the collision has it
#pragma unroll
      for (int i = 0; i < L::Q; ++i) rho += S::load(f[i * pop + o]);
      if constexpr (S::RESID) rho += a.resid[o];
      rho += (C)a.rho_ref;
    } else {
#pragma unroll
      for (int i = 0; i < L::Q; ++i) rho += dec<ST>(f[i * pop + o], (C)(L::w(i) * a.rho_ref));
    }
    psi[k] = psi_of(rho, rho0, inv_rho0);
  }
}

template <int LAT, int ST>
__global__ void tp_collide_kernel(const StepArgs a, const typename Storage<ST>::C *psi) {
  using L = Lattice<LAT>;
  using S = Storage<ST>;
  using T = typename S::T;
  using C = typename S::C;
  const int64_t N = a.NX * a.NY * a.NZ;
  const int64_t plane = a.px * a.NY, pop = plane * a.NZ;
  const T *f = static_cast<const T *>(a.fin);
  T *g = static_cast<T *>(a.fout);
  const C G = (C)a.G, tau = (C)a.tau, omega = (C)(1.0 / a.tau);
  const int NX = (int)a.NX, NY = (int)a.NY, NZ = (int)a.NZ;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x) {
    const Cell c = cell_of(k, a.NX, a.NY);
    const int64_t own = (int64_t)c.z * plane + (int64_t)c.y * a.px + c.x;
    C sx = 0, sy = 0, sz = 0;
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
      const int nx_ = wrapi(c.x + L::cx(i), NX), ny_ = wrapi(c.y + L::cy(i), NY),
                nz_ = wrapi(c.z + L::cz(i), NZ);
      const C wp = (C)L::w(i) * psi[((int64_t)nz_ * NY + ny_) * NX + nx_];
      sx += (C)L::cx(i) * wp;
      sy += (C)L::cy(i) * wp;
      sz += (C)L::cz(i) * wp;
    }
    const C gp = -G * psi[k];
    if constexpr (sizeof(C) == 8) {
      // FP64: the oracle's operation order on the populations themselves
      C fi[L::Q];
      C rho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        fi[i] = dec<ST>(f[i * pop + own], (C)(L::w(i) * a.rho_ref));
        rho += fi[i];
        jx += (C)L::cx(i) * fi[i];
        jy += (C)L::cy(i) * fi[i];
        jz += (C)L::cz(i) * fi[i];
      }
      const C ux = (jx + tau * gp * sx) / rho, uy = (jy + tau * gp * sy) / rho,
              uz = (jz + tau * gp * sz) / rho;
      const C uu = (C)1.5 * (ux * ux + uy * uy + uz * uz);
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        const C cu = (C)L::cx(i) * ux + (C)L::cy(i) * uy + (C)L::cz(i) * uz;
        const C feq = (C)L::w(i) * rho * ((C)1 + (C)3 * cu + (C)4.5 * cu * cu - uu);
        const int X = wrapi(c.x + L::cx(i), NX), Y = wrapi(c.y + L::cy(i), NY),
                  Z = wrapi(c.z + L::cz(i), NZ);
        g[i * pop + (int64_t)Z * plane + (int64_t)Y * a.px + X] =
            enc<ST>(fi[i] - (fi[i] - feq) / tau, (C)(L::w(i) * a.rho_ref));
      }
    } else {
      // FP32 on the offsets g_i = f_i - w_i rho_ref (rho = rho_ref + R with
      // R = sum g_i; rho_ref = 0 gives the plain populations): the
      // equilibrium offset is w_i (K + rho (3 c.u + 4.5 (c.u)^2)) with
      // K = R - 1.5 rho u.u, and the rest population takes R minus the
      // moving ones, so mass is conserved to FP32 rounding of the offsets
      C gi[L::Q];
      C R = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        gi[i] = S::load(f[i * pop + own]);
        R += gi[i];
        jx += (C)L::cx(i) * gi[i];
        jy += (C)L::cy(i) * gi[i];
        jz += (C)L::cz(i) * gi[i];
      }
      // residual forms: the cell's rounding residual of the last step is part
      // of its mass (it enters the rest population below)
      if constexpr (S::RESID) R += a.resid[own];
      const C rho = (C)a.rho_ref + R;
      const C ir = (C)1 / rho;
      const C ux = (jx + tau * gp * sx) * ir, uy = (jy + tau * gp * sy) * ir,
              uz = (jz + tau * gp * sz) * ir;
      const C K = R - (C)1.5 * rho * (ux * ux + uy * uy + uz * uz);
      C moved = 0;
      C racc = 0;  // residual forms: what this cell's stores round off
      auto put = [&](int64_t o, C off) {
        const T q = S::store(off);
        g[o] = q;
        if constexpr (S::RESID) racc += off - S::load(q);
      };
#pragma unroll
      for (int i = 1; i < L::Q; ++i) {
        const C cu = (C)L::cx(i) * ux + (C)L::cy(i) * uy + (C)L::cz(i) * uz;
        const C feq = (C)L::w(i) * (K + rho * ((C)3 * cu + (C)4.5 * cu * cu));
        const C gs = gi[i] - omega * (gi[i] - feq);
        moved += gs;
        const int X = wrapi(c.x + L::cx(i), NX), Y = wrapi(c.y + L::cy(i), NY),
                  Z = wrapi(c.z + L::cz(i), NZ);
        put(i * pop + (int64_t)Z * plane + (int64_t)Y * a.px + X, gs);
      }
      put(own, R - moved);
      if constexpr (S::RESID) a.resid[own] = racc;
    }
  }
}

template <int LAT, int ST>
__global__ void tp_inject_kernel(const StepArgs a) {
  using L = Lattice<LAT>;
  using S = Storage<ST>;
  using T = typename S::T;
  using C = typename S::C;
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= a.ngroups) return;
  double dm = 0.0;
  int s0 = -1;
  for (int q = a.group_off[gi]; q < a.group_off[gi + 1]; ++q) {
    const int s = a.group_site[q];
    s0 = s;
    const double b = a.budget[s];
    if (b > 0.0) {
      const double d = fmin(a.rate[s], b);
      a.budget[s] = b - d;
      dm += d;
    }
  }
  if (dm == 0.0 || s0 < 0) return;
  // the deposit is part of f* at the site, which has been pushed to x_s + c_i
  const int64_t plane = a.px * a.NY, pop = plane * a.NZ;
  T *g = static_cast<T *>(a.fout);
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const int X = wrapi(a.site_x[s0] + L::cx(i), (int)a.NX),
              Y = wrapi(a.site_y[s0] + L::cy(i), (int)a.NY),
              Z = wrapi(a.site_z[s0] + L::cz(i), (int)a.NZ);
    const int64_t cell = (int64_t)Z * plane + (int64_t)Y * a.px + X;
    T *o = g + i * pop + cell;
    const C wref = (C)(L::w(i) * a.rho_ref);
    if constexpr (S::RESID) {
      // the deposit on the offset itself; its rounding goes to the receiving
      // cell's residual (atomic: neighbouring sites can push into one cell)
      const C off = S::load(*o) + (C)(L::w(i) * dm);
      const T q = S::store(off);
      *o = q;
      atomicAdd(a.resid + cell, off - S::load(q));
    } else {
      *o = enc<ST>(dec<ST>(*o, wref) + (C)(L::w(i) * dm), wref);
    }
  }
}

template <int LAT, int ST>
static cudaError_t tp_launch_t(const StepArgs &a, void *psi, cudaStream_t s) {
  using C = typename Storage<ST>::C;
  const int64_t N = a.NX * a.NY * a.NZ;
  const int threads = 256;
  const int blocks = (int)((N + threads - 1) / threads < 1048576 ? (N + threads - 1) / threads
                                                                  : 1048576);
  tp_psi_kernel<LAT, ST><<<blocks, threads, 0, s>>>(a, static_cast<C *>(psi));
  tp_collide_kernel<LAT, ST><<<blocks, threads, 0, s>>>(a, static_cast<const C *>(psi));
  if (a.nsites > 0) tp_inject_kernel<LAT, ST><<<(a.ngroups + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t twopass_launch(int lat, int st, const StepArgs &a, void *psi, cudaStream_t s) {
  if (lat == D3Q19) {
    switch (st) {
      case ST_F64: return tp_launch_t<D3Q19, ST_F64>(a, psi, s);
      case ST_F32: return tp_launch_t<D3Q19, ST_F32>(a, psi, s);
      case ST_F16: return tp_launch_t<D3Q19, ST_F16>(a, psi, s);
      case ST_F16R: return tp_launch_t<D3Q19, ST_F16R>(a, psi, s);
      case ST_BF16R: return tp_launch_t<D3Q19, ST_BF16R>(a, psi, s);
      default: return tp_launch_t<D3Q19, ST_BF16>(a, psi, s);
    }
  }
  switch (st) {
    case ST_F64: return tp_launch_t<D2Q9, ST_F64>(a, psi, s);
    case ST_F32: return tp_launch_t<D2Q9, ST_F32>(a, psi, s);
    case ST_F16: return tp_launch_t<D2Q9, ST_F16>(a, psi, s);
    case ST_F16R: return tp_launch_t<D2Q9, ST_F16R>(a, psi, s);
    case ST_BF16R: return tp_launch_t<D2Q9, ST_BF16R>(a, psi, s);
    default: return tp_launch_t<D2Q9, ST_BF16>(a, psi, s);
  }
}

}  // namespace sclbm

// ---- allocation-free time step ---------------------------------------------
// Some callers cannot call cudaMalloc: a host framework that owns the whole
// device-memory pool and forbids allocations behind its back, a time loop
// that must not stall on the allocator (cudaMalloc and cudaFree can
// synchronise the device), or a program held to a fixed memory budget.  The
// two-pass step needs a psi field between its two kernels; this entry point
// keeps that field in a file-scope device array of fixed size, so it
// allocates nothing.  In host code the array's name is only a host-side
// stand-in: its device address is looked up with cudaGetSymbolAddress, once
// per CUDA context (keyed by the context's process-unique id, so a second
// context on the same device, or the new primary context after
// cudaDeviceReset, gets its own look-up).
namespace sclbm {
namespace {

constexpr int64_t kStaticPsiCells = 2097152;  // 8 MB of FP32: up to 128^3 cells
constexpr int kMaxContexts = 64;

static __device__ __align__(256) float g_static_psi[kStaticPsiCells];

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

std::mutex g_static_mu;
struct StaticEntry {
  unsigned long long ctx_id;
  float *psi;
};
StaticEntry g_static_cache[kMaxContexts];
int g_static_n = 0, g_static_next = 0;

// driver functions used to identify the current context (fetched once)
bool ctx_functions(CtxGetCurrentFn *cur, CtxGetIdFn *id) {
  static CtxGetCurrentFn f_cur = nullptr;
  static CtxGetIdFn f_id = nullptr;
  if (!f_cur || !f_id) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      f_cur = reinterpret_cast<CtxGetCurrentFn>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      f_id = reinterpret_cast<CtxGetIdFn>(p);
  }
  *cur = f_cur;
  *id = f_id;
  return f_cur && f_id;
}

// device address of g_static_psi in the current context (looked up on the
// first call in each context, then cached)
cudaError_t static_psi_address(float **out) {
  CtxGetCurrentFn get_cur;
  CtxGetIdFn get_id;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!ctx_functions(&get_cur, &get_id)) return cudaErrorNotSupported;
  CUcontext ctx = nullptr;
  if (get_cur(&ctx) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  if (!ctx) {
    // no context is current yet: cudaSetDevice makes the current device's
    // primary context current (it allocates nothing)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaSetDevice(dev);
    if (e != cudaSuccess) return e;
    if (get_cur(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
  }
  unsigned long long id = 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  for (int k = 0; k < g_static_n; ++k)
    if (g_static_cache[k].ctx_id == id) {
      *out = g_static_cache[k].psi;
      return cudaSuccess;
    }
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_psi);
  if (e != cudaSuccess) return e;
  // a full table reuses its oldest entry: a context evicted that way is
  // looked up again on its next call
  const int slot = g_static_n < kMaxContexts ? g_static_n++ : g_static_next;
  if (g_static_n == kMaxContexts) g_static_next = (slot + 1) % kMaxContexts;
  g_static_cache[slot] = StaticEntry{id, static_cast<float *>(p)};
  *out = static_cast<float *>(p);
  return cudaSuccess;
}

}  // namespace
}  // namespace sclbm

extern "C" lbm_status lbm_step_static_f32(int32_t lattice, int64_t nx, int64_t ny, int64_t nz,
                                          double tau, double G, double rho0, const float *f_in,
                                          float *f_out, void *stream) {
  using namespace sclbm;
  if (lattice != LBM_D2Q9 && lattice != LBM_D3Q19)
    return set_error(LBM_EINVAL, "lbm_step_static_f32: unknown lattice");
  if (nx < 1 || ny < 1 || nz < 1 || (lattice == LBM_D2Q9 && nz != 1))
    return set_error(LBM_EINVAL, "lbm_step_static_f32: extents must be >= 1 (nz = 1 for D2Q9)");
  // nx * ny * nz <= cap, tested by division so that no product can overflow
  if (nx > kStaticPsiCells || ny > kStaticPsiCells / nx || nz > kStaticPsiCells / (nx * ny))
    return set_error(LBM_EINVAL,
                     "lbm_step_static_f32: more than 2097152 cells, the size of the static "
                     "scratch array (use lbm_create/lbm_step for larger lattices)");
  if (!(tau > 0.5) || !std::isfinite(tau) || !(rho0 > 0) || !std::isfinite(rho0) ||
      !std::isfinite(G))
    return set_error(LBM_EINVAL,
                     "lbm_step_static_f32: tau must be finite and > 0.5, rho0 finite and > 0, "
                     "G finite");
  if (!f_in || !f_out || static_cast<const void *>(f_in) == static_cast<const void *>(f_out))
    return set_error(LBM_EINVAL, "lbm_step_static_f32: f_in and f_out must be distinct buffers");
  float *psi = nullptr;
  cudaError_t e = static_psi_address(&psi);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(LBM_ECUDA, cudaGetErrorString(e));
  }
  StepArgs a{};
  a.fin = f_in;
  a.fout = f_out;
  a.NX = nx;
  a.NY = lattice == LBM_D2Q9 ? 1 : ny;  // D2Q9 runs on the view (nx, 1, ny)
  a.NZ = lattice == LBM_D2Q9 ? ny : nz;
  a.px = nx;
  a.tau = tau;
  a.G = G;
  a.rho0 = rho0;
  a.rho_ref = 0.0;  // plain f_i, no offset
  a.nsites = 0;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  e = lattice == LBM_D2Q9 ? tp_launch_t<D2Q9, ST_F32>(a, psi, s) : tp_launch_t<D3Q19, ST_F32>(a, psi, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(LBM_ECUDA, cudaGetErrorString(e));
  }
  return LBM_OK;
}
