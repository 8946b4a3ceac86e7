// Fused Shan-Chen collide-stream-force step (one kernel per time step).
//
// A CTA owns a BX x BY column of the lattice (x, y) and marches along z
// through a chunk of planes.  For every destination plane P it stages, with
// one 4-D TMA box per population, the post-collision populations that stream
// into the column and its one-cell halo ring (pull scheme: population i of
// destination cell x comes from x - c_i).  From the staged plane it computes
// rho and psi of every cell of the column plus halo; psi lives in a ring of
// four planes in shared memory, so the Shan-Chen force of plane P - 1, which
// needs psi of planes P - 2 .. P, is available without a second pass over
// the populations.  The interior cell's own populations are kept in
// registers for the next iteration's collision.  Each cell is read from HBM
// once and written once per step; halo cells are re-read from L2.
//
// Periodic seams: TMA fills out-of-range boxes with zeros; CTAs whose halo
// crosses the x or y boundary overwrite those elements with the wrapped
// values using plain loads (the z coordinate is wrapped before the copy).
//
// Every wait on a TMA transaction is bounded (1 s); on timeout the CTA sets
// ERR_TMA_TIMEOUT in the status word, waits (bounded) for its other copies
// and returns without writing further planes.
#pragma once

#include "internal.h"
#include "lattice.cuh"

namespace sclbm {

template <int LAT, int ST, int BX_, int BY_, int NS_>
struct FusedK {
  using L = Lattice<LAT>;
  using S = Storage<ST>;
  using T = typename S::T;
  using C = typename S::C;
  static constexpr int BX = BX_, BY = BY_, NS = NS_;
  static constexpr int Q = L::Q;
  static constexpr int HY = L::HAS_Y ? 1 : 0;
  // x halo of the staged box: at least 2 source columns, rounded so that the
  // box starts on a 16-byte boundary
  static constexpr int HX = (16 / (int)sizeof(T)) > 2 ? 16 / (int)sizeof(T) : 2;
  static constexpr int BW = BX + 2 * HX;
  static constexpr int BH = BY + 2 * HY;
  static constexpr int BOX_BYTES = BW * BH * (int)sizeof(T);
  // a TMA box is at most 256 elements wide: rows wider than that are loaded
  // as NSUB side-by-side boxes of SUBW elements (16-byte multiples), which
  // is contiguous in shared memory only for single-row boxes
  static constexpr int pick_nsub() {
    for (int n = (BW + 255) / 256; n <= BW; ++n)
      if (BW % n == 0 && ((BW / n) * (int)sizeof(T)) % 16 == 0) return n;
    return -1;
  }
  static constexpr int NSUB = pick_nsub();
  static constexpr int SUBW = BW / NSUB;
  static_assert(NSUB > 0 && (NSUB == 1 || BH == 1), "unsupported tile width");
  static constexpr int BOX_STRIDE = (BOX_BYTES + 127) / 128 * 128;
  static constexpr int STAGE_BYTES = Q * BOX_STRIDE;
  static constexpr int PW = BX + 2;
  static constexpr int PH = BY + 2 * HY;
  static constexpr int RING_BYTES = (4 * PW * PH * (int)sizeof(C) + 15) / 16 * 16;
  static constexpr int NT = BX * BY;
  static constexpr int SMEM = NS * STAGE_BYTES + RING_BYTES + NS * 8 + 128;
};

__device__ __forceinline__ int imod(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

template <int LAT, int ST, int BX, int BY, int NS>
__global__ void __launch_bounds__(BX *BY)
    fused_step_kernel(const __grid_constant__ CUtensorMap tm, const StepArgs a, const int tiles_x,
                      const int tiles_y, const int zlen) {
  using K = FusedK<LAT, ST, BX, BY, NS>;
  using L = typename K::L;
  using S = typename K::S;
  using T = typename K::T;
  using C = typename K::C;
  constexpr int Q = K::Q, HY = K::HY, HX = K::HX, BW = K::BW, PW = K::PW, PH = K::PH,
                NT = K::NT;

  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
  C *ring = reinterpret_cast<C *>(smem + NS * K::STAGE_BYTES);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + NS * K::STAGE_BYTES + K::RING_BYTES);

  const int tid = threadIdx.x;
  const int tx = tid % BX, ty = tid / BX;
  const int item = blockIdx.x;
  const int ntiles = tiles_x * tiles_y;
  const int zc = item / ntiles, tt = item % ntiles;
  const int NX = (int)a.NX, NY = (int)a.NY, NZ = (int)a.NZ;
  const int x0 = (tt % tiles_x) * BX, y0 = (tt / tiles_x) * BY;
  const int BXe = min(BX, NX - x0), BYe = min(BY, NY - y0);
  const int zs = zc * zlen, ze = min(NZ, zs + zlen);
  if (zs >= ze) return;
  const int NPL = ze - zs + 2;  // staged destination planes zs-1 .. ze
  const bool seam =
      (x0 < 2) || (x0 + BXe + 2 > NX) || (HY && ((y0 < 2) || (y0 + BYe + 2 > NY)));
  const bool active = tx < BXe && ty < BYe;

  const int64_t plane = a.px * a.NY;
  const int64_t popstride = plane * a.NZ;
  const T *fin = static_cast<const T *>(a.fin);
  T *fout = static_cast<T *>(a.fout);

  const C G = (C)a.G, tau = (C)a.tau, omega = (C)(1.0 / a.tau), rho0 = (C)a.rho0,
          inv_rho0 = (C)(1.0 / a.rho0);
  C wref[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) wref[i] = (C)(L::w(i) * a.rho_ref);

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(&bars[s], 1);
    fence_barrier_init();
    fence_proxy_async_smem();
    prefetch_tmap(&tm);
  }
  __syncthreads();

  auto box = [&](int s, int i) -> const T * {
    return reinterpret_cast<const T *>(smem + s * K::STAGE_BYTES + i * K::BOX_STRIDE);
  };
  auto issue = [&](int k) {
    const int P = zs - 1 + k, s = k % NS;
    mbar_arrive_expect_tx(&bars[s], (uint32_t)(Q * K::BOX_BYTES));
#pragma unroll
    for (int i = 0; i < Q; ++i) {
#pragma unroll
      for (int j = 0; j < K::NSUB; ++j)
        tma_load_4d(smem + s * K::STAGE_BYTES + i * K::BOX_STRIDE + j * K::SUBW * (int)sizeof(T),
                    &tm, x0 - HX + j * K::SUBW, y0 - HY - L::cy(i), imod(P - L::cz(i), NZ), i,
                    &bars[s]);
    }
  };
  if (tid == 0) {
    for (int k = 0; k < NS && k < NPL; ++k) issue(k);
  }

  int sp = 0, send = 0;  // this CTA's injection sites, sorted by z
  if (a.nsites > 0) {
    sp = a.bucket_off[item];
    send = a.bucket_off[item + 1];
  }

  C cur[Q], nxt[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) cur[i] = nxt[i] = 0;

  for (int k = 0; k < NPL; ++k) {
    const int s = k % NS;
    const int P = zs - 1 + k;
    const bool ok = mbar_wait_bounded(&bars[s], (uint32_t)((k / NS) & 1), 1000000000ull);

    if (seam) {
      // Wrapped halo elements: TMA read zeros outside [0,NX) x [0,NY).
      const int rowsA = BYe + 2 * HY;
      const int nA = Q * rowsA * 4;
      const int nB = HY ? Q * 4 * (BXe + 4) : 0;
      for (int e = tid; e < nA + nB; e += NT) {
        int i, dy, lc;
        if (e < nA) {
          i = e / (rowsA * 4);
          const int r = e % (rowsA * 4);
          dy = r / 4 - HY;
          const int j = r % 4;
          lc = j < 2 ? j - 2 : BXe + j - 2;
        } else {
          const int e2 = e - nA;
          i = e2 / (4 * (BXe + 4));
          const int r = e2 % (4 * (BXe + 4));
          const int rs = r / (BXe + 4);
          dy = rs == 0 ? -1 : (rs == 1 ? 0 : (rs == 2 ? BYe - 1 : BYe));
          lc = r % (BXe + 4) - 2;
        }
        int cyi = 0, czi = 0;
#pragma unroll
        for (int m = 0; m < Q; ++m)
          if (m == i) {
            cyi = L::cy(m);
            czi = L::cz(m);
          }
        const int gx = x0 + lc, gy = y0 + dy - cyi;
        if (gx >= 0 && gx < NX && gy >= 0 && gy < NY) continue;
        const int64_t src = (int64_t)i * popstride + (int64_t)imod(P - czi, NZ) * plane +
                            (int64_t)imod(gy, NY) * a.px + imod(gx, NX);
        T *dst = reinterpret_cast<T *>(smem + s * K::STAGE_BYTES + i * K::BOX_STRIDE);
        dst[(dy + HY) * BW + lc + HX] = fin[src];
      }
      __syncthreads();
    }

    // ---- psi of plane P for the column and its halo ring
    C *rk = ring + (k & 3) * PW * PH;
    if (active) {
      C rho = 0;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const C v = S::load(box(s, i)[(ty + HY) * BW + tx - L::cx(i) + HX], wref[i]);
        nxt[i] = v;
        rho += v;
      }
      rk[(ty + HY) * PW + tx + 1] = psi_of(rho, rho0, inv_rho0);
    }
    const int nhalo = HY ? 2 * (BXe + 2) + 2 * BYe : 2;
    for (int h = tid; h < nhalo; h += NT) {
      int dx, dy;
      if (HY) {
        if (h < BXe + 2) {
          dx = h - 1;
          dy = -1;
        } else if (h < 2 * (BXe + 2)) {
          dx = h - (BXe + 2) - 1;
          dy = BYe;
        } else {
          const int h2 = h - 2 * (BXe + 2);
          dx = h2 < BYe ? -1 : BXe;
          dy = h2 < BYe ? h2 : h2 - BYe;
        }
      } else {
        dx = h == 0 ? -1 : BXe;
        dy = 0;
      }
      C rho = 0;
#pragma unroll
      for (int i = 0; i < Q; ++i)
        rho += S::load(box(s, i)[(dy + HY) * BW + dx - L::cx(i) + HX], wref[i]);
      rk[(dy + HY) * PW + dx + 1] = psi_of(rho, rho0, inv_rho0);
    }

    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(a.err, ERR_TMA_TIMEOUT);
        // wait (bounded) for copies still in flight into this CTA's stages
        for (int k2 = k + 1; k2 < NPL && k2 < k + NS; ++k2)
          mbar_wait_bounded(&bars[k2 % NS], (uint32_t)((k2 / NS) & 1), 100000000ull);
      }
      return;
    }
    if (tid == 0 && k + NS < NPL) {
      fence_proxy_async_smem();
      issue(k + NS);
    }

    // ---- collide plane P - 1 (needs psi of P - 2, P - 1, P)
    if (k >= 2) {
      const int Pc = P - 1;
      double dm = 0.0;  // blowing-agent mass deposited in this cell this step
      if (a.nsites > 0) {
        while (sp < send && a.site_z[a.bucket_site[sp]] < Pc) ++sp;
        for (int q = sp; q < send; ++q) {
          const int sidx = a.bucket_site[q];
          if (a.site_z[sidx] != Pc) break;
          if (active && a.site_x[sidx] == x0 + tx && a.site_y[sidx] == y0 + ty) {
            const double b = a.budget[sidx];
            if (b > 0.0) {
              const double d = fmin(a.rate[sidx], b);
              a.budget[sidx] = b - d;
              dm += d;
            }
          }
        }
      }
      if (active) {
        const C *pm = ring + ((k - 2) & 3) * PW * PH;
        const C *p0 = ring + ((k - 1) & 3) * PW * PH;
        const C *pp = ring + (k & 3) * PW * PH;
        const int c0 = (ty + HY) * PW + tx + 1;
        C rho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          rho += cur[i];
          jx += (C)L::cx(i) * cur[i];
          jy += (C)L::cy(i) * cur[i];
          jz += (C)L::cz(i) * cur[i];
        }
        C sx = 0, sy = 0, sz = 0;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
          const C *pl = L::cz(i) < 0 ? pm : (L::cz(i) > 0 ? pp : p0);
          const C wp = (C)L::w(i) * pl[c0 + L::cy(i) * PW + L::cx(i)];
          sx += (C)L::cx(i) * wp;
          sy += (C)L::cy(i) * wp;
          sz += (C)L::cz(i) * wp;
        }
        const C gp = -G * p0[c0];
        const C Fx = gp * sx, Fy = gp * sy, Fz = gp * sz;
        const C ir = (C)1 / rho;
        const C ux = (jx + tau * Fx) * ir, uy = (jy + tau * Fy) * ir, uz = (jz + tau * Fz) * ir;
        const C uu = (C)1.5 * (ux * ux + uy * uy + uz * uz);
        T *o = fout + (int64_t)Pc * plane + (int64_t)(y0 + ty) * a.px + x0 + tx;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const C cu = (C)L::cx(i) * ux + (C)L::cy(i) * uy + (C)L::cz(i) * uz;
          const C feq = (C)L::w(i) * rho * ((C)1 + (C)3 * cu + (C)4.5 * cu * cu - uu);
          C fs = cur[i] - omega * (cur[i] - feq);
          if (dm != 0.0) fs += (C)(L::w(i) * dm);
          o[(int64_t)i * popstride] = S::store(fs, wref[i]);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) cur[i] = nxt[i];
  }
}

template <int LAT, int ST, int BX, int BY, int NS>
cudaError_t fused_prepare_t() {
  using K = FusedK<LAT, ST, BX, BY, NS>;
  return cudaFuncSetAttribute(fused_step_kernel<LAT, ST, BX, BY, NS>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM);
}

template <int LAT, int ST, int BX, int BY, int NS>
cudaError_t fused_launch_t(const FusedPlan &p, const StepArgs &a, const CUtensorMap &tm,
                           cudaStream_t s) {
  using K = FusedK<LAT, ST, BX, BY, NS>;
  fused_step_kernel<LAT, ST, BX, BY, NS>
      <<<p.items, K::NT, K::SMEM, s>>>(tm, a, p.tiles_x, p.tiles_y, p.zlen);
  return cudaGetLastError();
}

template <int LAT, int ST, int BX, int BY, int NS>
int fused_smem_t() {
  return FusedK<LAT, ST, BX, BY, NS>::SMEM;
}

// Tile table shared by every storage type: id -> (BX, BY, NS).
#define SCLBM_D3Q19_TILES(X) \
  X(1, 32, 8, 3)             \
  X(2, 32, 4, 4)             \
  X(3, 64, 4, 3)             \
  X(4, 64, 8, 2)
#define SCLBM_D2Q9_TILES(X) \
  X(1, 256, 1, 4)           \
  X(2, 128, 1, 4)           \
  X(3, 512, 1, 4)

// Dispatch of one storage type over the tile table.
template <int ST>
cudaError_t fused_launch_st(int lat, const FusedPlan &p, const StepArgs &a, const CUtensorMap &tm,
                            cudaStream_t s) {
#define SCLBM_X3(id, bx, by, ns) \
  case id:                       \
    return fused_launch_t<D3Q19, ST, bx, by, ns>(p, a, tm, s);
#define SCLBM_X2(id, bx, by, ns) \
  case id:                       \
    return fused_launch_t<D2Q9, ST, bx, by, ns>(p, a, tm, s);
  if (lat == D3Q19) {
    switch (p.tile) { SCLBM_D3Q19_TILES(SCLBM_X3) }
  } else {
    switch (p.tile) { SCLBM_D2Q9_TILES(SCLBM_X2) }
  }
#undef SCLBM_X3
#undef SCLBM_X2
  return cudaErrorInvalidValue;
}

template <int ST>
cudaError_t fused_prepare_st(int lat, const FusedPlan &p) {
#define SCLBM_X3(id, bx, by, ns) \
  case id:                       \
    return fused_prepare_t<D3Q19, ST, bx, by, ns>();
#define SCLBM_X2(id, bx, by, ns) \
  case id:                       \
    return fused_prepare_t<D2Q9, ST, bx, by, ns>();
  if (lat == D3Q19) {
    switch (p.tile) { SCLBM_D3Q19_TILES(SCLBM_X3) }
  } else {
    switch (p.tile) { SCLBM_D2Q9_TILES(SCLBM_X2) }
  }
#undef SCLBM_X3
#undef SCLBM_X2
  return cudaErrorInvalidValue;
}

}  // namespace sclbm
