// Temporal blocking of the ensemble's D2Q9 FP32 step: one CTA takes a tile
// of TX x TZ cells of one domain through S time steps in shared memory.
//
// The step of Sec. 3.1 (psi of the density, the Shan-Chen force from the
// psi of the eight neighbours, BGK relaxation with the velocity shift, push
// streaming by one cell) makes a cell's new populations depend on cells at
// most two away: its pushing neighbours (one) and their psi neighbours
// (two).  So the CTA loads its tile with a halo of H = 2 S cells (periodic),
// and at step s (0-based) the populations are valid on the cells at least
// 2 s from the loaded region's edge: psi is formed there, the cells one
// further in collide and push into the other buffer, and after S steps the
// tile itself is valid and is stored.  A launch reads one lattice and
// writes the other, as a single step does.
//
// The per-cell arithmetic is the fused march's FP32 offset path, operation
// for operation (pair sums of opposite populations, the same FMA and
// fast-division forms), so the populations are bit-identical to those of S
// single-step launches.  Shared memory: two population buffers and a psi
// plane of the loaded region, 19 floats per cell.
#pragma once

#include "lattice.cuh"

namespace sclbm {

template <int TX_, int TZ_, int S_>
struct EnsTB {
  static constexpr int TX = TX_, TZ = TZ_, S = S_;
  static constexpr int H = 2 * S;  // halo cells on every side
  static constexpr int RX = TX + 2 * H, RZ = TZ + 2 * H, RC = RX * RZ;
  static constexpr int SMEM = (2 * 9 + 1) * RC * (int)sizeof(float);
};

// What one temporally blocked tile needs from its domain record.
struct TbDomain {
  int NX, NZ;
  int64_t px, popstride;
  float tau, omega, G, rho0, inv_rho0, rho_ref;
  const float *in;
  float *out;
};

// 4-byte asynchronous global -> shared copy (completes at cp_async_wait_all)
__device__ __forceinline__ void cp_async_4(float *dst, const float *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

template <class K, int NT>
__device__ __forceinline__ void ens_tb_tile(const TbDomain &D, int x0, int z0) {
  using L = Lattice<D2Q9>;
  constexpr int RX = K::RX, RZ = K::RZ, RC = K::RC, H = K::H, S = K::S;
  extern __shared__ float tb_smem[];
  float *cur = tb_smem, *nxt = tb_smem + 9 * RC, *psi = tb_smem + 18 * RC;
  const int tid = threadIdx.x;
  const int NX = D.NX, NZ = D.NZ;

  // the loaded region: cells (x0 - H .. x0 + TX + H - 1) x (z0 - H ..),
  // wrapped; every copy is issued before the first is waited for
  for (int r = tid; r < RC; r += NT) {
    const int rz = r / RX, rx = r - rz * RX;
    int gx = x0 - H + rx, gz = z0 - H + rz;
    while (gx < 0) gx += NX;
    while (gx >= NX) gx -= NX;
    while (gz < 0) gz += NZ;
    while (gz >= NZ) gz -= NZ;
    const float *src = D.in + gz * D.px + gx;
#pragma unroll
    for (int i = 0; i < 9; ++i) cp_async_4(cur + i * RC + r, src + i * D.popstride);
  }
  cp_async_wait_all();

  // the fused march's FP32 constants
  const float G = D.G, tau = D.tau, omega = D.omega, rho0 = D.rho0, inv_rho0 = D.inv_rho0;
  const float rho_ref = D.rho_ref;
  const float om1 = 1.0f - omega;
  float cW[2], c3[2], c45[2];
#pragma unroll
  for (int k2 = 0; k2 < 2; ++k2) {
    const float w = (float)L::w(L::rep(k2 == 0 ? 0 : L::NP - 1));
    cW[k2] = w * omega;
    c3[k2] = 3.0f * w * omega;
    c45[k2] = 4.5f * w * omega;
  }
  __syncthreads();

  // steps unrolled, so that each phase runs over exactly its window with
  // compile-time extents
  static_for<S>([&](auto sc) {
    constexpr int s = decltype(sc)::value;
    // ---- psi on the valid cells [2s, R - 2s)
    {
      constexpr int lo = 2 * s, wx = RX - 4 * s, wz = RZ - 4 * s;
      for (int c = tid; c < wx * wz; c += NT) {
        const int cz = c / wx;
        const int r = (lo + cz) * RX + lo + (c - cz * wx);
        float2 s2;
        static_for<L::NP>([&](auto kc) {
          constexpr int k2 = decltype(kc)::value, i = L::rep(k2), o = L::opp(i);
          const float2 v = make_float2(cur[i * RC + r], cur[o * RC + r]);
          s2 = k2 == 0 ? v : __fadd2_rn(s2, v);
        });
        const float rho = (s2.x + s2.y) + cur[r];
        psi[r] = psi_of(rho_ref + rho, rho0, inv_rho0);
      }
    }
    __syncthreads();
    // ---- collide the cells [2s + 1, R - 2s - 1) and push into nxt
    {
      constexpr int lo = 2 * s + 1, wx = RX - 4 * s - 2, wz = RZ - 4 * s - 2;
      for (int c = tid; c < wx * wz; c += NT) {
        const int cz = c / wx;
        const int r = (lo + cz) * RX + lo + (c - cz * wx);
        float2 cur2[L::NP];
        float2 s2;
        static_for<L::NP>([&](auto kc) {
          constexpr int k2 = decltype(kc)::value, i = L::rep(k2), o = L::opp(i);
          cur2[k2] = make_float2(cur[i * RC + r], cur[o * RC + r]);
          s2 = k2 == 0 ? cur2[k2] : __fadd2_rn(s2, cur2[k2]);
        });
        const float R = (s2.x + s2.y) + cur[r];
        auto psi_at = [&](int i) -> float { return psi[r + L::cz(i) * RX + L::cx(i)]; };
        float jx = -0.0f, jy = -0.0f, jz = -0.0f, sx = -0.0f, sy = -0.0f, sz = -0.0f;
        static_for<L::NP>([&](auto kc) {
          constexpr int k2 = decltype(kc)::value, i = L::rep(k2), o = L::opp(i);
          constexpr int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
          const float d = cur2[k2].x - cur2[k2].y;
          jx = cacc<cx>(jx, d);
          jy = cacc<cy>(jy, d);
          jz = cacc<cz>(jz, d);
          const float dps = psi_at(i) - psi_at(o), w = (float)L::w(i);
          sx = cfma<cx>(sx, w, dps);
          sy = cfma<cy>(sy, w, dps);
          sz = cfma<cz>(sz, w, dps);
        });
        const float rho = rho_ref + R;
        const float gp = -G * psi[r];
        const float ir = __fdividef(1.0f, rho);
        const float ux = (jx + tau * (gp * sx)) * ir, uy = (jy + tau * (gp * sy)) * ir,
                    uz = (jz + tau * (gp * sz)) * ir;
        const float Kc = fmaf(rho * -1.5f, ux * ux + uy * uy + uz * uz, R);
        const float wK[2] = {cW[0] * Kc, cW[1] * Kc};
        const float2 om1_2 = make_float2(om1, om1);
        float2 moved2;
        static_for<L::NP>([&](auto kc) {
          constexpr int k2 = decltype(kc)::value, i = L::rep(k2), o = L::opp(i);
          constexpr int wc = L::w(i) == L::w(L::rep(0)) ? 0 : 1;
          const float cu = cdot<L::cx(i), L::cy(i), L::cz(i)>(ux, uy, uz);
          const float a = rho * cu;
          const float A = fmaf(a, c45[wc] * cu, wK[wc]);
          const float B = c3[wc] * a;
          const float2 g = __ffma2_rn(om1_2, cur2[k2], make_float2(A + B, A - B));
          moved2 = k2 == 0 ? g : __fadd2_rn(moved2, g);
          nxt[i * RC + r + L::cz(i) * RX + L::cx(i)] = g.x;
          nxt[o * RC + r + L::cz(o) * RX + L::cx(o)] = g.y;
        });
        nxt[r] = R - (moved2.x + moved2.y);
      }
    }
    __syncthreads();
    float *t = cur;
    cur = nxt;
    nxt = t;
  });

  // ---- store the tile (valid after S steps), clipped to the domain
  for (int c = tid; c < 9 * K::TZ * K::TX; c += NT) {
    const int i = c / (K::TZ * K::TX), r = c - i * (K::TZ * K::TX);
    const int iz = r / K::TX, ix = r - iz * K::TX;
    const int gx = x0 + ix, gz = z0 + iz;
    if (gx < NX && gz < NZ)
      D.out[i * D.popstride + gz * D.px + gx] = cur[i * RC + (H + iz) * RX + H + ix];
  }
}

}  // namespace sclbm
