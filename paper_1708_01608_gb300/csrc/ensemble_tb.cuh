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
// The per-cell arithmetic is the fused marches' FP32 offset path, operation
// for operation (the same density order, FMA and fast-division forms), so the
// populations are bit-identical to those of S single-step launches.  Shared
// memory: two population buffers and a psi plane of the loaded region, 19
// floats per cell.
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

// Paired FP32 operations over two cells (vertical neighbours), each lane the
// scalar operation of the one-cell march
__device__ __forceinline__ float2 tb_f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 tb_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as a + (-b): negation is exact, so the lanes are the scalar a - b
__device__ __forceinline__ float2 tb_sub(float2 a, float2 b) {
  return __fadd2_rn(a, make_float2(-b.x, -b.y));
}
__device__ __forceinline__ float2 tb_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 tb_fma(float2 a, float2 b, float2 c) {
  return __ffma2_rn(a, b, c);
}
// acc + c v for a velocity component c in {-1, 0, 1} (cacc per lane)
template <int CC>
__device__ __forceinline__ float2 tb_acc(float2 acc, float2 v) {
  if constexpr (CC > 0) return tb_add(acc, v);
  else if constexpr (CC < 0) return tb_sub(acc, v);
  else return acc;
}
// acc + c w v (cfma per lane)
template <int CC>
__device__ __forceinline__ float2 tb_cfma(float2 acc, float w, float2 v) {
  if constexpr (CC > 0) return tb_fma(tb_f2(w), v, acc);
  else if constexpr (CC < 0) return tb_fma(tb_f2(-w), v, acc);
  else return acc;
}
// density of two cells in the x-pair kernel's order (rho_chain per lane)
template <class Ld>
__device__ __forceinline__ float2 tb_rho(Ld g) {
  float2 a = g(0), b = g(1);
#pragma unroll
  for (int i = 2; i + 1 < 9; i += 2) {
    a = tb_add(a, g(i));
    b = tb_add(b, g(i + 1));
  }
  a = tb_add(a, g(8));
  return tb_add(a, b);
}
// c.u (cdot per lane)
template <int A, int B, int Z>
__device__ __forceinline__ float2 tb_dot(float2 x, float2 y, float2 z) {
  float2 r;
  if constexpr (A != 0) r = A > 0 ? x : make_float2(-x.x, -x.y);
  else if constexpr (B != 0) r = B > 0 ? y : make_float2(-y.x, -y.y);
  else r = Z > 0 ? z : make_float2(-z.x, -z.y);
  if constexpr (A != 0 && B != 0) r = B > 0 ? tb_add(r, y) : tb_sub(r, y);
  if constexpr ((A != 0 || B != 0) && Z != 0) r = Z > 0 ? tb_add(r, z) : tb_sub(r, z);
  return r;
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
    // ---- psi on the valid cells [2s, R - 2s), two cells (rows r, r + RX)
    // per thread; wz is even
    {
      constexpr int lo = 2 * s, wx = RX - 4 * s, wz = RZ - 4 * s;
      static_assert(wz % 2 == 0, "windows hold whole pairs of rows");
      for (int c = tid; c < wx * (wz / 2); c += NT) {
        const int pz = c / wx;
        const int r = (lo + 2 * pz) * RX + lo + (c - pz * wx);
        auto g = [&](int i) { return make_float2(cur[i * RC + r], cur[i * RC + r + RX]); };
        const float2 rho = tb_rho(g);
        psi[r] = psi_of(rho_ref + rho.x, rho0, inv_rho0);
        psi[r + RX] = psi_of(rho_ref + rho.y, rho0, inv_rho0);
      }
    }
    __syncthreads();
    // ---- collide the cells [2s + 1, R - 2s - 1) and push into nxt, two
    // cells per thread
    {
      constexpr int lo = 2 * s + 1, wx = RX - 4 * s - 2, wz = RZ - 4 * s - 2;
      static_assert(wz % 2 == 0, "windows hold whole pairs of rows");
      for (int c = tid; c < wx * (wz / 2); c += NT) {
        const int pz = c / wx;
        const int r = (lo + 2 * pz) * RX + lo + (c - pz * wx);
        auto g = [&](int i) { return make_float2(cur[i * RC + r], cur[i * RC + r + RX]); };
        auto psi2 = [&](int i) {
          const int q = r + L::cz(i) * RX + L::cx(i);
          return make_float2(psi[q], psi[q + RX]);
        };
        float2 gI[L::NP], gO[L::NP];
        static_for<L::NP>([&](auto kc) {
          constexpr int k2 = decltype(kc)::value, i = L::rep(k2), o = L::opp(i);
          gI[k2] = g(i);
          gO[k2] = g(o);
        });
        const float2 R = tb_rho(g);
        float2 jx = tb_f2(-0.0f), jy = tb_f2(-0.0f), jz = tb_f2(-0.0f);
        float2 sx = tb_f2(-0.0f), sy = tb_f2(-0.0f), sz = tb_f2(-0.0f);
        static_for<L::NP>([&](auto kc) {
          constexpr int k2 = decltype(kc)::value, i = L::rep(k2), o = L::opp(i);
          constexpr int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
          const float2 d = tb_sub(gI[k2], gO[k2]);
          jx = tb_acc<cx>(jx, d);
          jy = tb_acc<cy>(jy, d);
          jz = tb_acc<cz>(jz, d);
          const float2 dps = tb_sub(psi2(i), psi2(o));
          const float w = (float)L::w(i);
          sx = tb_cfma<cx>(sx, w, dps);
          sy = tb_cfma<cy>(sy, w, dps);
          sz = tb_cfma<cz>(sz, w, dps);
        });
        const float2 rho = tb_add(tb_f2(rho_ref), R);
        const float2 gp = tb_mul(tb_f2(-G), make_float2(psi[r], psi[r + RX]));
        const float2 ir = make_float2(__fdividef(1.0f, rho.x), __fdividef(1.0f, rho.y));
        const float2 ux = tb_mul(tb_fma(tb_f2(tau), tb_mul(gp, sx), jx), ir);
        const float2 uy = tb_mul(tb_fma(tb_f2(tau), tb_mul(gp, sy), jy), ir);
        const float2 uz = tb_mul(tb_fma(tb_f2(tau), tb_mul(gp, sz), jz), ir);
        const float2 Kc =
            tb_fma(tb_mul(rho, tb_f2(-1.5f)), tb_fma(uz, uz, tb_fma(uy, uy, tb_mul(ux, ux))), R);
        const float2 wK[2] = {tb_mul(tb_f2(cW[0]), Kc), tb_mul(tb_f2(cW[1]), Kc)};
        float2 m = tb_f2(-0.0f);  // sum over the pairs of (g_i + g_o)
        static_for<L::NP>([&](auto kc) {
          constexpr int k2 = decltype(kc)::value, i = L::rep(k2), o = L::opp(i);
          constexpr int wc = L::w(i) == L::w(L::rep(0)) ? 0 : 1;
          const float2 cu = tb_dot<L::cx(i), L::cy(i), L::cz(i)>(ux, uy, uz);
          const float2 a = tb_mul(rho, cu);
          const float2 A = tb_fma(a, tb_mul(tb_f2(c45[wc]), cu), wK[wc]);
          const float2 gi = tb_fma(tb_f2(om1), gI[k2], tb_fma(tb_f2(c3[wc]), a, A));
          const float2 go = tb_fma(tb_f2(om1), gO[k2], tb_fma(tb_f2(-c3[wc]), a, A));
          m = tb_add(m, tb_add(gi, go));
          const int di = i * RC + r + L::cz(i) * RX + L::cx(i);
          const int dq = o * RC + r + L::cz(o) * RX + L::cx(o);
          nxt[di] = gi.x;
          nxt[di + RX] = gi.y;
          nxt[dq] = go.x;
          nxt[dq + RX] = go.y;
        });
        const float2 g0 = tb_sub(R, m);
        nxt[r] = g0.x;
        nxt[r + RX] = g0.y;
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
