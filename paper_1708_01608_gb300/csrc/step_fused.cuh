// Fused Shan-Chen collide-stream-force step (one kernel per time step).
//
// Populations are stored in push form: stored_i(x) = f_i(x, t), the value
// that has arrived at x.  A CTA owns a BX x BY column of the lattice (x, y)
// and marches along z through a chunk of planes.  For every plane P it
// stages, with TMA, the populations of the column and of its one-cell halo
// ring: one 4-D box {BX, BY, 1, Q} for the column (all Q populations in one
// copy), boxes of HX columns for the left and right halo, one-row boxes for
// the top and bottom halo and four corner boxes.  Each halo box is addressed
// with already-wrapped coordinates, so periodic seams need no special case;
// x boxes start on 16-byte boundaries (HX = 16 bytes of elements), which is
// why the fused path needs nx to be a multiple of HX.
//
// From the staged plane it computes rho and psi of the column and halo into
// a ring of four psi planes in shared memory; the interior cells'
// populations stay in registers, and one iteration later the plane is
// collided with psi of the planes above and below already in the ring.  The
// post-collision populations are pushed to x + c_i with plain coalesced
// stores.  Each population is read from HBM once and written once per step;
// halo boxes are re-read from L2.
//
// Every wait on a TMA transaction is bounded (1 s); on timeout the CTA sets
// ERR_TMA_TIMEOUT in the status word, waits (bounded) for its other copies
// and returns without writing further planes.
#pragma once

#include <climits>
#include <type_traits>

#include "internal.h"
#include "lattice.cuh"

namespace sclbm {

constexpr int round128(int b) { return (b + 127) / 128 * 128; }

template <int LAT, int ST, int BX_, int BY_, int NS_>
struct FusedK {
  using L = Lattice<LAT>;
  using S = Storage<ST>;
  using T = typename S::T;
  using C = typename S::C;
  static constexpr int BX = BX_, BY = BY_, NS = NS_;
  static constexpr int Q = L::Q;
  static constexpr int HY = L::HAS_Y ? 1 : 0;
  static constexpr int SZ = (int)sizeof(T);
  static constexpr int HX = 16 / SZ;  // halo columns loaded (one is used)
  // staged boxes of one plane, each at a 128-byte aligned offset
  static constexpr int MAIN_B = BX * BY * Q * SZ;  // [Q][BY][BX]
  static constexpr int COL_B = HX * BY * Q * SZ;   // [Q][BY][HX]
  static constexpr int ROW_B = BX * Q * SZ;        // [Q][BX]
  static constexpr int CRN_B = HX * Q * SZ;        // [Q][HX]
  static constexpr int OFF_L = round128(MAIN_B);
  static constexpr int OFF_R = OFF_L + round128(COL_B);
  static constexpr int OFF_T = OFF_R + round128(COL_B);
  static constexpr int OFF_B = OFF_T + (HY ? round128(ROW_B) : 0);
  static constexpr int OFF_TL = OFF_B + (HY ? round128(ROW_B) : 0);
  static constexpr int OFF_TR = OFF_TL + (HY ? round128(CRN_B) : 0);
  static constexpr int OFF_BL = OFF_TR + (HY ? round128(CRN_B) : 0);
  static constexpr int OFF_BR = OFF_BL + (HY ? round128(CRN_B) : 0);
  static constexpr int STAGE_BYTES = OFF_BR + (HY ? round128(CRN_B) : 0);
  static constexpr int TX_BYTES = MAIN_B + 2 * COL_B + (HY ? 2 * ROW_B + 4 * CRN_B : 0);
  static constexpr int PW = BX + 2;
  static constexpr int PH = BY + 2 * HY;
  static constexpr int RING_BYTES = (4 * PW * PH * (int)sizeof(C) + 15) / 16 * 16;
  static constexpr int NT = BX * BY;
  static constexpr int SMEM = NS * STAGE_BYTES + RING_BYTES + NS * 8 + 128;
  static_assert(BX <= 256 && BY <= 256 && Q <= 256, "TMA box dimensions are limited to 256");
  static_assert(BX % HX == 0, "tiles must start on 16-byte boundaries");
  static_assert(STAGE_BYTES % 128 == 0, "TMA destinations must be 128-byte aligned");
};

// What one CTA's march needs: lattice extents, constants, the TMA
// descriptors of the input lattice, its column and z chunk, its injection
// sites (sorted by z), and the status word.
struct MarchArgs {
  int NX, NY, NZ;
  int64_t px;
  double tau, G, rho0;  // FP64 arithmetic
  float tau_f, omega_f, G_f, rho0_f, inv_rho0_f, rho_ref_f;
  const FusedMaps *tm;
  int x0, y0, zs, ze;
  int32_t nsites;
  int sp, send;
  const int32_t *site_x, *site_y, *site_z, *bucket_site;
  const double *rate;
  double *budget;
  int *err;
  int debug_flags;
  float *resid;  // rounding residual per cell (16-bit residual forms), else NULL
};

// Once per CTA, before its first march: the NS stage barriers and the
// descriptor prefetch.  K gives the shared-memory layout (stages, then the
// psi ring, then the barriers).
template <class K>
__device__ __forceinline__ void fused_barriers_init_k(const MarchArgs &m) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + K::NS * K::STAGE_BYTES + K::RING_BYTES);
  if (threadIdx.x == 0) {
    for (int s = 0; s < K::NS; ++s) mbar_init(&bars[s], 1);
    fence_barrier_init();
    fence_proxy_async_smem();
    prefetch_tmap(&m.tm->main);
    prefetch_tmap(&m.tm->col);
    if (K::HY) {
      prefetch_tmap(&m.tm->row);
      prefetch_tmap(&m.tm->crn);
    }
  }
  __syncthreads();
}
template <int LAT, int ST, int BX, int BY, int NS>
__device__ __forceinline__ void fused_barriers_init(const MarchArgs &m) {
  fused_barriers_init_k<FusedK<LAT, ST, BX, BY, NS>>(m);
}

// Sum of the Q staged values of one cell in the order of the x-pair kernel's
// sum_q (even indices and odd indices in two chains, then their sum), so that
// the one-cell and the x-pair kernels give a cell the same density bits.
template <int Q, class Ld>
__device__ __forceinline__ float rho_chain(Ld ld) {
  float a = ld(0), b = ld(1);
#pragma unroll
  for (int i = 2; i + 1 < Q; i += 2) {
    a = a + ld(i);
    b = b + ld(i + 1);
  }
  if constexpr (Q % 2 == 1) a = a + ld(Q - 1);
  return a + b;
}

// The march of one CTA over planes zs..ze-1 of one column: TMA staging, psi
// ring, collision, push.  out_pop(i) returns the base of population i of the
// output lattice.  kb counts the planes this CTA staged before (stage slot
// and barrier phase continue across marches); it advances by the planes
// staged here.  Returns false after a TMA wait timed out.
template <int LAT, int ST, int BX, int BY, int NS, class OutPop>
__device__ __forceinline__ bool fused_march(const MarchArgs &m, OutPop out_pop, uint32_t &kb) {
  using K = FusedK<LAT, ST, BX, BY, NS>;
  using L = typename K::L;
  using S = typename K::S;
  using T = typename K::T;
  using C = typename K::C;
  constexpr int Q = K::Q, HY = K::HY, HX = K::HX, PW = K::PW, PH = K::PH, NT = K::NT;
  constexpr bool F64 = sizeof(C) == 8;
  // 16-bit residual forms: the cell's rounding residual of the last step
  // joins its mass R, and the new one is what this step's stores round off
  constexpr bool RESID = S::RESID;

  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
  C *ring = reinterpret_cast<C *>(smem + NS * K::STAGE_BYTES);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + NS * K::STAGE_BYTES + K::RING_BYTES);

  const int tid = threadIdx.x;
  const int tx = tid % BX, ty = tid / BX;
  const int NX = m.NX, NY = m.NY, NZ = m.NZ;
  const int x0 = m.x0, y0 = m.y0, zs = m.zs, ze = m.ze;
  const int BXe = min(BX, NX - x0), BYe = min(BY, NY - y0);
  if (zs >= ze) return true;
  const int NPL = ze - zs + 2;  // staged planes zs-1 .. ze
  const bool active = tx < BXe && ty < BYe;
  // wrapped coordinates of the halo boxes
  const int xl = x0 == 0 ? NX - HX : x0 - HX;
  const int xr = x0 + BXe == NX ? 0 : x0 + BXe;
  const int yt = y0 == 0 ? NY - 1 : y0 - 1;
  const int yb = y0 + BYe == NY ? 0 : y0 + BYe;

  const int64_t plane = m.px * NY;

  // constants in the arithmetic type (FP32 kernels execute no FP64 at all)
  const C G = F64 ? (C)m.G : (C)m.G_f, tau = F64 ? (C)m.tau : (C)m.tau_f,
          omega = F64 ? (C)(1.0 / m.tau) : (C)m.omega_f, rho0 = F64 ? (C)m.rho0 : (C)m.rho0_f,
          inv_rho0 = F64 ? (C)(1.0 / m.rho0) : (C)m.inv_rho0_f;
  // offset storage: the staged values are g_i = f_i - w_i rho_ref
  const C rho_ref = S::OFFSET ? (C)m.rho_ref_f : (C)0;

  const uint32_t k0 = kb;
  auto issue = [&](int k) {
    if ((m.debug_flags & 1) && k == 1) return;  // test hook: let the wait expire
    const int P = zs - 1 + k, s = (int)((k0 + k) % NS);
    const int zp = P < 0 ? P + NZ : (P >= NZ ? P - NZ : P);
    uint8_t *st = smem + s * K::STAGE_BYTES;
    mbar_arrive_expect_tx(&bars[s], (uint32_t)K::TX_BYTES);
    tma_load_4d(st, &m.tm->main, x0, y0, zp, 0, &bars[s]);
    tma_load_4d(st + K::OFF_L, &m.tm->col, xl, y0, zp, 0, &bars[s]);
    tma_load_4d(st + K::OFF_R, &m.tm->col, xr, y0, zp, 0, &bars[s]);
    if (HY) {
      tma_load_4d(st + K::OFF_T, &m.tm->row, x0, yt, zp, 0, &bars[s]);
      tma_load_4d(st + K::OFF_B, &m.tm->row, x0, yb, zp, 0, &bars[s]);
      tma_load_4d(st + K::OFF_TL, &m.tm->crn, xl, yt, zp, 0, &bars[s]);
      tma_load_4d(st + K::OFF_TR, &m.tm->crn, xr, yt, zp, 0, &bars[s]);
      tma_load_4d(st + K::OFF_BL, &m.tm->crn, xl, yb, zp, 0, &bars[s]);
      tma_load_4d(st + K::OFF_BR, &m.tm->crn, xr, yb, zp, 0, &bars[s]);
    }
  };
  if (tid == 0) {
    for (int k = 0; k < NS && k < NPL; ++k) issue(k);
  }

  // This CTA's injection sites [sp, send), sorted by z.  The next one is
  // held in registers (plane, cell, rate and budget: only this CTA changes
  // the budgets of its sites during the step), so that a site plane costs
  // no dependent global loads.
  int sp = m.sp;
  const int send = m.send;
  int next_z = INT_MAX, site_x = 0, site_y = 0, site_i = 0;
  double site_rate = 0.0, site_budget = 0.0;
  auto load_site = [&]() {
    if (sp < send) {
      site_i = m.bucket_site[sp];
      next_z = m.site_z[site_i];
      site_x = m.site_x[site_i];
      site_y = m.site_y[site_i];
      site_rate = m.rate[site_i];
      site_budget = m.budget[site_i];
    } else {
      next_z = INT_MAX;
    }
  };
  load_site();

  // destination coordinates of the push, fixed per thread (periodic)
  const int x = x0 + tx, y = y0 + ty;
  const int xm = x == 0 ? NX - 1 : x - 1, xp = x + 1 >= NX ? 0 : x + 1;
  const int ym = y == 0 ? NY - 1 : y - 1, yp = y + 1 >= NY ? 0 : y + 1;

  // The halo cell this thread computes psi for (at most one: nhalo <= NT),
  // as a byte offset of its population 0 inside a stage, the element
  // distance between populations and its slot in a psi plane.
  const int nhalo = HY ? 2 * (BXe + 2) + 2 * BYe : 2;
  int h_off = 0, h_pstride = 0, h_slot = 0;
  if (tid < nhalo) {
    int dx, dy;
    const int h = tid;
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
    const int cxr = dx < 0 ? 0 : (dx >= BXe ? 2 : 1);
    const int cyr = dy < 0 ? 0 : (dy >= BYe ? 2 : 1);
    int off, e;
    if (cyr == 1) {
      if (cxr == 1) {
        off = 0;
        e = dy * BX + dx;
        h_pstride = BY * BX;
      } else {
        off = cxr == 0 ? K::OFF_L : K::OFF_R;
        e = dy * HX + (cxr == 0 ? HX - 1 : 0);
        h_pstride = BY * HX;
      }
    } else if (cxr == 1) {
      off = cyr == 0 ? K::OFF_T : K::OFF_B;
      e = dx;
      h_pstride = BX;
    } else {
      off = cyr == 0 ? (cxr == 0 ? K::OFF_TL : K::OFF_TR) : (cxr == 0 ? K::OFF_BL : K::OFF_BR);
      e = cxr == 0 ? HX - 1 : 0;
      h_pstride = HX;
    }
    h_off = off + e * (int)sizeof(T);
    h_slot = (dy + HY) * PW + dx + 1;
  }
  static_assert(!HY || 2 * (BX + 2) + 2 * BY <= NT, "one halo cell per thread at most");

  // 32-bit offsets of the push destinations inside a population block
  const int32_t ox[3] = {xm, x, xp};
  const int32_t oy[3] = {(int32_t)(ym * m.px), (int32_t)(y * m.px), (int32_t)(yp * m.px)};

  // The staged values of this thread's cell: FP64 keeps them per velocity;
  // the FP32 path keeps the opposite pairs (i, opp(i)) as float2 so that
  // their sums and relaxations run as paired FP32 instructions.
  C cur[Q], nxt[Q];
  float2 cur2[L::NP], nxt2[L::NP];
  float cur0 = 0.0f, nxt0 = 0.0f;
  if constexpr (F64) {
#pragma unroll
    for (int i = 0; i < Q; ++i) cur[i] = nxt[i] = 0;
  } else {
#pragma unroll
    for (int k2 = 0; k2 < L::NP; ++k2) cur2[k2] = nxt2[k2] = make_float2(0.0f, 0.0f);
  }
  C Rcur = 0, Rnxt = 0;  // sum of the staged values of this thread's cell

  // FP32 relaxation constants per weight class (omega folded in)
  C om1 = (C)1 - omega, cW[2], c3[2], c45[2];
#pragma unroll
  for (int k2 = 0; k2 < 2; ++k2) {
    const C w = (C)L::w(L::rep(k2 == 0 ? 0 : L::NP - 1));
    cW[k2] = w * omega;
    c3[k2] = (C)3 * w * omega;
    c45[k2] = (C)4.5 * w * omega;
  }

  // two planes per iteration where registers allow (512-thread tiles): the
  // staged values then change register sets instead of being copied
  constexpr int UNROLL = NT > 256 ? 2 : 1;
#pragma unroll UNROLL
  for (int k = 0; k < NPL; ++k) {
    const int s = (int)((k0 + k) % NS);
    const int P = zs - 1 + k;
    const bool ok = mbar_wait_bounded(&bars[s], ((k0 + k) / NS) & 1u, 1000000000ull);
    const uint8_t *st = smem + s * K::STAGE_BYTES;
    const T *mainb = reinterpret_cast<const T *>(st);

    // ---- psi of plane P for the column and its halo ring
    C *rk = ring + (k & 3) * PW * PH;
    if (active) {
      C rho = 0;
      if constexpr (F64) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const C v = S::load(mainb[(i * BY + ty) * BX + tx]);
          nxt[i] = v;
          rho += v;
        }
      } else {
        static_for<L::NP>([&](auto kc) {
          constexpr int k2 = decltype(kc)::value, i = L::rep(k2), o = L::opp(i);
          nxt2[k2] = make_float2(S::load(mainb[(i * BY + ty) * BX + tx]),
                                 S::load(mainb[(o * BY + ty) * BX + tx]));
        });
        nxt0 = S::load(mainb[ty * BX + tx]);
        rho = rho_chain<Q>([&](int i) { return S::load(mainb[(i * BY + ty) * BX + tx]); });
      }
      rk[(ty + HY) * PW + tx + 1] = psi_of(rho_ref + rho, rho0, inv_rho0);
      Rnxt = rho;
    }
    if (tid < nhalo) {
      const T *b = reinterpret_cast<const T *>(st + h_off);
      C rho = 0;
      if constexpr (F64) {
#pragma unroll
        for (int i = 0; i < Q; ++i) rho += S::load(b[i * h_pstride]);
      } else {
        rho = rho_chain<Q>([&](int i) { return S::load(b[i * h_pstride]); });
      }
      rk[h_slot] = psi_of(rho_ref + rho, rho0, inv_rho0);
    }

    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        if (m.err) atomicOr(m.err, ERR_TMA_TIMEOUT);
        // wait (bounded) for copies still in flight into this CTA's stages
        for (int k2 = k + 1; k2 < NPL && k2 < k + NS; ++k2)
          mbar_wait_bounded(&bars[(k0 + k2) % NS], ((k0 + k2) / NS) & 1u, 100000000ull);
      }
      return false;
    }
    if (tid == 0 && k + NS < NPL) issue(k + NS);

    // ---- collide plane P - 1 (needs psi of P - 2, P - 1, P) and push
    if (k >= 2) {
      const int Pc = P - 1;
      C dmc = 0;  // blowing-agent mass deposited in this cell this step
      bool site = false;
      if (Pc == next_z) {  // sites of this CTA in this plane (rare)
        double dm = 0.0;
        while (next_z == Pc) {
          if (active && site_x == x && site_y == y && site_budget > 0.0) {
            const double d = fmin(site_rate, site_budget);
            m.budget[site_i] = site_budget - d;
            dm += d;
            site = true;
          }
          ++sp;
          load_site();
        }
        dmc = (C)dm;
      }
      if (active) {
        const C *pm = ring + ((k - 2) & 3) * PW * PH;
        const C *p0 = ring + ((k - 1) & 3) * PW * PH;
        const C *pp = ring + (k & 3) * PW * PH;
        const int c0 = (ty + HY) * PW + tx + 1;
        const int zm = Pc == 0 ? NZ - 1 : Pc - 1, zp = Pc + 1 >= NZ ? 0 : Pc + 1;
        const int32_t oz[3] = {(int32_t)(zm * plane), (int32_t)(Pc * plane), (int32_t)(zp * plane)};
        auto dst = [&](int i) -> T * {
          return out_pop(i) + (oz[L::cz(i) + 1] + oy[L::cy(i) + 1] + ox[L::cx(i) + 1]);
        };
        auto psi_at = [&](int i) -> C {
          const C *pl = L::cz(i) < 0 ? pm : (L::cz(i) > 0 ? pp : p0);
          return pl[c0 + L::cy(i) * PW + L::cx(i)];
        };
        if constexpr (F64) {
          // FP64: the oracle's operation order, velocity by velocity
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
            const C wp = (C)L::w(i) * psi_at(i);
            sx += (C)L::cx(i) * wp;
            sy += (C)L::cy(i) * wp;
            sz += (C)L::cz(i) * wp;
          }
          const C gp = -G * p0[c0];
          const C ux = (jx + tau * (gp * sx)) / rho, uy = (jy + tau * (gp * sy)) / rho,
                  uz = (jz + tau * (gp * sz)) / rho;
          const C uu = (C)1.5 * (ux * ux + uy * uy + uz * uz);
#pragma unroll
          for (int i = 0; i < Q; ++i) {
            const C cu = (C)L::cx(i) * ux + (C)L::cy(i) * uy + (C)L::cz(i) * uz;
            const C feq = (C)L::w(i) * rho * ((C)1 + (C)3 * cu + (C)4.5 * cu * cu - uu);
            C fs = cur[i] - (cur[i] - feq) / tau;
            if (site) fs += L::w(i) * dmc;
            *dst(i) = S::store(fs);
          }
        } else {
          // FP32 on offsets g_i = f_i - w_i rho_ref: with R = sum g (so that
          // rho = rho_ref + R) the equilibrium offset is
          //   w_i (K + rho (3 c.u + 4.5 (c.u)^2)),  K = R - 1.5 rho u.u,
          // evaluated for opposite velocities in pairs, with omega = 1/tau
          // folded into the per-weight constants:
          //   g_i* = (1 - omega) g_i + omega w_i (K + 4.5 rho (c.u)^2) + omega 3 w_i rho c.u.
          // The rest population takes R minus the moving ones, so mass is
          // conserved to rounding.  The residual forms add the cell's
          // rounding residual of the last step to R and keep what this
          // step's 16-bit stores round off (deposit included) as the next
          // one, so stored mass plus residual is conserved to FP32 rounding.
          const int32_t own = oz[1] + oy[1] + ox[1];
          C R = Rcur;
          if constexpr (RESID) R += m.resid[own];
          // -0 is the additive identity, so the first term is no addition
          C jx = -0.0f, jy = -0.0f, jz = -0.0f, sx = -0.0f, sy = -0.0f, sz = -0.0f;
          static_for<L::NP>([&](auto kc) {
            constexpr int k2 = decltype(kc)::value, i = L::rep(k2), o = L::opp(i);
            constexpr int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
            const C d = cur2[k2].x - cur2[k2].y;
            jx = cacc<cx>(jx, d);
            jy = cacc<cy>(jy, d);
            jz = cacc<cz>(jz, d);
            const C dps = psi_at(i) - psi_at(o), w = (C)L::w(i);
            sx = cfma<cx>(sx, w, dps);
            sy = cfma<cy>(sy, w, dps);
            sz = cfma<cz>(sz, w, dps);
          });
          const C rho = rho_ref + R;
          const C gp = -G * p0[c0];
          const C ir = __fdividef((C)1, rho);
          // every FMA written out, so that the temporally blocked ensemble
          // kernel can repeat this arithmetic bit for bit
          const C ux = fmaf(tau, gp * sx, jx) * ir, uy = fmaf(tau, gp * sy, jy) * ir,
                  uz = fmaf(tau, gp * sz, jz) * ir;
          const C K = fmaf(rho * (C)-1.5, fmaf(uz, uz, fmaf(uy, uy, ux * ux)), R);
          const C wK[2] = {cW[0] * K, cW[1] * K};
          const float2 om1_2 = make_float2(om1, om1);
          // relax and push; SITE adds the blowing agent w_i dm to every
          // population of the cell (a separate copy of the loop, run only
          // by the site cell's warp)
          C racc = 0;
          auto put = [&](T *p, C v) {
            const T q = S::store(v);
            *p = q;
            if constexpr (RESID) racc += v - S::load(q);
          };
          auto relax_push = [&](auto with_site) {
            constexpr bool SITE = decltype(with_site)::value;
            C moved = -0.0f;  // sum over the pairs of (g_i + g_o), as the x-pair kernel
            static_for<L::NP>([&](auto kc) {
              constexpr int k2 = decltype(kc)::value, i = L::rep(k2), o = L::opp(i);
              constexpr int wc = L::w(i) == L::w(L::rep(0)) ? 0 : 1;
              const C cu = cdot<L::cx(i), L::cy(i), L::cz(i)>(ux, uy, uz);
              const C a = rho * cu;
              const C A = fmaf(a, c45[wc] * cu, wK[wc]);
              // (g_i, g_o) = (1 - omega) (g_i, g_o) + (A + B, A - B), B = c3 a,
              // with A +- B as FMAs: one paired FMA
              const float2 g = __ffma2_rn(
                  om1_2, cur2[k2], make_float2(fmaf(c3[wc], a, A), fmaf(-c3[wc], a, A)));
              moved = moved + (g.x + g.y);
              const C gi = g.x, go = g.y;
              if (SITE) {
                put(dst(i), gi + (C)L::w(i) * dmc);
                put(dst(o), go + (C)L::w(o) * dmc);
              } else {
                put(dst(i), gi);
                put(dst(o), go);
              }
            });
            const C g0 = R - moved;
            put(dst(0), SITE ? g0 + (C)L::w(0) * dmc : g0);
          };
          if (site)
            relax_push(std::true_type{});
          else
            relax_push(std::false_type{});
          if constexpr (RESID) m.resid[own] = racc;
        }
      }
    }
    if constexpr (F64) {
#pragma unroll
      for (int i = 0; i < Q; ++i) cur[i] = nxt[i];
    } else {
#pragma unroll
      for (int k2 = 0; k2 < L::NP; ++k2) cur2[k2] = nxt2[k2];
      cur0 = nxt0;
    }
    Rcur = Rnxt;
  }
  kb = k0 + NPL;
  return true;
}

// The march of CTA blockIdx.x of a step launch: item = zc * tiles + tt.
__device__ __forceinline__ MarchArgs march_args_of(const FusedMaps &tm, const StepArgs &a,
                                                   int tiles_x, int tiles_y, int zlen, int BX,
                                                   int BY) {
  const int item = blockIdx.x;
  const int ntiles = tiles_x * tiles_y;
  const int zc = item / ntiles, tt = item % ntiles;
  MarchArgs m;
  m.NX = (int)a.NX;
  m.NY = (int)a.NY;
  m.NZ = (int)a.NZ;
  m.px = a.px;
  m.tau = a.tau;
  m.G = a.G;
  m.rho0 = a.rho0;
  m.tau_f = a.tau_f;
  m.omega_f = a.omega_f;
  m.G_f = a.G_f;
  m.rho0_f = a.rho0_f;
  m.inv_rho0_f = a.inv_rho0_f;
  m.rho_ref_f = a.rho_ref_f;
  m.tm = &tm;
  m.x0 = (tt % tiles_x) * BX;
  m.y0 = (tt / tiles_x) * BY;
  m.zs = zc * zlen;
  m.ze = min(m.NZ, m.zs + zlen);
  m.nsites = a.nsites;
  m.sp = a.nsites > 0 ? a.bucket_off[item] : 0;
  m.send = a.nsites > 0 ? a.bucket_off[item + 1] : 0;
  m.site_x = a.site_x;
  m.site_y = a.site_y;
  m.site_z = a.site_z;
  m.bucket_site = a.bucket_site;
  m.rate = a.rate;
  m.budget = a.budget;
  m.resid = a.resid;
  m.err = a.err;
  m.debug_flags = a.debug_flags;
  return m;
}

// One launch per time step: CTA (item) = BX x BY tile tt and z chunk zc,
// item = zc * tiles + tt, so the CTAs resident together cover neighbouring
// columns at the same planes (their halo rows meet in L2).
// 256-thread tiles are register-limited to 3 CTAs per SM, the larger ones run one
template <int LAT, int ST, int BX, int BY, int NS>
__global__ void __launch_bounds__(BX *BY, BX *BY <= 256 ? 3 : 1)
    fused_step_kernel(const __grid_constant__ FusedMaps tm, const StepArgs a, const int tiles_x,
                      const int tiles_y, const int zlen) {
  using T = typename Storage<ST>::T;
  const MarchArgs m = march_args_of(tm, a, tiles_x, tiles_y, zlen, BX, BY);
  fused_barriers_init<LAT, ST, BX, BY, NS>(m);
  // Programmatic dependent launch: the shared-memory set-up above overlaps
  // the previous step's tail.  Before the wait only the launch's own
  // read-only inputs are read (the injection buckets); the lattices and the
  // site budgets are touched only after the previous step has completed
  // and its writes are visible.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  uint32_t kb = 0;
  fused_march<LAT, ST, BX, BY, NS>(m, [&](int i) { return static_cast<T *>(a.out_pop[i]); }, kb);
}

template <int LAT, int ST, int BX, int BY, int NS>
cudaError_t fused_prepare_t(int *blocks_per_sm) {
  using K = FusedK<LAT, ST, BX, BY, NS>;
  cudaError_t e = cudaFuncSetAttribute(fused_step_kernel<LAT, ST, BX, BY, NS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM);
  if (e == cudaSuccess && blocks_per_sm)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        blocks_per_sm, fused_step_kernel<LAT, ST, BX, BY, NS>, K::NT, K::SMEM);
  return e;
}

template <int LAT, int ST, int BX, int BY, int NS>
cudaError_t fused_launch_t(const FusedPlan &p, const StepArgs &a, const FusedMaps &tm,
                           cudaStream_t s) {
  using K = FusedK<LAT, ST, BX, BY, NS>;
  // launched as a programmatic dependent of the previous kernel in the stream
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)p.items);
  cfg.blockDim = dim3((unsigned)K::NT);
  cfg.dynamicSmemBytes = (size_t)K::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fused_step_kernel<LAT, ST, BX, BY, NS>, tm, a, p.tiles_x,
                            p.tiles_y, p.zlen);
}

// Tile table shared by every storage type: id -> (BX, BY, NS).
#define SCLBM_D3Q19_TILES(X) \
  X(1, 32, 8, 3)             \
  X(2, 32, 4, 4)             \
  X(3, 64, 4, 3)             \
  X(4, 64, 8, 2)             \
  X(5, 128, 4, 2)            \
  X(6, 32, 8, 2)             \
  X(7, 64, 4, 2)             \
  X(8, 128, 4, 3)            \
  X(9, 64, 8, 3)             \
  X(10, 64, 8, 4)            \
  X(11, 128, 4, 4)           \
  X(12, 32, 8, 4)            \
  X(13, 64, 4, 4)
#define SCLBM_D2Q9_TILES(X) \
  X(1, 256, 1, 4)           \
  X(2, 128, 1, 4)           \
  X(3, 64, 1, 6)
// x-pair tiles (two cells per thread, step_fused_x2.cuh; FP32 and 16-bit
// storage only): id -> (BX, BY, NS)
#define SCLBM_D3Q19_X2_TILES(X) \
  X(14, 64, 8, 3)               \
  X(15, 64, 8, 4)               \
  X(16, 128, 4, 3)              \
  X(17, 128, 4, 4)              \
  X(18, 64, 4, 4)               \
  X(19, 128, 8, 2)              \
  X(20, 128, 8, 3)              \
  X(21, 64, 16, 3)              \
  X(22, 32, 8, 4)               \
  X(23, 64, 8, 2)               \
  X(24, 128, 4, 2)              \
  X(25, 64, 7, 3)
#define SCLBM_D2Q9_X2_TILES(X) \
  X(4, 256, 1, 4)              \
  X(5, 256, 1, 6)              \
  X(6, 128, 1, 6)

// Dispatch of one storage type over the tile table.
template <int ST>
cudaError_t fused_launch_st(int lat, const FusedPlan &p, const StepArgs &a, const FusedMaps &tm,
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
cudaError_t fused_prepare_st(int lat, const FusedPlan &p, int *blocks_per_sm) {
#define SCLBM_X3(id, bx, by, ns) \
  case id:                       \
    return fused_prepare_t<D3Q19, ST, bx, by, ns>(blocks_per_sm);
#define SCLBM_X2(id, bx, by, ns) \
  case id:                       \
    return fused_prepare_t<D2Q9, ST, bx, by, ns>(blocks_per_sm);
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
int fused_smem_st(int lat, int tile) {
#define SCLBM_X3(id, bx, by, ns) \
  case id:                       \
    return FusedK<D3Q19, ST, bx, by, ns>::SMEM;
#define SCLBM_X2(id, bx, by, ns) \
  case id:                       \
    return FusedK<D2Q9, ST, bx, by, ns>::SMEM;
  if (lat == D3Q19) {
    switch (tile) { SCLBM_D3Q19_TILES(SCLBM_X3) }
  } else {
    switch (tile) { SCLBM_D2Q9_TILES(SCLBM_X2) }
  }
#undef SCLBM_X3
#undef SCLBM_X2
  return -1;
}

}  // namespace sclbm
