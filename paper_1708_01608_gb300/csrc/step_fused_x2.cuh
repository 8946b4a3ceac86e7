// Fused Shan-Chen step, x-pair form: each thread owns two neighbouring cells
// (x, x + 1) of a row, x even.
//
// Staging (TMA boxes, NS-stage mbarrier pipeline), the psi ring and the push
// are those of the one-cell march in step_fused.cuh.  What changes is the
// unit of work: the thread carries the two cells' values as float2, so every
// FP32 operation of the collision (moments, force, velocity shift,
// equilibria, relaxation) is one paired instruction for two cells; staged
// populations come in as one 32/64-bit shared load per velocity, and the
// push of a velocity with cx = 0 is one 32/64-bit store for both cells.
//
// psi is kept twice per ring plane: N[j] = psi at tile column j - 2 and
// S[j] = N[j + 1].  The psi pairs a thread needs are then aligned float2
// loads: N at its own column for cx = 0, S at its own column for cx = +1 and
// S two columns left for cx = -1.
//
// 16-bit storage reads the staged populations of plane P once, into
// registers as packed pairs (psi of P must be complete before plane P - 1
// can be collided, so P waits there one iteration); its stage is refilled
// right after the psi phase and NS planes are in flight.  FP32 storage
// reads plane P a second time, into registers, after the collision of
// P - 1 (holding two planes of float pairs would cost 38 registers): its
// stage is free one iteration after it was consumed, and NS - 1 planes are
// in flight ahead of the plane being summed.
#pragma once

#include "step_fused.cuh"

namespace sclbm {

// ---- paired FP32 helpers -----------------------------------------------------
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b, rounded once (b * -1 is exact)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
// acc + c v and acc + c w v for c in {-1, 0, 1} (no term for c = 0)
template <int CC>
__device__ __forceinline__ float2 cacc2(float2 acc, float2 v) {
  if constexpr (CC > 0) return add2(acc, v);
  else if constexpr (CC < 0) return sub2(acc, v);
  else return acc;
}
template <int CC>
__device__ __forceinline__ float2 cfma2(float2 acc, float w, float2 v) {
  if constexpr (CC > 0) return fma2(f2(w), v, acc);
  else if constexpr (CC < 0) return fma2(f2(-w), v, acc);
  else return acc;
}
// c.u for a moving velocity, nonzero terms only, starting from a positive
// component (every representative of an opposite pair has one)
template <int A, int B, int Z>
__device__ __forceinline__ float2 cdot2(float2 x, float2 y, float2 z) {
  static_assert(A > 0 || B > 0 || Z > 0, "a velocity with a positive component");
  if constexpr (A > 0) return cacc2<Z>(cacc2<B>(x, y), z);
  else if constexpr (B > 0) return cacc2<Z>(cacc2<A>(y, x), z);
  else return cacc2<B>(cacc2<A>(z, x), y);
}
// psi(rho) = rho0 (1 - exp(-rho/rho0)), evaluated as rho0 - rho0 e; the
// scalar and the paired forms give the same bits for the same rho
__device__ __forceinline__ float psi_x2(float rho, float rho0, float inv_rho0) {
  return fmaf(-rho0, __expf(rho * -inv_rho0), rho0);
}
__device__ __forceinline__ float2 psi_x2(float2 rho, float rho0, float inv_rho0) {
  const float2 t = mul2(rho, f2(-inv_rho0));
  return fma2(f2(-rho0), make_float2(__expf(t.x), __expf(t.y)), f2(rho0));
}

// two neighbouring stored values <-> float2
template <int ST>
struct Storage2;
template <>
struct Storage2<ST_F32> {
  using T2 = float2;
  __device__ static float2 load(T2 v) { return v; }
  __device__ static T2 store(float2 v) { return v; }
};
template <>
struct Storage2<ST_F16> {
  using T2 = __half2;
  __device__ static float2 load(T2 v) { return __half22float2(v); }
  __device__ static T2 store(float2 v) { return __float22half2_rn(v); }
};
template <>
struct Storage2<ST_BF16> {
  using T2 = __nv_bfloat162;
  __device__ static float2 load(T2 v) { return __bfloat1622float2(v); }
  __device__ static T2 store(float2 v) { return __float22bfloat162_rn(v); }
};
template <>
struct Storage2<ST_F16R> : Storage2<ST_F16> {};
template <>
struct Storage2<ST_BF16R> : Storage2<ST_BF16> {};

// a + v for a 16-bit v, widened inside the add: the widening is exact, so
// the result has the bits of converting v first and adding in FP32, with
// one instruction instead of two
__device__ __forceinline__ float add_w(float a, __half v) {
  float d;
  asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(__half_as_ushort(v)), "f"(a));
  return d;
}
__device__ __forceinline__ float add_w(float a, __nv_bfloat16 v) {
  float d;
  asm("add.rn.f32.bf16 %0, %1, %2;" : "=f"(d) : "h"(__bfloat16_as_ushort(v)), "f"(a));
  return d;
}
// v - c for a 16-bit v, widened inside the subtraction (exact widening)
__device__ __forceinline__ float sub_w(__half v, float c) {
  float d;
  asm("sub.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(__half_as_ushort(v)), "f"(c));
  return d;
}
__device__ __forceinline__ float sub_w(__nv_bfloat16 v, float c) {
  float d;
  asm("sub.rn.f32.bf16 %0, %1, %2;" : "=f"(d) : "h"(__bfloat16_as_ushort(v)), "f"(c));
  return d;
}
// a * v + c for 16-bit a and v, both widened inside the FMA: when a holds a
// float exactly, the result has the bits of fmaf((float)a, (float)v, c)
__device__ __forceinline__ float fma_w(__half a, __half v, float c) {
  float d;
  asm("fma.rn.f32.f16 %0, %1, %2, %3;"
      : "=f"(d)
      : "h"(__half_as_ushort(a)), "h"(__half_as_ushort(v)), "f"(c));
  return d;
}
__device__ __forceinline__ float fma_w(__nv_bfloat16 a, __nv_bfloat16 v, float c) {
  float d;
  asm("fma.rn.f32.bf16 %0, %1, %2, %3;"
      : "=f"(d)
      : "h"(__bfloat16_as_ushort(a)), "h"(__bfloat16_as_ushort(v)), "f"(c));
  return d;
}
__device__ __forceinline__ __half lo16(__half2 v) { return __low2half(v); }
__device__ __forceinline__ __half hi16(__half2 v) { return __high2half(v); }
__device__ __forceinline__ __nv_bfloat16 lo16(__nv_bfloat162 v) { return __low2bfloat16(v); }
__device__ __forceinline__ __nv_bfloat16 hi16(__nv_bfloat162 v) { return __high2bfloat16(v); }

// Sum of the Q staged values of one cell (or of a pair of cells), in one
// fixed order for the scalar and the paired form: the same cell gets the
// same rho whether its own CTA or a neighbour's halo computes it.
__device__ __forceinline__ float addv(float a, float b) { return a + b; }
__device__ __forceinline__ float2 addv(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <int Q, class V, class Ld>
__device__ __forceinline__ V sum_q(Ld ld) {
  V a = ld(0), b = ld(1);
#pragma unroll
  for (int i = 2; i + 1 < Q; i += 2) {
    a = addv(a, ld(i));
    b = addv(b, ld(i + 1));
  }
  if constexpr (Q % 2 == 1) a = addv(a, ld(Q - 1));
  return addv(a, b);
}
// The same sums from 16-bit stored values, each widened inside its add
// (0 + v is v exactly, so the bits are those of sum_q on converted values):
// one cell, and a pair of cells from packed pairs.
template <int Q, class Ld>
__device__ __forceinline__ float sum_q_w1(Ld ld) {
  float a = 0.0f, b = 0.0f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (i % 2 == 0)
      a = add_w(a, ld(i));
    else
      b = add_w(b, ld(i));
  }
  return a + b;
}
template <int Q, class Ld>
__device__ __forceinline__ float2 sum_q_w2(Ld ld) {
  float ax = 0.0f, ay = 0.0f, bx = 0.0f, by = 0.0f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const auto v = ld(i);
    if (i % 2 == 0) {
      ax = add_w(ax, lo16(v));
      ay = add_w(ay, hi16(v));
    } else {
      bx = add_w(bx, lo16(v));
      by = add_w(by, hi16(v));
    }
  }
  return __fadd2_rn(make_float2(ax, ay), make_float2(bx, by));
}

template <int LAT, int ST, int BX_, int BY_, int NS_>
struct FusedK2 {
  using B = FusedK<LAT, ST, BX_, BY_, NS_>;
  using L = typename B::L;
  using T = typename B::T;
  static constexpr int BX = BX_, BY = BY_, NS = NS_;
  static constexpr int Q = B::Q, HY = B::HY, HX = B::HX;
  static constexpr int TPX = BX / 2;  // threads along x
  static constexpr int NT = TPX * BY;
  static constexpr int PW = BX + 4;   // ring columns: tile x - 2 .. x + BX + 1
  static constexpr int PH = BY + 2 * HY;
  static constexpr int RP = PW * PH;  // floats of one ring plane
  static constexpr int STAGE_BYTES = B::STAGE_BYTES;
  static constexpr int RING_BYTES = 2 * 4 * RP * (int)sizeof(float);
  static constexpr int SMEM = NS * STAGE_BYTES + RING_BYTES + NS * 8 + 128;
  // halo work: pairs of the top and bottom halo rows, four corners, two side
  // columns (D2Q9 view: two side cells)
  static constexpr int NUNITS = HY ? BX + 4 + 2 * BY : 2;
  static_assert(BX % 2 == 0 && HX % 2 == 0, "pairs start on even columns");
  static_assert(NUNITS <= NT, "one halo unit per thread at most");
  static_assert(NS >= 2, "one stage is consumed while the next is summed");
};

// OM16: 1 - omega is exactly a value of the 16-bit storage type, so the
// relaxation's (1 - omega) g_i takes the stored g_i unconverted (fma_w)
template <int LAT, int ST, int BX, int BY, int NS, bool OM16 = false, class OutPop>
__device__ __forceinline__ bool fused_march_x2(const MarchArgs &m, OutPop out_pop, uint32_t &kb) {
  using K = FusedK2<LAT, ST, BX, BY, NS>;
  using B = typename K::B;
  using L = typename K::L;
  using T = typename K::T;
  using S1 = Storage<ST>;
  using S2 = Storage2<ST>;
  using T2 = typename S2::T2;
  constexpr int Q = K::Q, HY = K::HY, HX = K::HX, PW = K::PW, PH = K::PH, RP = K::RP,
                TPX = K::TPX;
  (void)PH;
  // 16-bit residual forms: each cell's rounding residual of the last step
  // joins its mass R, and the new one is what this step's stores round off
  constexpr bool RESID = S1::RESID;
  // 16-bit storage keeps a staged plane in registers as packed pairs (19
  // registers): read from its stage once, for psi, it is collided one
  // iteration later, and the stage is refilled right after the psi phase,
  // so NS planes are in flight.  FP32 pairs would take 38 registers more;
  // there the plane is read from its stage a second time after the
  // collision, and NS - 1 planes are in flight.
  constexpr bool KEEP = sizeof(T) == 2;

  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
  float *ringN = reinterpret_cast<float *>(smem + NS * K::STAGE_BYTES);
  float *ringS = ringN + 4 * RP;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + NS * K::STAGE_BYTES + K::RING_BYTES);

  const int tid = threadIdx.x;
  const int tp = tid % TPX, ty = tid / TPX;
  const int tx = 2 * tp;  // tile column of cell a; cell b is tx + 1
  const int NX = m.NX, NY = m.NY, NZ = m.NZ;
  const int x0 = m.x0, y0 = m.y0, zs = m.zs, ze = m.ze;
  const int BXe = min(BX, NX - x0), BYe = min(BY, NY - y0);  // BXe is even
  if (zs >= ze) return true;
  const int NPL = ze - zs + 2;  // staged planes zs-1 .. ze
  const bool active = tx < BXe && ty < BYe;
  const int xl = x0 == 0 ? NX - HX : x0 - HX;
  const int xr = x0 + BXe == NX ? 0 : x0 + BXe;
  const int yt = y0 == 0 ? NY - 1 : y0 - 1;
  const int yb = y0 + BYe == NY ? 0 : y0 + BYe;
  const int64_t plane = m.px * NY;

  const float G = m.G_f, tau = m.tau_f, omega = m.omega_f, rho0 = m.rho0_f,
              inv_rho0 = m.inv_rho0_f, rho_ref = m.rho_ref_f;

  const uint32_t k0 = kb;
  auto issue = [&](int k) {
    if ((m.debug_flags & 1) && k == 1) return;  // test hook: let the wait expire
    const int P = zs - 1 + k, s = (int)((k0 + k) % NS);
    const int zp = P < 0 ? P + NZ : (P >= NZ ? P - NZ : P);
    uint8_t *st = smem + s * K::STAGE_BYTES;
    mbar_arrive_expect_tx(&bars[s], (uint32_t)B::TX_BYTES);
    tma_load_4d(st, &m.tm->main, x0, y0, zp, 0, &bars[s]);
    tma_load_4d(st + B::OFF_L, &m.tm->col, xl, y0, zp, 0, &bars[s]);
    tma_load_4d(st + B::OFF_R, &m.tm->col, xr, y0, zp, 0, &bars[s]);
    if (HY) {
      tma_load_4d(st + B::OFF_T, &m.tm->row, x0, yt, zp, 0, &bars[s]);
      tma_load_4d(st + B::OFF_B, &m.tm->row, x0, yb, zp, 0, &bars[s]);
      tma_load_4d(st + B::OFF_TL, &m.tm->crn, xl, yt, zp, 0, &bars[s]);
      tma_load_4d(st + B::OFF_TR, &m.tm->crn, xr, yt, zp, 0, &bars[s]);
      tma_load_4d(st + B::OFF_BL, &m.tm->crn, xl, yb, zp, 0, &bars[s]);
      tma_load_4d(st + B::OFF_BR, &m.tm->crn, xr, yb, zp, 0, &bars[s]);
    }
  };
  if (tid == 0) {
    for (int k = 0; k < NS && k < NPL; ++k) issue(k);
  }

  // injection sites of this CTA, sorted by z; the next one in registers
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

  // push destinations (periodic).  Cell a = (x, y), cell b = (x + 1, y);
  // only a's -x and b's +x destinations can wrap.
  const int x = x0 + tx, y = y0 + ty;
  const int32_t dam = (x == 0 ? NX - 1 : x - 1) - x;  // a, cx = -1: -1 or NX - 1
  const int32_t dbp = (x + 2 >= NX ? 0 : x + 2) - x;  // b, cx = +1: 2 or -x
  const int ym = y == 0 ? NY - 1 : y - 1, yp = y + 1 >= NY ? 0 : y + 1;
  const int32_t oy[3] = {(int32_t)(ym * m.px), (int32_t)(y * m.px), (int32_t)(yp * m.px)};

  // The halo unit of this thread: a pair of cells of the top or bottom halo
  // row, or one cell of the corners and side columns.  h_off: byte offset of
  // its population 0 in a stage; h_pstride: elements between populations;
  // h_j: its ring index (column of cell a).
  const int nunits = HY ? BXe + 4 + 2 * BYe : 2;
  int h_off = 0, h_pstride = 0, h_j = 0;
  bool h_pair = false;
  if (tid < nunits) {
    int dx, dy;
    if (HY) {
      const int np = BXe / 2;
      if (tid < 2 * np) {
        h_pair = true;
        dy = tid < np ? -1 : BYe;
        dx = 2 * (tid < np ? tid : tid - np);
      } else if (tid < 2 * np + 4) {
        const int h = tid - 2 * np;
        dx = (h & 1) ? BXe : -1;
        dy = (h & 2) ? BYe : -1;
      } else {
        const int h = tid - 2 * np - 4;
        dx = h < BYe ? -1 : BXe;
        dy = h < BYe ? h : h - BYe;
      }
    } else {
      dx = tid == 0 ? -1 : BXe;
      dy = 0;
    }
    const int cxr = dx < 0 ? 0 : (dx >= BXe ? 2 : 1);
    const int cyr = dy < 0 ? 0 : (dy >= BYe ? 2 : 1);
    int off, e;
    if (cyr == 1) {  // side column (never the interior)
      off = cxr == 0 ? B::OFF_L : B::OFF_R;
      e = dy * HX + (cxr == 0 ? HX - 1 : 0);
      h_pstride = BY * HX;
    } else if (cxr == 1) {  // top or bottom row
      off = cyr == 0 ? B::OFF_T : B::OFF_B;
      e = dx;
      h_pstride = BX;
    } else {
      off = cyr == 0 ? (cxr == 0 ? B::OFF_TL : B::OFF_TR) : (cxr == 0 ? B::OFF_BL : B::OFF_BR);
      e = cxr == 0 ? HX - 1 : 0;
      h_pstride = HX;
    }
    h_off = off + e * (int)sizeof(T);
    h_j = (dy + HY) * PW + dx + 2;
  }

  // staged values (cells a, b) as stored: cur of plane P - 1 for the
  // collision; with KEEP, nxt of plane P, read once from its stage for psi
  T2 cur[Q], nxt[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) cur[i] = nxt[i] = S2::store(f2(0.0f));
  float2 Rcur = f2(0.0f), Rnxt = f2(0.0f);  // sums of the staged values

  const float om1 = 1.0f - omega;
  float cW[2], c3[2], c45[2];
#pragma unroll
  for (int k2 = 0; k2 < 2; ++k2) {
    const float w = (float)L::w(L::rep(k2 == 0 ? 0 : L::NP - 1));
    cW[k2] = w * omega;
    c3[k2] = 3.0f * w * omega;
    c45[k2] = 4.5f * w * omega;
  }
  const int c0 = (ty + HY) * PW + tx + 2;  // ring index of cell a

  for (int k = 0; k < NPL; ++k) {
    const int s = (int)((k0 + k) % NS);
    const int P = zs - 1 + k;
    const bool ok = mbar_wait_bounded(&bars[s], ((k0 + k) / NS) & 1u, 1000000000ull);
    const uint8_t *st = smem + s * K::STAGE_BYTES;
    const T2 *main2 = reinterpret_cast<const T2 *>(st);

    // ---- psi of plane P: interior pairs and halo units
    float *rN = ringN + (k & 3) * RP;
    float *rS = ringS + (k & 3) * RP;
    if (active) {
      if constexpr (KEEP) {
#pragma unroll
        for (int i = 0; i < Q; ++i) nxt[i] = main2[(i * BY + ty) * TPX + tp];
      }
      float2 r2;
      if constexpr (sizeof(T) == 2)
        r2 = sum_q_w2<Q>([&](int i) { return KEEP ? nxt[i] : main2[(i * BY + ty) * TPX + tp]; });
      else
        r2 = sum_q<Q, float2>([&](int i) { return S2::load(main2[(i * BY + ty) * TPX + tp]); });
      const float2 ps = psi_x2(add2(f2(rho_ref), r2), rho0, inv_rho0);
      *reinterpret_cast<float2 *>(rN + c0) = ps;
      rS[c0 - 1] = ps.x;
      rS[c0] = ps.y;
      Rnxt = r2;
    }
    if (tid < nunits) {
      if (h_pair) {
        const T2 *b2 = reinterpret_cast<const T2 *>(st + h_off);
        const int ps2 = h_pstride / 2;
        float2 r2;
        if constexpr (sizeof(T) == 2)
          r2 = sum_q_w2<Q>([&](int i) { return b2[i * ps2]; });
        else
          r2 = sum_q<Q, float2>([&](int i) { return S2::load(b2[i * ps2]); });
        const float2 ps = psi_x2(add2(f2(rho_ref), r2), rho0, inv_rho0);
        *reinterpret_cast<float2 *>(rN + h_j) = ps;
        rS[h_j - 1] = ps.x;
        rS[h_j] = ps.y;
      } else {
        const T *b1 = reinterpret_cast<const T *>(st + h_off);
        float r;
        if constexpr (sizeof(T) == 2)
          r = sum_q_w1<Q>([&](int i) { return b1[i * h_pstride]; });
        else
          r = sum_q<Q, float>([&](int i) { return S1::load(b1[i * h_pstride]); });
        rS[h_j - 1] = psi_x2(rho_ref + r, rho0, inv_rho0);  // N of side cells is never read
      }
    }

    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        if (m.err) atomicOr(m.err, ERR_TMA_TIMEOUT);
        // wait (bounded) for the copies still in flight into this CTA's stages
        const int hi = KEEP ? min(NPL, k + NS) : min(NPL, max(NS, k + NS - 1));
        for (int k2 = k + 1; k2 < hi; ++k2)
          mbar_wait_bounded(&bars[(k0 + k2) % NS], ((k0 + k2) / NS) & 1u, 100000000ull);
      }
      return false;
    }
    if constexpr (KEEP) {
      // the stage of plane P was last read before this barrier (its values
      // are in registers now): refill it with plane P + NS
      if (tid == 0 && k + NS < NPL) issue(k + NS);
    } else {
      // the stage of plane P - 1 was last read before this barrier
      if (tid == 0 && k >= 1 && k - 1 + NS < NPL) issue(k - 1 + NS);
    }

    // ---- collide plane P - 1 (psi of P - 2, P - 1, P in the ring) and push
    if (k >= 2) {
      const int Pc = P - 1;
      float2 dmc = f2(0.0f);
      bool site = false;
      if (Pc == next_z) {  // sites of this CTA in this plane (rare)
        double dma = 0.0, dmb = 0.0;
        while (next_z == Pc) {
          if (active && site_y == y && (site_x == x || site_x == x + 1) && site_budget > 0.0) {
            const double d = fmin(site_rate, site_budget);
            m.budget[site_i] = site_budget - d;
            if (site_x == x)
              dma += d;
            else
              dmb += d;
            site = true;
          }
          ++sp;
          load_site();
        }
        dmc = make_float2((float)dma, (float)dmb);
      }
      if (active) {
        const int km = (k - 2) & 3, k0p = (k - 1) & 3, kp = k & 3;
        const int zm = Pc == 0 ? NZ - 1 : Pc - 1, zp = Pc + 1 >= NZ ? 0 : Pc + 1;
        const int32_t oz[3] = {(int32_t)(zm * plane), (int32_t)(Pc * plane), (int32_t)(zp * plane)};
        // psi of the two cells' neighbours along velocity i
        auto psi2_at = [&](auto ic) -> float2 {
          constexpr int i = decltype(ic)::value;
          constexpr int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
          const int pl = cz < 0 ? km : (cz > 0 ? kp : k0p);
          const float *r = (cx == 0 ? ringN : ringS) + pl * RP;
          return *reinterpret_cast<const float2 *>(r + c0 + cy * PW + (cx < 0 ? -2 : 0));
        };
        // push of velocity i for cells a and b; the residual forms sum what
        // the 16-bit stores round off, per cell
        float2 racc = f2(0.0f);
        auto put = [&](auto ic, float2 v) {
          constexpr int i = decltype(ic)::value;
          constexpr int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
          T *p = out_pop(i) + (oz[cz + 1] + oy[cy + 1] + x);
          if constexpr (cx == 0) {
            const T2 q = S2::store(v);
            *reinterpret_cast<T2 *>(p) = q;
            if constexpr (RESID) racc = add2(racc, sub2(v, S2::load(q)));
          } else {
            const T qa = S1::store(v.x), qb = S1::store(v.y);
            if constexpr (cx > 0) {
              p[1] = qa;
              p[dbp] = qb;
            } else {
              p[dam] = qa;
              p[0] = qb;
            }
            if constexpr (RESID)
              racc = add2(racc, make_float2(v.x - S1::load(qa), v.y - S1::load(qb)));
          }
        };

        // moments and the Shan-Chen force sum, opposite velocities in pairs
        const int32_t own = oz[1] + oy[1] + x;  // cell a; b is own + 1
        float2 R = Rcur;
        if constexpr (RESID) R = add2(R, *reinterpret_cast<const float2 *>(m.resid + own));
        float2 jx = f2(-0.0f), jy = f2(-0.0f), jz = f2(-0.0f);
        float2 sx = f2(-0.0f), sy = f2(-0.0f), sz = f2(-0.0f);
        static_for<L::NP>([&](auto kc) {
          constexpr int k2 = decltype(kc)::value, i = L::rep(k2), o = L::opp(i);
          constexpr int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
          float2 d;
          if constexpr (sizeof(T) == 2) {
            const float2 vo = S2::load(cur[o]);
            d = make_float2(sub_w(lo16(cur[i]), vo.x), sub_w(hi16(cur[i]), vo.y));
          } else {
            d = sub2(S2::load(cur[i]), S2::load(cur[o]));
          }
          jx = cacc2<cx>(jx, d);
          jy = cacc2<cy>(jy, d);
          jz = cacc2<cz>(jz, d);
          const float2 dps = sub2(psi2_at(std::integral_constant<int, i>{}),
                                  psi2_at(std::integral_constant<int, o>{}));
          const float w = (float)L::w(i);
          sx = cfma2<cx>(sx, w, dps);
          sy = cfma2<cy>(sy, w, dps);
          sz = cfma2<cz>(sz, w, dps);
        });
        const float2 rho = add2(f2(rho_ref), R);
        const float2 gp = mul2(f2(-G), *reinterpret_cast<const float2 *>(ringN + k0p * RP + c0));
        const float2 ir = make_float2(__fdividef(1.0f, rho.x), __fdividef(1.0f, rho.y));
        const float2 ux = mul2(fma2(f2(tau), mul2(gp, sx), jx), ir);
        const float2 uy = mul2(fma2(f2(tau), mul2(gp, sy), jy), ir);
        const float2 uz = mul2(fma2(f2(tau), mul2(gp, sz), jz), ir);
        const float2 uu = fma2(uz, uz, fma2(uy, uy, mul2(ux, ux)));
        const float2 Kc = fma2(mul2(rho, f2(-1.5f)), uu, R);
        const float2 wK[2] = {mul2(f2(cW[0]), Kc), mul2(f2(cW[1]), Kc)};
        const float2 om1_2 = f2(om1);
        [[maybe_unused]] T om1h;
        if constexpr (OM16) om1h = S1::store(om1);
        // relax and push (offset form, as in the one-cell march):
        //   g_i* = (1 - omega) g_i + omega w_i (K + 4.5 rho (c.u)^2) + 3 omega w_i rho c.u
        // SITE adds w_i dm to every population of the site cell
        auto relax_push = [&](auto with_site) {
          constexpr bool SITE = decltype(with_site)::value;
          float2 moved = f2(-0.0f);
          static_for<L::NP>([&](auto kc) {
            constexpr int k2 = decltype(kc)::value, i = L::rep(k2), o = L::opp(i);
            constexpr int wc = L::w(i) == L::w(L::rep(0)) ? 0 : 1;
            const float2 cu = cdot2<L::cx(i), L::cy(i), L::cz(i)>(ux, uy, uz);
            const float2 a = mul2(rho, cu);
            const float2 A = fma2(a, mul2(f2(c45[wc]), cu), wK[wc]);
            // A +- B with B = 3 omega w_i a, as FMAs (the one-cell march's form)
            const float2 Ai = fma2(f2(c3[wc]), a, A), Ao = fma2(f2(-c3[wc]), a, A);
            float2 gi, go;
            if constexpr (OM16) {
              gi = make_float2(fma_w(om1h, lo16(cur[i]), Ai.x), fma_w(om1h, hi16(cur[i]), Ai.y));
              go = make_float2(fma_w(om1h, lo16(cur[o]), Ao.x), fma_w(om1h, hi16(cur[o]), Ao.y));
            } else {
              gi = fma2(om1_2, S2::load(cur[i]), Ai);
              go = fma2(om1_2, S2::load(cur[o]), Ao);
            }
            moved = add2(moved, add2(gi, go));
            if (SITE) {
              put(std::integral_constant<int, i>{}, fma2(f2((float)L::w(i)), dmc, gi));
              put(std::integral_constant<int, o>{}, fma2(f2((float)L::w(o)), dmc, go));
            } else {
              put(std::integral_constant<int, i>{}, gi);
              put(std::integral_constant<int, o>{}, go);
            }
          });
          const float2 g0 = sub2(R, moved);
          put(std::integral_constant<int, 0>{},
              SITE ? fma2(f2((float)L::w(0)), dmc, g0) : g0);
        };
        if (site)
          relax_push(std::true_type{});
        else
          relax_push(std::false_type{});
        if constexpr (RESID) *reinterpret_cast<float2 *>(m.resid + own) = racc;
      }
    }
    // ---- plane P is collided in the next iteration
    if constexpr (KEEP) {
#pragma unroll
      for (int i = 0; i < Q; ++i) cur[i] = nxt[i];
    } else if (active && k >= 1 && k + 1 < NPL) {
#pragma unroll
      for (int i = 0; i < Q; ++i) cur[i] = main2[(i * BY + ty) * TPX + tp];
    }
    Rcur = Rnxt;
  }
  kb = k0 + NPL;
  return true;
}

template <int LAT, int ST, int BX, int BY, int NS, bool OM16 = false>
__global__ void __launch_bounds__(BX / 2 * BY, BX / 2 * BY <= 256 ? 512 / (BX / 2 * BY) : 1)
    fused_step_kernel_x2(const __grid_constant__ FusedMaps tm, const StepArgs a, const int tiles_x,
                         const int tiles_y, const int zlen) {
  using T = typename Storage<ST>::T;
  const MarchArgs m = march_args_of(tm, a, tiles_x, tiles_y, zlen, BX, BY);
  fused_barriers_init_k<FusedK2<LAT, ST, BX, BY, NS>>(m);
  // programmatic dependent launch, as in the one-cell kernel
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  uint32_t kb = 0;
  fused_march_x2<LAT, ST, BX, BY, NS, OM16>(
      m, [&](int i) { return static_cast<T *>(a.out_pop[i]); }, kb);
}

// 16-bit storage: does 1 - omega convert to the storage type exactly?
template <int ST>
bool om1_is_16bit(float omega) {
  using T = typename Storage<ST>::T;
  if constexpr (sizeof(T) != 2) {
    (void)omega;
    return false;
  } else {
    const float om1 = 1.0f - omega;
    if constexpr (std::is_same_v<T, __half>)
      return __half2float(__float2half_rn(om1)) == om1;
    else
      return __bfloat162float(__float2bfloat16_rn(om1)) == om1;
  }
}

template <int LAT, int ST, int BX, int BY, int NS>
cudaError_t fused_x2_prepare_t(int *blocks_per_sm) {
  using K = FusedK2<LAT, ST, BX, BY, NS>;
  cudaError_t e = cudaFuncSetAttribute(fused_step_kernel_x2<LAT, ST, BX, BY, NS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM);
  if constexpr (sizeof(typename Storage<ST>::T) == 2) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fused_step_kernel_x2<LAT, ST, BX, BY, NS, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM);
  }
  if (e == cudaSuccess && blocks_per_sm)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        blocks_per_sm, fused_step_kernel_x2<LAT, ST, BX, BY, NS>, K::NT, K::SMEM);
  return e;
}

template <int LAT, int ST, int BX, int BY, int NS>
cudaError_t fused_x2_launch_t(const FusedPlan &p, const StepArgs &a, const FusedMaps &tm,
                              cudaStream_t s) {
  using K = FusedK2<LAT, ST, BX, BY, NS>;
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
  if constexpr (sizeof(typename Storage<ST>::T) == 2) {
    if (!(a.debug_flags & 2) && om1_is_16bit<ST>(a.omega_f))  // 2: LBM_DEBUG_CONVERT_BEFORE_FMA
      return cudaLaunchKernelEx(&cfg, fused_step_kernel_x2<LAT, ST, BX, BY, NS, true>, tm, a,
                                p.tiles_x, p.tiles_y, p.zlen);
  }
  return cudaLaunchKernelEx(&cfg, fused_step_kernel_x2<LAT, ST, BX, BY, NS>, tm, a, p.tiles_x,
                            p.tiles_y, p.zlen);
}

// Dispatch of one storage type over the x-pair tile table.
template <int ST>
cudaError_t fused_x2_launch_st(int lat, const FusedPlan &p, const StepArgs &a,
                               const FusedMaps &tm, cudaStream_t s) {
#define SCLBM_X3(id, bx, by, ns) \
  case id:                       \
    return fused_x2_launch_t<D3Q19, ST, bx, by, ns>(p, a, tm, s);
#define SCLBM_X2(id, bx, by, ns) \
  case id:                       \
    return fused_x2_launch_t<D2Q9, ST, bx, by, ns>(p, a, tm, s);
  if (lat == D3Q19) {
    switch (p.tile) { SCLBM_D3Q19_X2_TILES(SCLBM_X3) }
  } else {
    switch (p.tile) { SCLBM_D2Q9_X2_TILES(SCLBM_X2) }
  }
#undef SCLBM_X3
#undef SCLBM_X2
  return cudaErrorInvalidValue;
}

template <int ST>
cudaError_t fused_x2_prepare_st(int lat, const FusedPlan &p, int *blocks_per_sm) {
#define SCLBM_X3(id, bx, by, ns) \
  case id:                       \
    return fused_x2_prepare_t<D3Q19, ST, bx, by, ns>(blocks_per_sm);
#define SCLBM_X2(id, bx, by, ns) \
  case id:                       \
    return fused_x2_prepare_t<D2Q9, ST, bx, by, ns>(blocks_per_sm);
  if (lat == D3Q19) {
    switch (p.tile) { SCLBM_D3Q19_X2_TILES(SCLBM_X3) }
  } else {
    switch (p.tile) { SCLBM_D2Q9_X2_TILES(SCLBM_X2) }
  }
#undef SCLBM_X3
#undef SCLBM_X2
  return cudaErrorInvalidValue;
}

template <int ST>
int fused_x2_smem_st(int lat, int tile) {
#define SCLBM_X3(id, bx, by, ns) \
  case id:                       \
    return FusedK2<D3Q19, ST, bx, by, ns>::SMEM;
#define SCLBM_X2(id, bx, by, ns) \
  case id:                       \
    return FusedK2<D2Q9, ST, bx, by, ns>::SMEM;
  if (lat == D3Q19) {
    switch (tile) { SCLBM_D3Q19_X2_TILES(SCLBM_X3) }
  } else {
    switch (tile) { SCLBM_D2Q9_X2_TILES(SCLBM_X2) }
  }
#undef SCLBM_X3
#undef SCLBM_X2
  return -1;
}

}  // namespace sclbm
