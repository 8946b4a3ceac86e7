// Host side of the fused step: tile table, launch plan, TMA descriptors and
// dispatch to the per-storage translation units.
#include <climits>
#include <algorithm>

#include "step_fused.cuh"

namespace sclbm {

bool fused_tile_shape(int lat, int st, int tile, int *bx, int *by, int *nstage, int *xc) {
  int cells = 1;
#define SCLBM_T(id, BX, BY, NS) \
  case id:                      \
    *bx = BX;                   \
    *by = BY;                   \
    *nstage = NS;               \
    if (xc) *xc = cells;        \
    return true;
  if (lat == D3Q19) {
    switch (tile) { SCLBM_D3Q19_TILES(SCLBM_T) }
  } else {
    switch (tile) { SCLBM_D2Q9_TILES(SCLBM_T) }
  }
  if (st == ST_F64) return false;  // the x-pair kernel computes in FP32
  cells = 2;
  if (lat == D3Q19) {
    switch (tile) { SCLBM_D3Q19_X2_TILES(SCLBM_T) }
  } else {
    switch (tile) { SCLBM_D2Q9_X2_TILES(SCLBM_T) }
  }
#undef SCLBM_T
  return false;
}

static int fused_smem_bytes(int lat, int st, int tile, int xc) {
  if (xc == 2) {
    switch (st) {
      case ST_F32: return fused_x2_smem_f32(lat, tile);
      case ST_F16: return fused_x2_smem_f16(lat, tile);
      case ST_BF16: return fused_x2_smem_bf16(lat, tile);
      default: return -1;
    }
  }
  switch (st) {
    case ST_F64: return fused_smem_f64(lat, tile);
    case ST_F32: return fused_smem_f32(lat, tile);
    default: return fused_smem_h16(lat, st, tile);
  }
}

cudaError_t fused_make_plan(int lat, int st, int tile, int64_t NX, int64_t NY, int64_t NZ,
                            int nzc, FusedPlan *p) {
  int bx, by, ns, xc;
  if (tile <= 0) tile = 1;
  if (!fused_tile_shape(lat, st, tile, &bx, &by, &ns, &xc)) return cudaErrorInvalidValue;
  p->tile = tile;
  p->bx = bx;
  p->by = by;
  p->nstage = ns;
  p->xc = xc;
  p->threads = bx * by / xc;
  p->hx = (int)(16 / storage_bytes(st));
  p->smem = fused_smem_bytes(lat, st, tile, xc);
  if (NX % p->hx != 0) return cudaErrorInvalidValue;  // halo boxes must start on 16 bytes
  int dev = 0, nsm = 0, smem_optin = 0, smem_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (p->smem <= 0 || p->smem > smem_optin) return cudaErrorInvalidValue;
  p->tiles_x = (int)((NX + bx - 1) / bx);
  p->tiles_y = (int)((NY + by - 1) / by);
  const int ntiles = p->tiles_x * p->tiles_y;
  if (nzc <= 0) {
    // resident CTA slots: SMs x the kernel's occupancy (registers, shared
    // memory and threads)
    int per_sm = 0;
    if (fused_prepare(lat, st, *p, &per_sm) != cudaSuccess || per_sm < 1) {
      cudaGetLastError();
      per_sm = std::max(1, std::min(smem_sm / (p->smem + 1024), 2048 / p->threads));
    }
    // Time model: CTAs run in waves of `slots`, a chunk of zlen planes
    // stages zlen + 2; pick the number of chunks (at least 4 planes each)
    // with the fewest staged planes per slot, the smaller one on ties.
    const int64_t slots = (int64_t)nsm * per_sm;
    const int64_t max_nzc = std::max<int64_t>(1, NZ / 4);
    int64_t best_cost = INT64_MAX;
    if (nzc < 0)  // one wave: as many chunks as fill every slot once
      best_cost = 0, nzc = (int)std::min<int64_t>(std::max<int64_t>(1, slots / ntiles), max_nzc);
    for (int64_t c = 1; c <= max_nzc && best_cost > 0; ++c) {
      const int64_t zl = (NZ + c - 1) / c;
      const int64_t n = (NZ + zl - 1) / zl;  // chunks actually formed
      const int64_t waves = (ntiles * n + slots - 1) / slots;
      const int64_t cost = waves * (zl + 2);
      if (cost < best_cost) {
        best_cost = cost;
        nzc = (int)n;
      }
    }
  }
  nzc = (int)std::min<int64_t>(std::max(nzc, 1), NZ);
  p->zlen = (int)((NZ + nzc - 1) / nzc);
  p->nzc = (int)((NZ + p->zlen - 1) / p->zlen);
  p->items = ntiles * p->nzc;
  return cudaSuccess;
}

int fused_item_of(const FusedPlan &p, int64_t x, int64_t y, int64_t z) {
  const int tx = (int)(x / p.bx), ty = (int)(y / p.by), zc = (int)(z / p.zlen);
  return (zc * p.tiles_y + ty) * p.tiles_x + tx;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
  }
  return fn;
}

CUresult fused_encode_maps(int lat, int st, const FusedPlan &p, const void *base, int64_t NX,
                           int64_t NY, int64_t NZ, int64_t px, FusedMaps *tm) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return CUDA_ERROR_NOT_FOUND;
  const int Q = lat == D3Q19 ? 19 : 9;
  const size_t sz = storage_bytes(st);
  CUtensorMapDataType dt = st == ST_F64   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                           : st == ST_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                           : st == ST_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                          : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  cuuint64_t dims[4] = {(cuuint64_t)NX, (cuuint64_t)NY, (cuuint64_t)NZ, (cuuint64_t)Q};
  cuuint64_t strides[3] = {(cuuint64_t)(px * sz), (cuuint64_t)(px * NY * sz),
                           (cuuint64_t)(px * NY * NZ * sz)};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  const cuuint32_t bx = p.bx, by = p.by, hx = p.hx, q = Q;
  const cuuint32_t boxes[4][4] = {{bx, by, 1, q}, {hx, by, 1, q}, {bx, 1, 1, q}, {hx, 1, 1, q}};
  CUtensorMap *maps[4] = {&tm->main, &tm->col, &tm->row, &tm->crn};
  for (int m = 0; m < 4; ++m) {
    CUresult r = enc(maps[m], dt, 4, const_cast<void *>(base), dims, strides, boxes[m], estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return r;
  }
  return CUDA_SUCCESS;
}

cudaError_t fused_launch(int lat, int st, const FusedPlan &p, const StepArgs &a,
                         const FusedMaps &tm, cudaStream_t s) {
  if (p.xc == 2) {
    switch (st) {
      case ST_F32: return fused_x2_launch_f32(lat, p, a, tm, s);
      case ST_F16: return fused_x2_launch_f16(lat, p, a, tm, s);
      case ST_BF16: return fused_x2_launch_bf16(lat, p, a, tm, s);
      case ST_F16R:
      case ST_BF16R: return fused_x2_launch_h16r(lat, st, p, a, tm, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (st) {
    case ST_F64:
      return fused_launch_f64(lat, p, a, tm, s);
    case ST_F32:
      return fused_launch_f32(lat, p, a, tm, s);
    case ST_F16R:
    case ST_BF16R:
      return fused_launch_h16r(lat, st, p, a, tm, s);
    default:
      return fused_launch_h16(lat, st, p, a, tm, s);
  }
}

cudaError_t fused_prepare(int lat, int st, const FusedPlan &p, int *blocks_per_sm) {
  if (p.xc == 2) {
    switch (st) {
      case ST_F32: return fused_x2_prepare_f32(lat, p, blocks_per_sm);
      case ST_F16: return fused_x2_prepare_f16(lat, p, blocks_per_sm);
      case ST_BF16: return fused_x2_prepare_bf16(lat, p, blocks_per_sm);
      case ST_F16R:
      case ST_BF16R: return fused_x2_prepare_h16r(lat, st, p, blocks_per_sm);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (st) {
    case ST_F64:
      return fused_prepare_f64(lat, p, blocks_per_sm);
    case ST_F32:
      return fused_prepare_f32(lat, p, blocks_per_sm);
    case ST_F16R:
    case ST_BF16R:
      return fused_prepare_h16r(lat, st, p, blocks_per_sm);
    default:
      return fused_prepare_h16(lat, st, p, blocks_per_sm);
  }
}

}  // namespace sclbm
