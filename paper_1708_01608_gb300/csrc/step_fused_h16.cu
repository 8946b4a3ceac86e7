// Fused step kernels, 16-bit offset storage (FP16 / BF16), FP32 arithmetic.
#include "step_fused.cuh"

namespace sclbm {
cudaError_t fused_launch_h16(int lat, int st, const FusedPlan &p, const StepArgs &a,
                             const FusedMaps &tm, cudaStream_t s) {
  return st == ST_F16 ? fused_launch_st<ST_F16>(lat, p, a, tm, s)
                      : fused_launch_st<ST_BF16>(lat, p, a, tm, s);
}
cudaError_t fused_prepare_h16(int lat, int st, const FusedPlan &p, int *blocks_per_sm) {
  return st == ST_F16 ? fused_prepare_st<ST_F16>(lat, p, blocks_per_sm)
                      : fused_prepare_st<ST_BF16>(lat, p, blocks_per_sm);
}
int fused_smem_h16(int lat, int st, int tile) {
  return st == ST_F16 ? fused_smem_st<ST_F16>(lat, tile) : fused_smem_st<ST_BF16>(lat, tile);
}
}  // namespace sclbm
