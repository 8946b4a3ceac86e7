// x-pair fused step kernels, FP32 storage, FP32 arithmetic.
#include "step_fused_x2.cuh"

namespace sclbm {
cudaError_t fused_x2_launch_f32(int lat, const FusedPlan &p, const StepArgs &a,
                                const FusedMaps &tm, cudaStream_t s) {
  return fused_x2_launch_st<ST_F32>(lat, p, a, tm, s);
}
cudaError_t fused_x2_prepare_f32(int lat, const FusedPlan &p, int *blocks_per_sm) {
  return fused_x2_prepare_st<ST_F32>(lat, p, blocks_per_sm);
}
int fused_x2_smem_f32(int lat, int tile) { return fused_x2_smem_st<ST_F32>(lat, tile); }
}  // namespace sclbm
