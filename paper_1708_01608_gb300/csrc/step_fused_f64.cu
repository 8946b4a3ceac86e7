// Fused step kernels, FP64 storage and arithmetic.
#include "step_fused.cuh"

namespace sclbm {
cudaError_t fused_launch_f64(int lat, const FusedPlan &p, const StepArgs &a, const FusedMaps &tm,
                             cudaStream_t s) {
  return fused_launch_st<ST_F64>(lat, p, a, tm, s);
}
cudaError_t fused_prepare_f64(int lat, const FusedPlan &p, int *blocks_per_sm) {
  return fused_prepare_st<ST_F64>(lat, p, blocks_per_sm);
}
int fused_smem_f64(int lat, int tile) { return fused_smem_st<ST_F64>(lat, tile); }
}  // namespace sclbm
