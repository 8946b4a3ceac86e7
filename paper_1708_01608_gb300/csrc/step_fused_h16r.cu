// Fused step kernels, 16-bit offset storage with the per-cell rounding
// residual (ST_F16R / ST_BF16R), FP32 arithmetic.
#include "step_fused.cuh"

namespace sclbm {
cudaError_t fused_launch_h16r(int lat, int st, const FusedPlan &p, const StepArgs &a,
                              const FusedMaps &tm, cudaStream_t s) {
  return st == ST_F16R ? fused_launch_st<ST_F16R>(lat, p, a, tm, s)
                       : fused_launch_st<ST_BF16R>(lat, p, a, tm, s);
}
cudaError_t fused_prepare_h16r(int lat, int st, const FusedPlan &p, int *blocks_per_sm) {
  return st == ST_F16R ? fused_prepare_st<ST_F16R>(lat, p, blocks_per_sm)
                       : fused_prepare_st<ST_BF16R>(lat, p, blocks_per_sm);
}
}  // namespace sclbm
