// Fused operator kernels in double-word arithmetic (FP64 arrays, FP32 pipes),
// N = r+1 = 7 (see dgx_fused.cuh, dgx_df64.cuh); one degree per translation
// unit so that the build compiles the large double-word kernels in parallel.
#include "dgx_fused_launch.cuh"

namespace dgx {
DGX_FUSED_INSTANTIATE(df64, 7)
DGX_FUSED_MULTI_INSTANTIATE(df64, 7)
}  // namespace dgx
