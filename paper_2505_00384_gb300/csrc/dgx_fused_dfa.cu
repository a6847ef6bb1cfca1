// Fused operator kernels in double-word arithmetic (FP64 arrays, FP32 pipes),
// N = r+1 in {2, 3, 4} (see dgx_fused.cuh, dgx_df64.cuh).
#include "dgx_fused_launch.cuh"

namespace dgx {
DGX_FUSED_INSTANTIATE(df64, 2)
DGX_FUSED_MULTI_INSTANTIATE(df64, 2)
DGX_FUSED_INSTANTIATE(df64, 3)
DGX_FUSED_MULTI_INSTANTIATE(df64, 3)
DGX_FUSED_INSTANTIATE(df64, 4)
DGX_FUSED_MULTI_INSTANTIATE(df64, 4)
}  // namespace dgx
