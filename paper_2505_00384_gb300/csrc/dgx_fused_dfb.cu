// Fused operator kernels in double-word arithmetic (FP64 arrays, FP32 pipes),
// N = r+1 in {5, 6, 7} (see dgx_fused.cuh, dgx_df64.cuh).
#include "dgx_fused_launch.cuh"

namespace dgx {
DGX_FUSED_INSTANTIATE(df64, 5)
DGX_FUSED_MULTI_INSTANTIATE(df64, 5)
DGX_FUSED_INSTANTIATE(df64, 6)
DGX_FUSED_MULTI_INSTANTIATE(df64, 6)
DGX_FUSED_INSTANTIATE(df64, 7)
DGX_FUSED_MULTI_INSTANTIATE(df64, 7)
}  // namespace dgx
