// Fused operator kernels, float, N = r+1 in {2, 3, 4} (see dgx_fused.cuh).
#include "dgx_fused_launch.cuh"

namespace dgx {
DGX_FUSED_INSTANTIATE(float, 2)
DGX_FUSED_MULTI_INSTANTIATE(float, 2)
DGX_FUSED_INSTANTIATE(float, 3)
DGX_FUSED_MULTI_INSTANTIATE(float, 3)
DGX_FUSED_INSTANTIATE(float, 4)
DGX_FUSED_MULTI_INSTANTIATE(float, 4)
}  // namespace dgx
