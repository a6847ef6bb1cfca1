// Fused operator kernels, float, N = r+1 in {5, 6, 7} (see dgx_fused.cuh).
#include "dgx_fused_launch.cuh"

namespace dgx {
DGX_FUSED_INSTANTIATE(float, 5)
DGX_FUSED_MULTI_INSTANTIATE(float, 5)
DGX_FUSED_INSTANTIATE(float, 6)
DGX_FUSED_MULTI_INSTANTIATE(float, 6)
DGX_FUSED_INSTANTIATE(float, 7)
DGX_FUSED_MULTI_INSTANTIATE(float, 7)
}  // namespace dgx
