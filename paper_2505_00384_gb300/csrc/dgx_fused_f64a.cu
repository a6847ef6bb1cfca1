// Fused operator kernels, double, N = r+1 in {2, 3, 4} (see dgx_fused.cuh).
#include "dgx_fused_launch.cuh"

namespace dgx {
DGX_FUSED_INSTANTIATE(double, 2)
DGX_FUSED_INSTANTIATE(double, 3)
DGX_FUSED_INSTANTIATE(double, 4)
}  // namespace dgx
