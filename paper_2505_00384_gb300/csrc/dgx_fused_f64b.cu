// Fused operator kernels, double, N = r+1 in {5, 6, 7} (see dgx_fused.cuh).
#include "dgx_fused_launch.cuh"

namespace dgx {
DGX_FUSED_INSTANTIATE(double, 5)
DGX_FUSED_INSTANTIATE(double, 6)
DGX_FUSED_INSTANTIATE(double, 7)
}  // namespace dgx
