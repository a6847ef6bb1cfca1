// Allocation-free variant of the pressure-operator application.
//
// Some callers cannot allocate device memory when they apply the operator:
// an application that hands all device memory to its own pool allocator at
// start-up and forbids any later cudaMalloc, or a time-critical loop where an
// allocation (which may synchronise the device) is not acceptable.  This entry
// point needs no per-call or per-context scratch: the intermediate
// V = A^-1 B x lives in a fixed, file-scope device array that the CUDA
// runtime creates when the library's module is loaded.  Every GPU that loads
// the library holds this array until the process exits.
#include <mutex>

#include "dgx_common.cuh"

namespace {

// Scratch for V (3N elements of the requested precision).
static __device__ __align__(256) unsigned char g_noalloc_scratch[DGX_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of the scratch array on `device`.  In host code the array's
// name is only a host-side stand-in, so the address is looked up once per
// device, with that device current, and cached.
int scratch_address(dgx_ctx *c, void **out) {
  if (c->device < 0 || c->device >= kMaxDevices)
    return dgx::set_error(c, DGX_ERR_ARG, "device %d outside 0..%d", c->device, kMaxDevices - 1);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[c->device]) {
    int prev = -1;
    if (int e = dgx::check_cuda(c, cudaGetDevice(&prev), "cudaGetDevice")) return e;
    if (prev != c->device)
      if (int e = dgx::check_cuda(c, cudaSetDevice(c->device), "cudaSetDevice")) return e;
    void *p = nullptr;
    const cudaError_t rc = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (prev != c->device) cudaSetDevice(prev);
    if (int e = dgx::check_cuda(c, rc, "cudaGetSymbolAddress(scratch)")) return e;
    if (!p) return dgx::set_error(c, DGX_ERR_CUDA, "null scratch address");
    g_addr[c->device] = p;
  }
  *out = g_addr[c->device];
  return 0;
}

template <typename T>
int apply_noalloc(dgx_ctx *c, const T *x, T *y) {
  const double need = 3.0 * (double)c->N * sizeof(T);
  if (need > (double)DGX_NOALLOC_SCRATCH_BYTES)
    return dgx::set_error(c, DGX_ERR_ARG,
                          "dgx_apply_operator_noalloc: mesh needs %.0f bytes of scratch (3N = %lld elements of %d "
                          "bytes), above the fixed %u bytes; use dgx_apply_operator",
                          need, 3LL * c->N, (int)sizeof(T), (unsigned)DGX_NOALLOC_SCRATCH_BYTES);
  void *scratch = nullptr;
  if (int e = scratch_address(c, &scratch)) return e;
  T *V = reinterpret_cast<T *>(scratch);
  const T *rho, *pk;
  if constexpr (sizeof(T) == 8) {
    rho = reinterpret_cast<const T *>(c->rho64);
    pk = reinterpret_cast<const T *>(c->pk64);
  } else {
    rho = reinterpret_cast<const T *>(c->rho32);
    pk = reinterpret_cast<const T *>(c->pk32);
  }
  // k_grad writes all 3N entries of V before k_div reads them (same stream):
  // nothing left from an earlier call is read, so no clearing is needed.
  if (int e = dgx::launch_grad<T>(c, x, rho, V, c->stream)) return e;
  return dgx::launch_div<T>(c, V, x, pk, y, c->stream);
}

}  // namespace

extern "C" int dgx_apply_operator_noalloc(dgx_ctx *c, int prec, const void *x, void *y) {
  if (!c) return DGX_ERR_ARG;
  if (!c->has_mesh) return dgx::set_error(c, DGX_ERR_STATE, "no mesh (call dgx_mesh_build)");
  if (!c->has_coef) return dgx::set_error(c, DGX_ERR_STATE, "no coefficients (call dgx_set_coefficients)");
  if (c->nc) return dgx::set_error(c, DGX_ERR_STATE, "not available on non-conforming meshes (use dgx_apply_operator)");
  if (!x || !y || x == y) return dgx::set_error(c, DGX_ERR_ARG, "x, y must be distinct non-null arrays");
  if (prec == DGX_F64) return apply_noalloc<double>(c, (const double *)x, (double *)y);
  if (prec == DGX_F32) return apply_noalloc<float>(c, (const float *)x, (float *)y);
  return dgx::set_error(c, DGX_ERR_ARG, "precision %d", prec);
}
