// Launchers of the fused operator kernels (dgx_fused.cuh), instantiated per
// precision and degree by the small dgx_fused_*.cu translation units so that
// the build compiles them in parallel.
#pragma once

#include <set>
#include <utility>

#include "dgx_fused.cuh"

namespace dgx {
namespace {

// Dynamic shared memory above 48 KB and the maximum carveout, set once per
// kernel and device (so that launches inside stream capture make no calls).
template <typename Kern>
int fprep(dgx_ctx *c, Kern k, size_t smem) {
  static std::mutex mu;
  static std::set<std::pair<int, const void *>> done;
  const std::pair<int, const void *> key(c->device, reinterpret_cast<const void *>(k));
  {
    std::lock_guard<std::mutex> lk(mu);
    if (done.count(key)) return 0;
  }
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> lk(mu);
    done.insert(key);
  }
  return check_cuda(c, e, "cudaFuncSetAttribute (fused operator)");
}

// One launch per patch of the mesh (two on non-conforming meshes), each on its
// own cells with its own parameters; the component stride stays c->N.
template <typename T, int N, bool CURVED, bool INV, int CPB, int NT>
int fgrad_go(dgx_ctx *c, double alpha, const store_t<T> *p, const store_t<T> *rho, store_t<T> *V, cudaStream_t s) {
  const size_t smem = sizeof(T) * (size_t)CPB * FGradL<N, CURVED>::per_cell;
  if (smem > kFusedMaxSmem) return set_error(c, DGX_ERR_ARG, "fused gradient kernel: %zu bytes of shared memory", smem);
  auto k = kf_grad<T, N, CURVED, INV, CPB, NT>;
  if (int e = fprep(c, k, smem)) return e;
  for (int pi = 0; pi < num_patches(c); ++pi) {
    OpP<T> P = make_params<T>(c, pi);
    if (alpha >= 0.0) P.alpha = (T)alpha;
    const int ncell = (int)patch_ncell(c, pi);
    const long long o = patch_cell0(c, pi) * N * N * N;
    count_launch();
    k<<<(unsigned)((ncell + CPB - 1) / CPB), NT, smem, s>>>(P, p + o, rho + o, V + o, c->N, ncell);
  }
  return check_cuda(c, cudaGetLastError(), "kf_grad launch");
}

template <typename T, int N, bool CURVED, bool KQ, int CPB, int NT>
int fdiv_go(dgx_ctx *c, double alpha, const store_t<T> *V, const store_t<T> *p, const store_t<T> *pk, store_t<T> *y,
            const store_t<T> *kq, cudaStream_t s) {
  const size_t smem = sizeof(T) * (size_t)CPB * FDivL<N, CURVED, KQ>::per_cell;
  if (smem > kFusedMaxSmem) return set_error(c, DGX_ERR_ARG, "fused divergence kernel: %zu bytes of shared memory", smem);
  auto k = kf_div<T, N, CURVED, KQ, CPB, NT>;
  if (int e = fprep(c, k, smem)) return e;
  constexpr int Q = 2 * N - 1;
  for (int pi = 0; pi < num_patches(c); ++pi) {
    OpP<T> P = make_params<T>(c, pi);
    if (alpha >= 0.0) P.alpha = (T)alpha;
    const int ncell = (int)patch_ncell(c, pi);
    const long long o = patch_cell0(c, pi) * N * N * N, oq = patch_cell0(c, pi) * Q * Q * Q;
    count_launch();
    k<<<(unsigned)((ncell + CPB - 1) / CPB), NT, smem, s>>>(P, V + o, p + o, pk + o, y + o, c->N, ncell,
                                                           kq ? kq + oq : nullptr);
  }
  return check_cuda(c, cudaGetLastError(), "kf_div launch");
}

}  // namespace

template <typename T, int N, bool CURVED>
int fused_grad(dgx_ctx *c, const store_t<T> *p, const store_t<T> *rho, store_t<T> *V, cudaStream_t s, bool inv,
               double alpha, int cfg) {
  if (int e = upload_fused_tables(c)) return e;
  if (!inv) return fgrad_go<T, N, CURVED, false, fused_cpb(N, 0), fused_nt(N, 0)>(c, alpha, p, rho, V, s);
  if (cfg == 1) return fgrad_go<T, N, CURVED, true, fused_cpb(N, 1), fused_nt(N, 1)>(c, alpha, p, rho, V, s);
  return fgrad_go<T, N, CURVED, true, fused_cpb(N, 0), fused_nt(N, 0)>(c, alpha, p, rho, V, s);
}

template <typename T, int N, bool CURVED>
int fused_div(dgx_ctx *c, const store_t<T> *V, const store_t<T> *p, const store_t<T> *pk, store_t<T> *y,
              cudaStream_t s, double alpha, const store_t<T> *kq, int cfg) {
  if (int e = upload_fused_tables(c)) return e;
  if constexpr (sizeof(store_t<T>) == 8) {
    if (kq) {
      if (cfg == 1) return fdiv_go<T, N, CURVED, true, fused_cpb(N, 1), fused_nt(N, 1)>(c, alpha, V, p, pk, y, kq, s);
      return fdiv_go<T, N, CURVED, true, fused_cpb(N, 0), fused_nt(N, 0)>(c, alpha, V, p, pk, y, kq, s);
    }
    return fdiv_go<T, N, CURVED, false, fused_cpb(N, 0), fused_nt(N, 0)>(c, alpha, V, p, pk, y, nullptr, s);
  } else {
    if (cfg == 1) return fdiv_go<T, N, CURVED, false, fused_cpb(N, 1), fused_nt(N, 1)>(c, alpha, V, p, pk, y, nullptr, s);
    return fdiv_go<T, N, CURVED, false, fused_cpb(N, 0), fused_nt(N, 0)>(c, alpha, V, p, pk, y, nullptr, s);
  }
}

// Multi-mesh operator y = S x of ensemble members of degree N = r+1 in fused
// configuration cfg; cta_off (device, nmem + 1 entries) from fused_cpb(N, cfg).
template <typename T, int N, bool CURVED>
int fused_operator_multi(dgx_ctx *c0, const EnsMember<T> *mem, int nmem, const int *cta_off, int nblocks,
                         const store_t<T> *x, store_t<T> *y, cudaStream_t s, int cfg) {
  if (int e = upload_fused_tables(c0)) return e;
  auto go = [&](auto kg, auto kd, int cpb, int nt) -> int {
    const size_t sg = sizeof(T) * (size_t)cpb * FGradL<N, CURVED>::per_cell;
    const size_t sd = sizeof(T) * (size_t)cpb * FDivL<N, CURVED, false>::per_cell;
    if (sg > kFusedMaxSmem || sd > kFusedMaxSmem) return set_error(c0, DGX_ERR_ARG, "fused multi-mesh kernels do not fit");
    if (int e = fprep(c0, kg, sg)) return e;
    if (int e = fprep(c0, kd, sd)) return e;
    count_launch(2);
    kg<<<(unsigned)nblocks, nt, sg, s>>>(mem, nmem, cta_off, x);
    kd<<<(unsigned)nblocks, nt, sd, s>>>(mem, nmem, cta_off, x, y);
    return check_cuda(c0, cudaGetLastError(), "fused multi-mesh operator launch");
  };
  if (cfg == 1)
    return go(kf_grad_multi<T, N, CURVED, fused_cpb(N, 1), fused_nt(N, 1)>,
              kf_div_multi<T, N, CURVED, fused_cpb(N, 1), fused_nt(N, 1)>, fused_cpb(N, 1), fused_nt(N, 1));
  return go(kf_grad_multi<T, N, CURVED, fused_cpb(N, 0), fused_nt(N, 0)>,
            kf_div_multi<T, N, CURVED, fused_cpb(N, 0), fused_nt(N, 0)>, fused_cpb(N, 0), fused_nt(N, 0));
}

// Shared memory of one fused configuration (bytes), for the variant list.
template <typename T, int N, bool CURVED>
size_t fused_smem(int cfg) {
  const int cpb = fused_cpb(N, cfg);
  const size_t g = sizeof(T) * (size_t)cpb * FGradL<N, CURVED>::per_cell;
  const size_t d = sizeof(T) * (size_t)cpb * FDivL<N, CURVED, sizeof(store_t<T>) == 8>::per_cell;
  return g > d ? g : d;
}

#define DGX_FUSED_INSTANTIATE(T, NN)                                                                           \
  template int fused_grad<T, NN, false>(dgx_ctx *, const store_t<T> *, const store_t<T> *, store_t<T> *,       \
                                        cudaStream_t, bool, double, int);                                      \
  template int fused_grad<T, NN, true>(dgx_ctx *, const store_t<T> *, const store_t<T> *, store_t<T> *,        \
                                       cudaStream_t, bool, double, int);                                       \
  template int fused_div<T, NN, false>(dgx_ctx *, const store_t<T> *, const store_t<T> *, const store_t<T> *,  \
                                       store_t<T> *, cudaStream_t, double, const store_t<T> *, int);           \
  template int fused_div<T, NN, true>(dgx_ctx *, const store_t<T> *, const store_t<T> *, const store_t<T> *,   \
                                      store_t<T> *, cudaStream_t, double, const store_t<T> *, int);            \
  template size_t fused_smem<T, NN, false>(int);                                                                \
  template size_t fused_smem<T, NN, true>(int);

#define DGX_FUSED_MULTI_INSTANTIATE(T, NN)                                                                     \
  template int fused_operator_multi<T, NN, false>(dgx_ctx *, const EnsMember<T> *, int, const int *, int,       \
                                                  const store_t<T> *, store_t<T> *, cudaStream_t, int);         \
  template int fused_operator_multi<T, NN, true>(dgx_ctx *, const EnsMember<T> *, int, const int *, int,        \
                                                 const store_t<T> *, store_t<T> *, cudaStream_t, int);

}  // namespace dgx
