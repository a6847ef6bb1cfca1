// Consistent density-weighted mass and its inverse (arXiv:2505.00384, Sec. 3.3).
//
// The fast inverse of the block-diagonal operator A(rho) integrates with the
// r+1 point Gauss rule, so that A = Ia^T J Ia is inverted in closed form; the
// integration it replaces uses the consistent 2r+1 point rule of all other
// integrals, A_c = I^T J_c I, whose inverse has no closed form.  Here:
//   k_mass_cons (inverse = 0)  out = A_c(rho) in
//   k_mass_cons (inverse = 1)  out = A_c(rho)^-1 in by preconditioned conjugate
//                              gradients inside each cell, preconditioned by
//                              the fast inverse (spectrally close to A_c^-1,
//                              so a few iterations reach rounding level)
// for nf <= 3 fields of N^3 nodal values per cell.  One CTA per cell; every
// vector of the iteration lives in shared memory; the cell's scalars (one per
// field) come from deterministic block reductions, so every thread takes the
// same branch.  J_c = rho(x_q) w_q det J(x_q) at the (2r+1)^3 Gauss points.
#include "dgx_sweep.cuh"

namespace dgx {
namespace {

constexpr int kMcThreads = 128;
constexpr int kMcWarps = kMcThreads / 32;
constexpr int kMcRedDoubles = 16;  // kMcWarps * 3 partials + 3 results, padded
static_assert(kMcWarps * 3 + 3 <= kMcRedDoubles, "reduction scratch");

template <int N, int Q>
struct McL {
  static constexpr int N2 = N * N, N3 = N * N * N, Q2 = Q * Q, Q3 = Q * Q * Q;
  static constexpr int TAB = (tab_size(N, Q) + 1) & ~1;
  // tables, rho and rho at the fast points, J_c, the five vectors X R Z P W
  // (nf fields each), the sweep scratch S1 (Q N N), S2 (Q Q N), S3 (Q Q Q)
  static constexpr long long total(int nf) {
    return TAB + 2 * N3 + Q3 + 5LL * nf * N3 + (long long)nf * (N2 * Q + N * Q2 + Q3);
  }
};

// Sums over the cell of a_f . b_f for the nf fields (N3 values each), in
// double, fixed reduction order; every thread returns the same values.
template <typename T>
__device__ __forceinline__ void block_dots(int nf, int n, const T *a, const T *b, double *red, double out[3]) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    s0 += (double)a[i] * (double)b[i];
    if (nf > 1) s1 += (double)a[n + i] * (double)b[n + i];
    if (nf > 2) s2 += (double)a[2 * n + i] * (double)b[2 * n + i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, o);
    s1 += __shfl_down_sync(0xffffffffu, s1, o);
    s2 += __shfl_down_sync(0xffffffffu, s2, o);
  }
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  if (lane == 0) {
    red[wp * 3 + 0] = s0;
    red[wp * 3 + 1] = s1;
    red[wp * 3 + 2] = s2;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int w = 0; w < kMcWarps; ++w) t += red[w * 3 + threadIdx.x];
    red[kMcWarps * 3 + threadIdx.x] = t;
  }
  __syncthreads();
  out[0] = red[kMcWarps * 3 + 0];
  out[1] = red[kMcWarps * 3 + 1];
  out[2] = red[kMcWarps * 3 + 2];
  __syncthreads();  // the scratch is reused by the next call
}

// out = A_c v for nf fields: interpolate to the consistent points, scale by
// J_c, test with the basis (the transposed interpolation).
template <typename T, int N, int Q>
__device__ __forceinline__ void cons_apply(int nf, const T *Jc, const T *v, T *out, T *S1, T *S2, T *S3) {
  constexpr int Q3 = Q * Q * Q;
  sweep<T, N, 0, Q, N, N, N, N, M_I, M_I, M_I>(nf, 0u, v, S1);
  __syncthreads();
  sweep<T, N, 1, Q, N, Q, N, N, M_I, M_I, M_I>(nf, 0u, S1, S2);
  __syncthreads();
  sweep<T, N, 2, Q, N, Q, Q, N, M_I, M_I, M_I>(nf, 0u, S2, S3);
  __syncthreads();
  for (int idx = threadIdx.x; idx < nf * Q3; idx += blockDim.x) S3[idx] *= Jc[idx % Q3];
  __syncthreads();
  sweep<T, N, 2, N, Q, Q, Q, Q, M_IT, M_IT, M_IT>(nf, 0u, S3, S2);
  __syncthreads();
  sweep<T, N, 1, N, Q, Q, Q, N, M_IT, M_IT, M_IT>(nf, 0u, S2, S1);
  __syncthreads();
  sweep<T, N, 0, N, Q, Q, N, N, M_IT, M_IT, M_IT>(nf, 0u, S1, out);
  __syncthreads();
}

// stats[0]: largest iteration count of any cell; stats[1]: cells that did not
// reach the tolerance within maxit (or met a non-finite residual).
template <typename T, int N, int Q, bool CURVED>
__global__ void __launch_bounds__(kMcThreads) k_mass_cons(const OpP<T> P, const T *in, const T *__restrict__ rho,
                                                          T *out, long long Ntot, int nf, int inverse, int maxit,
                                                          double tol, int *__restrict__ stats) {
  using L = McL<N, Q>;
  constexpr int N2 = L::N2, N3 = L::N3, Q2 = L::Q2, Q3 = L::Q3;
  extern __shared__ __align__(16) unsigned char smraw[];
  double *red = reinterpret_cast<double *>(smraw);
  T *tab = reinterpret_cast<T *>(smraw + kMcRedDoubles * sizeof(double));
  T *s_rho = tab + L::TAB, *s_rq = s_rho + N3, *Jc = s_rq + N3;
  T *X = Jc + Q3, *R = X + nf * N3, *Z = R + nf * N3, *Pd = Z + nf * N3, *W = Pd + nf * N3;
  T *S1 = W + nf * N3, *S2 = S1 + nf * N2 * Q, *S3 = S2 + nf * N * Q2;
  const long long cell = blockIdx.x;
  const CellPos cp = cell_pos(P, cell);
  const T *colp = CURVED ? P.col + (long long)(cp.cx + P.nx * cp.cy) * col_size(N, Q) : nullptr;
  load_tables<T, N, Q>(P.tab, tab);
  for (int i = threadIdx.x; i < nf * N3; i += blockDim.x) {
    const int d = i / N3, node = i - d * N3;
    R[i] = in[(long long)d * Ntot + cell * N3 + node];
    if (d == 0) s_rho[node] = rho[cell * N3 + node];
  }
  __syncthreads();
  // J_c at the consistent points
  sweep<T, N, 0, Q, N, N, N, N, M_I, M_I, M_I>(1, 0u, s_rho, S1);
  __syncthreads();
  sweep<T, N, 1, Q, N, Q, N, N, M_I, M_I, M_I>(1, 0u, S1, S2);
  __syncthreads();
  sweep<T, N, 2, Q, N, Q, Q, N, M_I, M_I, M_I>(1, 0u, S2, S3);
  __syncthreads();
  const T *wq = tab + tab_off_wq(N, Q);
  for (int idx = threadIdx.x; idx < Q3; idx += blockDim.x) {
    const int i = idx % Q, j = (idx / Q) % Q, k = idx / Q2;
    T det = P.dx * P.dy * P.dz;
    if (CURVED) det *= T(1) - colp[col_off_hq(N, Q) + i + Q * j] * P.invH;
    Jc[idx] = S3[idx] * wq[i] * wq[j] * wq[k] * det;
  }
  __syncthreads();
  if (!inverse) {
    cons_apply<T, N, Q>(nf, Jc, R, W, S1, S2, S3);
    for (int i = threadIdx.x; i < nf * N3; i += blockDim.x) {
      const int d = i / N3, node = i - d * N3;
      out[(long long)d * Ntot + cell * N3 + node] = W[i];
    }
    return;
  }
  rho_fast<T, N, Q>(tab, s_rho, S1, S2, s_rq);
  double bn2[3], rz[3], rr[3], pq[3], rzn[3];
  block_dots<T>(nf, N3, R, R, red, bn2);
  // X = M^-1 b (M = fast mass); R = b - A_c X; Z = M^-1 R; P = Z
  for (int i = threadIdx.x; i < nf * N3; i += blockDim.x) X[i] = R[i];
  __syncthreads();
  fast_inverse<T, N, Q, CURVED>(P, tab, colp, s_rq, nf, X, S1);
  cons_apply<T, N, Q>(nf, Jc, X, W, S1, S2, S3);
  for (int i = threadIdx.x; i < nf * N3; i += blockDim.x) {
    R[i] -= W[i];
    Z[i] = R[i];
  }
  __syncthreads();
  fast_inverse<T, N, Q, CURVED>(P, tab, colp, s_rq, nf, Z, S1);
  for (int i = threadIdx.x; i < nf * N3; i += blockDim.x) Pd[i] = Z[i];
  __syncthreads();
  block_dots<T>(nf, N3, R, Z, red, rz);
  const double tol2 = tol * tol;
  int it = 0;
  bool converged = false;
  for (;;) {
    block_dots<T>(nf, N3, R, R, red, rr);
    bool done[3], all = true, finite = true;
    for (int f = 0; f < 3; ++f) {
      finite = finite && (f >= nf || isfinite(rr[f]));
      done[f] = f >= nf || rr[f] <= tol2 * bn2[f];
      all = all && done[f];
    }
    if (all) {
      converged = true;
      break;
    }
    if (!finite || it >= maxit) break;
    cons_apply<T, N, Q>(nf, Jc, Pd, W, S1, S2, S3);
    block_dots<T>(nf, N3, Pd, W, red, pq);
    double al[3];
    for (int f = 0; f < 3; ++f) al[f] = (done[f] || !(pq[f] > 0.0)) ? 0.0 : rz[f] / pq[f];
    for (int i = threadIdx.x; i < nf * N3; i += blockDim.x) {
      const T a = T(al[i / N3]);
      X[i] += a * Pd[i];
      R[i] -= a * W[i];
      Z[i] = R[i];
    }
    __syncthreads();
    fast_inverse<T, N, Q, CURVED>(P, tab, colp, s_rq, nf, Z, S1);
    block_dots<T>(nf, N3, R, Z, red, rzn);
    double be[3];
    for (int f = 0; f < 3; ++f) {
      be[f] = (done[f] || rz[f] == 0.0) ? 0.0 : rzn[f] / rz[f];
      rz[f] = rzn[f];
    }
    for (int i = threadIdx.x; i < nf * N3; i += blockDim.x) Pd[i] = Z[i] + T(be[i / N3]) * Pd[i];
    __syncthreads();
    ++it;
  }
  for (int i = threadIdx.x; i < nf * N3; i += blockDim.x) {
    const int d = i / N3, node = i - d * N3;
    out[(long long)d * Ntot + cell * N3 + node] = X[i];
  }
  if (stats && threadIdx.x == 0) {
    atomicMax(&stats[0], it);
    if (!converged) atomicAdd(&stats[1], 1);
  }
}

template <typename Kern>
int prep_mc(dgx_ctx *c, Kern k, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  return check_cuda(c, e, "cudaFuncSetAttribute (k_mass_cons)");
}

constexpr size_t kMcMaxSmem = 227 * 1024;

template <typename T, int N, bool CURVED>
int mcons_impl(dgx_ctx *c, const T *in, const T *rho, T *out, cudaStream_t s, int nf, int inverse) {
  constexpr int Q = 2 * N - 1;
  auto k = k_mass_cons<T, N, Q, CURVED>;
  const double tol = sizeof(T) == 8 ? c->mass_tol : std::fmax(c->mass_tol, 1e-5);
  // all fields in one pass when they fit in shared memory, else one field per pass
  const int per = (kMcRedDoubles * sizeof(double) + sizeof(T) * (size_t)McL<N, Q>::total(nf) <= kMcMaxSmem) ? nf : 1;
  const size_t smem = kMcRedDoubles * sizeof(double) + sizeof(T) * (size_t)McL<N, Q>::total(per);
  if (smem > kMcMaxSmem) return set_error(c, DGX_ERR_ARG, "consistent mass: degree %d needs %zu bytes of shared memory", N - 1, smem);
  if (int e = prep_mc(c, k, smem)) return e;
  const OpP<T> P = make_params<T>(c);
  for (int f0 = 0; f0 < nf; f0 += per) {
    count_launch();
    k<<<(unsigned)c->ncell, kMcThreads, smem, s>>>(P, in + (size_t)f0 * c->N, rho, out + (size_t)f0 * c->N, c->N,
                                                   per, inverse, c->mass_maxit, tol, c->mass_stats);
    if (int e = check_cuda(c, cudaGetLastError(), "k_mass_cons launch")) return e;
  }
  return 0;
}

#define DGX_DISPATCH_MC(CALL)                                                      \
  switch (c->n) {                                                                  \
    case 2: return c->curved ? CALL(2, true) : CALL(2, false);                     \
    case 3: return c->curved ? CALL(3, true) : CALL(3, false);                     \
    case 4: return c->curved ? CALL(4, true) : CALL(4, false);                     \
    case 5: return c->curved ? CALL(5, true) : CALL(5, false);                     \
    case 6: return c->curved ? CALL(6, true) : CALL(6, false);                     \
    case 7: return c->curved ? CALL(7, true) : CALL(7, false);                     \
    default: return set_error(c, DGX_ERR_ARG, "unsupported degree %d", c->n - 1);  \
  }

}  // namespace

template <typename T>
int launch_mass_cons(dgx_ctx *c, const T *in, const T *rho, T *out, cudaStream_t s, int nf, int inverse) {
  if (nf < 1 || nf > 3) return set_error(c, DGX_ERR_ARG, "consistent mass: 1 to 3 fields");
  if (int e = upload_const_tables(c)) return e;
#define CALL_MC(NN, CC) mcons_impl<T, NN, CC>(c, in, rho, out, s, nf, inverse)
  DGX_DISPATCH_MC(CALL_MC)
#undef CALL_MC
}
template int launch_mass_cons<double>(dgx_ctx *, const double *, const double *, double *, cudaStream_t, int, int);
template int launch_mass_cons<float>(dgx_ctx *, const float *, const float *, float *, cudaStream_t, int, int);

}  // namespace dgx
