// Geometric multigrid preconditioner for the pressure system (arXiv:2505.00384,
// Sec. 3.1: conjugate gradients with geometric multigrid for the SPD systems;
// for the non-symmetric Schur system the paper notes that no theory covers
// multigrid, so there it is an experiment).
//
// Hierarchy: level 0 is the context's own mesh and coefficients; level l has
// nx, ny, nz halved l times (same domain, degree, terrain and boundaries), so
// that a coarse cell is the union of 2 x 2 x 2 fine cells and the reference
// coordinates nest exactly.  Each coarse level is a context of its own (its
// mesh tables, coefficient copies, Jacobi diagonals, operator kernels and
// autotuning) working on the same stream.
//   prolongation P  coarse cell polynomial evaluated at the fine GLL nodes of
//                   each child (k_prolong), exact for the coarse polynomial;
//   restriction R   = P^T (k_restrict: each coarse cell gathers its 8 children,
//                   no atomics);
//   coefficients    rho, p_k at the coarse nodes by evaluating the fine field
//                   in the child that holds the node (k_inject; at a child
//                   interface the lower child);
//   smoother        Chebyshev iteration on D^-1 S (Saad, Iterative Methods for
//                   Sparse Linear Systems, Alg. 12.1) over
//                   [lambda_max / range, 1.1 lambda_max], D the Helmholtz
//                   diagonal of the level, lambda_max from power iteration on
//                   D^-1 S from the fixed vector v_i = frac(0.618... (i+1)) - 1/2;
//   coarsest level  CG (SPD) or FGMRES with the Helmholtz Jacobi, to a relative
//                   tolerance within a bounded number of iterations;
//   V-cycle         from zero: pre-smooth, restrict the residual, cycle one
//                   level down, prolong and correct, post-smooth.
#include <cmath>
#include <cstring>
#include <vector>

#include "dgx_common.cuh"

namespace dgx {

struct Multigrid {
  dgx_mg_opts o{};
  std::vector<dgx_ctx *> lv;                   // lv[0] = the owning context (not owned here)
  std::vector<double *> rho, pk;               // coefficient copies of levels >= 1
  std::vector<double *> b, x, r, d, t;         // work vectors per level (b[0], x[0] unused)
  std::vector<double> lmax;                    // power-iteration estimates per level
  double *E = nullptr, *F = nullptr;           // device transfer tables
  int *side = nullptr;
  double *dred = nullptr;                      // reduction scratch (device, 1 value)
  long long coef_version = -1;                 // of the owning context when set up
  std::vector<void *> owned;
};

namespace {

constexpr int kT = 256;

int blocks_for(long long n) {
  const long long b = (n + kT - 1) / kT;
  return (int)(b < 1 ? 1 : (b > 65535LL * 16 ? 65535LL * 16 : b));
}

// fine DoF i -> value of the parent coarse cell's polynomial at that node
template <int N>
__global__ void __launch_bounds__(kT) k_prolong(int cnx, int cny, const double *__restrict__ E,
                                                const double *__restrict__ xc, double *__restrict__ xf, long long nf) {
  constexpr int N2 = N * N, N3 = N2 * N;
  __shared__ double sE[2 * N2];
  for (int k = threadIdx.x; k < 2 * N2; k += blockDim.x) sE[k] = E[k];
  __syncthreads();
  const int fnx = 2 * cnx, fny = 2 * cny;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nf; i += (long long)gridDim.x * blockDim.x) {
    const long long fc = i / N3;
    const int node = (int)(i - fc * N3), a = node % N, b = (node / N) % N, c = node / N2;
    const int fx = (int)(fc % fnx), fy = (int)((fc / fnx) % fny), fz = (int)(fc / ((long long)fnx * fny));
    const long long parent = (fx >> 1) + (long long)cnx * ((fy >> 1) + (long long)cny * (fz >> 1));
    const double *Ex = sE + (fx & 1) * N2 + a * N, *Ey = sE + (fy & 1) * N2 + b * N, *Ez = sE + (fz & 1) * N2 + c * N;
    const double *src = xc + parent * N3;
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      double sj = 0.0;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        double si = 0.0;
#pragma unroll
        for (int ii = 0; ii < N; ++ii) si += Ex[ii] * src[ii + N * j + N2 * k];
        sj += Ey[j] * si;
      }
      s += Ez[k] * sj;
    }
    xf[i] = s;
  }
}

// coarse DoF (node (i, j, k) of cell cc) <- sum over its 8 children of P^T
template <int N>
__global__ void __launch_bounds__(kT) k_restrict(int cnx, int cny, const double *__restrict__ E,
                                                 const double *__restrict__ rf, double *__restrict__ xc, long long nc) {
  constexpr int N2 = N * N, N3 = N2 * N;
  __shared__ double sE[2 * N2];
  for (int k = threadIdx.x; k < 2 * N2; k += blockDim.x) sE[k] = E[k];
  __syncthreads();
  const int fnx = 2 * cnx, fny = 2 * cny;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < nc; id += (long long)gridDim.x * blockDim.x) {
    const long long cc = id / N3;
    const int node = (int)(id - cc * N3), i = node % N, j = (node / N) % N, k = node / N2;
    const int cx = (int)(cc % cnx), cy = (int)((cc / cnx) % cny), cz = (int)(cc / ((long long)cnx * cny));
    double s = 0.0;
    for (int sz = 0; sz < 2; ++sz)
      for (int sy = 0; sy < 2; ++sy)
        for (int sx = 0; sx < 2; ++sx) {
          const long long child = (2 * cx + sx) + (long long)fnx * ((2 * cy + sy) + (long long)fny * (2 * cz + sz));
          const double *src = rf + child * N3;
          double sc = 0.0;
#pragma unroll
          for (int c = 0; c < N; ++c) {
            double sb = 0.0;
#pragma unroll
            for (int b = 0; b < N; ++b) {
              double sa = 0.0;
#pragma unroll
              for (int a = 0; a < N; ++a) sa += sE[sx * N2 + a * N + i] * src[a + N * b + N2 * c];
              sb += sE[sy * N2 + b * N + j] * sa;
            }
            sc += sE[sz * N2 + c * N + k] * sb;
          }
          s += sc;
        }
    xc[id] = s;
  }
}

// coarse nodal value of a fine field: the fine child holding the node, evaluated there
template <int N>
__global__ void __launch_bounds__(kT) k_inject(int cnx, int cny, const int *__restrict__ side,
                                               const double *__restrict__ F, const double *__restrict__ vf,
                                               double *__restrict__ vc, long long nc) {
  constexpr int N2 = N * N, N3 = N2 * N;
  __shared__ double sF[N2];
  __shared__ int sS[N];
  for (int k = threadIdx.x; k < N2; k += blockDim.x) sF[k] = F[k];
  for (int k = threadIdx.x; k < N; k += blockDim.x) sS[k] = side[k];
  __syncthreads();
  const int fnx = 2 * cnx, fny = 2 * cny;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < nc; id += (long long)gridDim.x * blockDim.x) {
    const long long cc = id / N3;
    const int node = (int)(id - cc * N3), a = node % N, b = (node / N) % N, c = node / N2;
    const int cx = (int)(cc % cnx), cy = (int)((cc / cnx) % cny), cz = (int)(cc / ((long long)cnx * cny));
    const long long child = (2 * cx + sS[a]) + (long long)fnx * ((2 * cy + sS[b]) + (long long)fny * (2 * cz + sS[c]));
    const double *src = vf + child * N3;
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      double sj = 0.0;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        double si = 0.0;
#pragma unroll
        for (int i = 0; i < N; ++i) si += sF[a * N + i] * src[i + N * j + N2 * k];
        sj += sF[b * N + j] * si;
      }
      s += sF[c * N + k] * sj;
    }
    vc[id] = s;
  }
}

#define MG_DISPATCH(N_, CALL) \
  switch (N_) {               \
    case 2: CALL(2); break;   \
    case 3: CALL(3); break;   \
    case 4: CALL(4); break;   \
    case 5: CALL(5); break;   \
    case 6: CALL(6); break;   \
    case 7: CALL(7); break;   \
    default: return set_error(c, DGX_ERR_ARG, "unsupported degree"); \
  }

// coarse level cf (its mesh) <-> fine level ff
int prolong(dgx_ctx *c, Multigrid &G, dgx_ctx *cf, const double *xc, double *xf) {
  const int cnx = cf->mesh.nx, cny = cf->mesh.ny;
  const long long nf = 8 * cf->N;
#define CALLP(NN)     \
  count_launch();     \
  k_prolong<NN><<<blocks_for(nf), kT, 0, c->stream>>>(cnx, cny, G.E, xc, xf, nf)
  MG_DISPATCH(c->n, CALLP)
#undef CALLP
  return check_cuda(c, cudaGetLastError(), "k_prolong");
}

int restrict_(dgx_ctx *c, Multigrid &G, dgx_ctx *cf, const double *rf, double *xc) {
  const int cnx = cf->mesh.nx, cny = cf->mesh.ny;
  const long long nc = cf->N;
#define CALLR(NN)     \
  count_launch();     \
  k_restrict<NN><<<blocks_for(nc), kT, 0, c->stream>>>(cnx, cny, G.E, rf, xc, nc)
  MG_DISPATCH(c->n, CALLR)
#undef CALLR
  return check_cuda(c, cudaGetLastError(), "k_restrict");
}

int inject(dgx_ctx *c, Multigrid &G, dgx_ctx *cf, const double *vf, double *vc) {
  const int cnx = cf->mesh.nx, cny = cf->mesh.ny;
  const long long nc = cf->N;
#define CALLI(NN)     \
  count_launch();     \
  k_inject<NN><<<blocks_for(nc), kT, 0, c->stream>>>(cnx, cny, G.side, G.F, vf, vc, nc)
  MG_DISPATCH(c->n, CALLI)
#undef CALLI
  return check_cuda(c, cudaGetLastError(), "k_inject");
}

int norm2(dgx_ctx *c, Multigrid &G, dgx_ctx *lc, const double *v, double *out) {
  vec_dot<double>(lc->N, v, v, lc->red, G.dred, c->stream);
  if (int e = check_cuda(c, cudaMemcpyAsync(out, G.dred, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "memcpy"))
    return e;
  return check_cuda(c, cudaStreamSynchronize(c->stream), "sync");
}

int apply_level(dgx_ctx *c, dgx_ctx *lc, const double *x, double *y) {
  if (int e = dgx_apply_operator(lc, DGX_F64, x, y)) return lc == c ? e : set_error(c, e, "level: %s", lc->err.c_str());
  return 0;
}

// lambda_max of D^-1 S on level l by power iteration from the fixed vector
int power_lambda(dgx_ctx *c, Multigrid &G, int l) {
  dgx_ctx *lc = G.lv[l];
  const long long n = lc->N;
  std::vector<double> v0(n);
  for (long long i = 0; i < n; ++i) {
    const double v = 0.6180339887498949 * ((double)i + 1.0);
    v0[i] = v - std::floor(v) - 0.5;
  }
  double *v = G.r[l], *w = G.t[l];
  if (int e = check_cuda(c, cudaMemcpyAsync(v, v0.data(), n * sizeof(double), cudaMemcpyHostToDevice, c->stream), "memcpy"))
    return e;
  double nn = 0.0;
  if (int e = norm2(c, G, lc, v, &nn)) return e;
  vec_axpby<double>(n, 1.0 / std::sqrt(nn), v, 0.0, v, c->stream);
  double lam = 0.0;
  for (int k = 0; k < G.o.power_its; ++k) {
    if (int e = apply_level(c, lc, v, w)) return e;
    vec_mul<double>(n, lc->dinv64[DGX_PC_HELMHOLTZ], w, w, c->stream);
    if (int e = norm2(c, G, lc, w, &nn)) return e;
    lam = std::sqrt(nn);
    if (!(lam > 0.0) || !std::isfinite(lam)) return set_error(c, DGX_ERR_BREAKDOWN, "multigrid: power iteration on level %d", l);
    vec_axpby<double>(n, 1.0 / lam, w, 0.0, v, c->stream);
  }
  G.lmax[l] = lam;
  return 0;
}

// coefficients of levels >= 1 from the owning context's current ones, diagonals, bounds
int refresh(dgx_ctx *c, Multigrid &G) {
  const int L = (int)G.lv.size();
  for (int l = 1; l < L; ++l) {
    dgx_ctx *f = G.lv[l - 1], *lc = G.lv[l];
    if (int e = inject(c, G, lc, f->rho64, G.rho[l])) return e;
    if (int e = inject(c, G, lc, f->pk64, G.pk[l])) return e;
    if (int e = dgx_set_coefficients(lc, G.rho[l], G.pk[l], c->alpha, c->gamma))
      return set_error(c, e, "level %d: %s", l, lc->err.c_str());
  }
  for (int l = 0; l < L; ++l) {
    if (int e = ensure_diag(G.lv[l], true)) return l ? set_error(c, e, "level %d: %s", l, G.lv[l]->err.c_str()) : e;
    if (int e = power_lambda(c, G, l)) return e;
  }
  G.coef_version = c->coef_version;
  return 0;
}

// Saad Alg. 12.1 on D^-1 S x = D^-1 b, degree steps from x (zero_start: x = 0)
int chebyshev(dgx_ctx *c, Multigrid &G, int l, const double *b, double *x, bool zero_start) {
  dgx_ctx *lc = G.lv[l];
  const long long n = lc->N;
  const double *dinv = lc->dinv64[DGX_PC_HELMHOLTZ];
  const double lmax = 1.1 * G.lmax[l], lmin = G.lmax[l] / G.o.smooth_range;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
  double *r = G.r[l], *d = G.d[l], *t = G.t[l];
  if (zero_start) {
    cudaMemsetAsync(x, 0, n * sizeof(double), c->stream);
    cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  } else {
    if (int e = apply_level(c, lc, x, t)) return e;
    cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    vec_axpby<double>(n, -1.0, t, 1.0, r, c->stream);
  }
  double rho = 1.0 / sigma;
  vec_mul<double>(n, dinv, r, d, c->stream);
  vec_axpby<double>(n, 0.0, d, 1.0 / theta, d, c->stream);  // d = dinv r / theta
  for (int k = 0; k < G.o.degree; ++k) {
    vec_axpby<double>(n, 1.0, d, 1.0, x, c->stream);
    if (k + 1 == G.o.degree) break;
    if (int e = apply_level(c, lc, d, t)) return e;
    vec_axpby<double>(n, -1.0, t, 1.0, r, c->stream);
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    vec_mul<double>(n, dinv, r, t, c->stream);
    vec_axpby<double>(n, 2.0 * rho_new / delta, t, rho_new * rho, d, c->stream);
    rho = rho_new;
  }
  return 0;
}

int vcycle(dgx_ctx *c, Multigrid &G, int l, const double *b, double *x) {
  dgx_ctx *lc = G.lv[l];
  const long long n = lc->N;
  const int L = (int)G.lv.size();
  if (l == L - 1) {  // coarsest: Krylov with the Helmholtz Jacobi from zero
    dgx_solve_opts so;
    dgx_default_solve_opts(&so);
    so.method = G.o.coarse_solver == 1 ? DGX_SOLVER_FGMRES : DGX_SOLVER_CG;
    so.pc = DGX_PC_HELMHOLTZ;
    so.tol = G.o.coarse_tol;
    so.maxit = G.o.coarse_maxit;
    so.use_x0 = 0;
    dgx_solve_info si;
    const int e = dgx_solve_pressure(lc, b, x, &so, &si);
    if (e < 0) return lc == c ? e : set_error(c, e, "coarsest level: %s", lc->err.c_str());
    return 0;
  }
  if (int e = chebyshev(c, G, l, b, x, true)) return e;
  double *r = G.r[l], *t = G.t[l];
  if (int e = apply_level(c, lc, x, t)) return e;
  cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  vec_axpby<double>(n, -1.0, t, 1.0, r, c->stream);
  dgx_ctx *cc = G.lv[l + 1];
  if (int e = restrict_(c, G, cc, r, G.b[l + 1])) return e;
  if (int e = vcycle(c, G, l + 1, G.b[l + 1], G.x[l + 1])) return e;
  if (int e = prolong(c, G, cc, G.x[l + 1], t)) return e;
  vec_axpby<double>(n, 1.0, t, 1.0, x, c->stream);
  return chebyshev(c, G, l, b, x, false);
}

template <typename T>
int galloc(dgx_ctx *c, Multigrid &G, T **p, size_t elems) {
  void *q = nullptr;
  if (int e = check_cuda(c, cudaMalloc(&q, (elems ? elems : 1) * sizeof(T)), "cudaMalloc (multigrid)")) return e;
  G.owned.push_back(q);
  *p = reinterpret_cast<T *>(q);
  return 0;
}

}  // namespace

void mg_free(dgx_ctx *c) {
  if (!c || !c->mg) return;
  Multigrid *G = c->mg;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  for (size_t l = 1; l < G->lv.size(); ++l) dgx_destroy(G->lv[l]);
  for (void *p : G->owned) cudaFree(p);
  delete G;
  c->mg = nullptr;
}

bool mg_ready(const dgx_ctx *c) { return c && c->mg != nullptr; }

int mg_vcycle(dgx_ctx *c, const double *b, double *z) {
  if (!c->mg) return set_error(c, DGX_ERR_STATE, "no multigrid hierarchy (call dgx_mg_setup)");
  Multigrid &G = *c->mg;
  if (G.coef_version != c->coef_version)  // coefficients changed since the set-up
    if (int e = refresh(c, G)) return e;
  return vcycle(c, G, 0, b, z);
}

}  // namespace dgx

using namespace dgx;

extern "C" {

void dgx_default_mg_opts(dgx_mg_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->levels = 3;
  o->degree = 3;
  o->power_its = 15;
  o->coarse_maxit = 500;
  o->coarse_solver = 0;
  o->smooth_range = 15.0;
  o->coarse_tol = 1e-10;
}

int dgx_mg_setup(dgx_ctx *c, const dgx_mg_opts *opts) {
  if (!c) return DGX_ERR_ARG;
  if (!c->has_mesh) return set_error(c, DGX_ERR_STATE, "no mesh (call dgx_mesh_build)");
  if (!c->has_coef) return set_error(c, DGX_ERR_STATE, "no coefficients (call dgx_set_coefficients)");
  if (c->nc) return set_error(c, DGX_ERR_STATE, "multigrid is not available on non-conforming meshes");
  dgx_mg_opts o;
  if (opts) o = *opts;
  else dgx_default_mg_opts(&o);
  if (o.levels < 2 || o.levels > 12 || o.degree < 1 || o.power_its < 1 || o.coarse_maxit < 1 || !(o.smooth_range > 1.0) ||
      !(o.coarse_tol > 0.0) || (o.coarse_solver != 0 && o.coarse_solver != 1))
    return set_error(c, DGX_ERR_ARG, "multigrid options: need 2 <= levels <= 12, degree >= 1, power_its >= 1, "
                                     "coarse_maxit >= 1, smooth_range > 1, coarse_tol > 0, coarse_solver 0 or 1");
  const int f = 1 << (o.levels - 1);
  if (c->mesh.nx % f || c->mesh.ny % f || c->mesh.nz % f)
    return set_error(c, DGX_ERR_ARG, "multigrid: nx, ny, nz must be divisible by 2^(levels-1) = %d", f);
  mg_free(c);
  Multigrid *G = new Multigrid();
  c->mg = G;
  G->o = o;
  auto fail = [&](int e) {
    mg_free(c);
    return e;
  };
  std::vector<double> E, F;
  std::vector<int> side;
  if (!child_tables(c->n - 1, E, side, F)) return fail(set_error(c, DGX_ERR_ARG, "multigrid tables"));
  int e;
  if ((e = galloc(c, *G, &G->E, E.size())) || (e = galloc(c, *G, &G->F, F.size())) ||
      (e = galloc(c, *G, &G->side, side.size())) || (e = galloc(c, *G, &G->dred, 1)))
    return fail(e);
  cudaMemcpy(G->E, E.data(), E.size() * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(G->F, F.data(), F.size() * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(G->side, side.data(), side.size() * sizeof(int), cudaMemcpyHostToDevice);
  G->lv.push_back(c);
  for (int l = 1; l < o.levels; ++l) {
    dgx_ctx *lc = nullptr;
    if ((e = dgx_create(&lc, c->device, c->stream))) return fail(set_error(c, e, "level %d: context", l));
    G->lv.push_back(lc);
    dgx_mesh_desc d = c->mesh;
    d.nx >>= l;
    d.ny >>= l;
    d.nz >>= l;
    if ((e = dgx_mesh_build(lc, &d))) return fail(set_error(c, e, "level %d: %s", l, lc->err.c_str()));
  }
  const int L = o.levels;
  G->rho.assign(L, nullptr);
  G->pk.assign(L, nullptr);
  G->b.assign(L, nullptr);
  G->x.assign(L, nullptr);
  G->r.assign(L, nullptr);
  G->d.assign(L, nullptr);
  G->t.assign(L, nullptr);
  G->lmax.assign(L, 0.0);
  for (int l = 0; l < L; ++l) {
    const size_t n = (size_t)G->lv[l]->N;
    if (l > 0 && ((e = galloc(c, *G, &G->rho[l], n)) || (e = galloc(c, *G, &G->pk[l], n)) ||
                  (e = galloc(c, *G, &G->b[l], n)) || (e = galloc(c, *G, &G->x[l], n))))
      return fail(e);
    if ((e = galloc(c, *G, &G->r[l], n)) || (e = galloc(c, *G, &G->d[l], n)) || (e = galloc(c, *G, &G->t[l], n)))
      return fail(e);
  }
  if ((e = refresh(c, *G))) return fail(e);
  return check_cuda(c, cudaStreamSynchronize(c->stream), "multigrid set-up");
}

int dgx_mg_vcycle(dgx_ctx *c, const double *r, double *z) {
  if (!c) return DGX_ERR_ARG;
  if (!r || !z || r == z) return set_error(c, DGX_ERR_ARG, "r, z must be distinct non-null arrays");
  return mg_vcycle(c, r, z);
}

int dgx_mg_levels(dgx_ctx *c, int *levels, double *lambda_max, int capacity) {
  if (!c) return DGX_ERR_ARG;
  if (!c->mg) return set_error(c, DGX_ERR_STATE, "no multigrid hierarchy (call dgx_mg_setup)");
  Multigrid &G = *c->mg;
  if (G.coef_version != c->coef_version)
    if (int e = refresh(c, G)) return e;
  if (levels) *levels = (int)G.lv.size();
  for (int l = 0; l < (int)G.lv.size() && l < capacity; ++l)
    if (lambda_max) lambda_max[l] = G.lmax[l];
  return DGX_OK;
}

}  // extern "C"
