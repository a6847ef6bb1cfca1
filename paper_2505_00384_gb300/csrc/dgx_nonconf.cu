// Non-conforming meshes (arXiv:2505.00384, Sec. 3: neighbouring cells of
// different resolution horizontally and vertically): the terms of the 2:1
// hanging faces between the children block and the base cells.
//
// The per-patch kernels skip every face that touches the other patch (their
// neighbour lookup returns -2 there); the kernels here add those faces' terms
// on both sides.  A base cell's hanging face is the union of four children's
// faces; each is integrated with the child's Q x Q Gauss rule, the base
// cell's trace evaluated at the child's points (coarse reference coordinates
// (sig + g_i) / 2 along each tangential direction) and the child's face
// geometry on both sides (a child's map is its parent's map restricted, so
// the two agree; using one of them makes the two sides' fluxes cancel
// exactly).  The work list holds every cell with a hanging face; one CTA per
// cell sums all of that cell's hanging-face terms and adds them to its own
// entries only, so there are no write conflicts.
//   k_hang_grad   V += A^-1 B_h p  (or V += B_h p): central p_hat, the fast
//                 inverse of the cell's density-weighted mass (Sec. 3.3)
//   k_hang_div    y -= C_h V: central flux of kappa V, kappa = gamma p_k / (gamma - 1)
//   k_hang_expl   explicit tendencies: local Lax-Friedrichs flux of rho, rho u, rho k
// The interface is O(surface) of the children block, a few percent of the
// cells: these kernels favour simplicity (direct evaluation at each point)
// over the sum factorisation of the volume kernels.
#include <algorithm>
#include <vector>

#include "dgx_common.cuh"
#include "dgx_sweep.cuh"

namespace dgx {

// One cell with hanging faces: its faces f (2k+s) and across each either the
// four children (base cell; sig1 + 2 sig2 order) or the base cell and this
// child's position (nb[i][0], nb[i][1] = sig1 + 2 sig2).
struct HangCell {
  int cell, nface;
  int f[6];
  int nb[6][4];
};

namespace {

// 1D tables of the hanging-face kernels: I[q][a] = l_a(g_q), then
// Lsig[q][a] = l_a((sig + g_q) / 2) for sig = 0, 1, then the Gauss weights.
__host__ __device__ constexpr int hang_tab_size(int N, int Q) { return 3 * Q * N + Q; }

template <typename T, int N, int Q>
struct HangTabs {
  const T *I, *L0, *L1, *w;
  __device__ HangTabs(const T *t) : I(t), L0(t + Q * N), L1(t + 2 * Q * N), w(t + 3 * Q * N) {}
  // 1D basis of the trace side at point index i of a face: own-rule
  // interpolation, or the base cell's at child position sig
  __device__ const T *row(bool coarse, int sig, int i) const { return (coarse ? (sig ? L1 : L0) : I) + i * N; }
};

// value at a face point of a face-nodal field F (N x N, index t1 + N t2)
template <typename T, int N>
__device__ __forceinline__ T trace(const T *F, const T *r1, const T *r2) {
  T v = T(0);
#pragma unroll
  for (int b = 0; b < N; ++b) {
    T a0 = T(0);
#pragma unroll
    for (int a = 0; a < N; ++a) a0 += r1[a] * F[a + N * b];
    v += r2[b] * a0;
  }
  return v;
}

// Geometry of hanging point pt of face f of cell `cell`: outward normal times
// area element times the Gauss weights, from the child's face.
template <typename T, int N, int Q, bool CURVED>
__device__ __forceinline__ void hang_normal(const OpP<T> &P1, long long ncell0, int cell, int f, bool base,
                                            const int *nb, int pt, const T *wq, T nA[3]) {
  const int sig = pt / (Q * Q), t = pt % (Q * Q), i = t % Q, j = t / Q;
  const long long child = (base ? nb[sig] : cell) - ncell0;
  const CellPos cp = cell_pos(P1, child);
  const T *colp = CURVED ? P1.col + (long long)(cp.cx + P1.nx * cp.cy) * col_size(N, Q) : nullptr;
  face_normal<T, N, Q, CURVED>(P1, colp, T(cp.cz) * P1.dz, base ? (f ^ 1) : f, i, j, nA);
  const T w = (base ? -wq[i] : wq[i]) * wq[j];
  nA[0] *= w;
  nA[1] *= w;
  nA[2] *= w;
}

// Load nf face-nodal fields of the hanging face (own side into own[fld][N2],
// the other side into oth[sig][fld][N2]).
template <typename T, int N>
__device__ __forceinline__ void load_faces(int nf, const T *const *fields, long long Ntot, int cell, int f, bool base,
                                           const int *nb, T *own, T *oth) {
  constexpr int N2 = N * N, N3 = N * N * N;
  const int k = f >> 1, s = f & 1, nside = base ? 4 : 1;
  for (int idx = threadIdx.x; idx < nf * N2 * (1 + nside); idx += blockDim.x) {
    const int t = idx % N2, t1 = t % N, t2 = t / N, fld = (idx / N2) % nf, which = idx / (N2 * nf);
    if (which == 0) {
      own[fld * N2 + t] = fields[fld][(long long)cell * N3 + face_node<N>(k, s ? N - 1 : 0, t1, t2)];
    } else {
      const long long o = (long long)nb[which - 1] * N3 + face_node<N>(k, s ? 0 : N - 1, t1, t2);
      oth[((which - 1) * nf + fld) * N2 + t] = fields[fld][o];
    }
  }
}

template <typename T, int N, bool CURVED, bool INV>
__global__ void __launch_bounds__(128) k_hang_grad(const OpP<T> P0, const OpP<T> P1, const HangCell *__restrict__ hc,
                                                   const T *__restrict__ htab, const T *__restrict__ p,
                                                   const T *__restrict__ rho, T *__restrict__ V, long long Ntot,
                                                   long long ncell0) {
  constexpr int Q = 2 * N - 1, N2 = N * N, N3 = N * N * N, Q2 = Q * Q;
  constexpr int TAB = (tab_size(N, Q) + 1) & ~1, HT = (hang_tab_size(N, Q) + 1) & ~1;
  __shared__ __align__(16) T tab[TAB];
  __shared__ __align__(16) T ht[HT];
  __shared__ T own[N2], oth[4 * N2], coef[4 * Q2 * 3], g[3 * N3], a[3 * N3], b[3 * N3], s_rho[N3], s_rq[N3];
  __shared__ HangCell H;
  if (threadIdx.x == 0) H = hc[blockIdx.x];
  for (int i = threadIdx.x; i < hang_tab_size(N, Q); i += blockDim.x) ht[i] = htab[i];
  for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) g[i] = T(0);
  __syncthreads();
  const HangTabs<T, N, Q> L(ht);
  const bool base = H.cell < ncell0;
  const OpP<T> &P = base ? P0 : P1;
  const T *fields[1] = {p};
  for (int hf = 0; hf < H.nface; ++hf) {
    const int f = H.f[hf], k = f >> 1, s = f & 1;
    const int *nb = H.nb[hf];
    load_faces<T, N>(1, fields, Ntot, H.cell, f, base, nb, own, oth);
    __syncthreads();
    const int np = base ? 4 * Q2 : Q2;
    for (int pt = threadIdx.x; pt < np; pt += blockDim.x) {
      const int sig = base ? pt / Q2 : nb[1], t = pt % Q2, i = t % Q, j = t / Q;
      const T pm = trace<T, N>(own, L.row(base, sig & 1, i), L.row(base, sig >> 1, j));
      const T pp = trace<T, N>(oth + (base ? sig : 0) * N2, L.row(!base, sig & 1, i), L.row(!base, sig >> 1, j));
      T nA[3];
      hang_normal<T, N, Q, CURVED>(P1, ncell0, H.cell, f, base, nb, pt, L.w, nA);
      const T ph = P.alpha * T(0.5) * (pm + pp);
      coef[3 * pt] = ph * nA[0];
      coef[3 * pt + 1] = ph * nA[1];
      coef[3 * pt + 2] = ph * nA[2];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 3 * N2; idx += blockDim.x) {
      const int d = idx / N2, t = idx % N2, t1 = t % N, t2 = t / N;
      T acc = T(0);
      for (int pt = 0; pt < np; ++pt) {
        const int sig = base ? pt / Q2 : nb[1], q = pt % Q2;
        acc += coef[3 * pt + d] * L.row(base, sig & 1, q % Q)[t1] * L.row(base, sig >> 1, q / Q)[t2];
      }
      g[d * N3 + face_node<N>(k, s ? N - 1 : 0, t1, t2)] += acc;
    }
    __syncthreads();
  }
  const long long o = (long long)H.cell * N3;
  if (INV) {
    const CellPos cp = cell_pos(P, base ? H.cell : H.cell - ncell0);
    const T *colp = CURVED ? P.col + (long long)(cp.cx + P.nx * cp.cy) * col_size(N, Q) : nullptr;
    load_tables<T, N, Q>(P.tab, tab);
    for (int i = threadIdx.x; i < N3; i += blockDim.x) s_rho[i] = rho[o + i];
    for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) a[i] = g[i];
    __syncthreads();
    rho_fast<T, N, Q>(tab, s_rho, b, b + N3, s_rq);
    fast_inverse<T, N, Q, CURVED>(P, tab, colp, s_rq, 3, a, b);
    for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) V[(i / N3) * Ntot + o + i % N3] += a[i];
  } else {
    for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) V[(i / N3) * Ntot + o + i % N3] += g[i];
  }
}

template <typename T, int N, bool CURVED>
__global__ void __launch_bounds__(128) k_hang_div(const OpP<T> P0, const OpP<T> P1, const HangCell *__restrict__ hc,
                                                  const T *__restrict__ htab, const T *__restrict__ V,
                                                  const T *__restrict__ pk, T *__restrict__ y, long long Ntot,
                                                  long long ncell0) {
  constexpr int Q = 2 * N - 1, N2 = N * N, N3 = N * N * N, Q2 = Q * Q;
  constexpr int HT = (hang_tab_size(N, Q) + 1) & ~1;
  __shared__ __align__(16) T ht[HT];
  __shared__ T own[4 * N2], oth[4 * 4 * N2], coef[4 * Q2], g[N3];
  __shared__ HangCell H;
  if (threadIdx.x == 0) H = hc[blockIdx.x];
  for (int i = threadIdx.x; i < hang_tab_size(N, Q); i += blockDim.x) ht[i] = htab[i];
  for (int i = threadIdx.x; i < N3; i += blockDim.x) g[i] = T(0);
  __syncthreads();
  const HangTabs<T, N, Q> L(ht);
  const bool base = H.cell < ncell0;
  const OpP<T> &P = base ? P0 : P1;
  const T *fields[4] = {pk, V, V + Ntot, V + 2 * Ntot};
  for (int hf = 0; hf < H.nface; ++hf) {
    const int f = H.f[hf], k = f >> 1, s = f & 1;
    const int *nb = H.nb[hf];
    load_faces<T, N>(4, fields, Ntot, H.cell, f, base, nb, own, oth);
    __syncthreads();
    const int np = base ? 4 * Q2 : Q2;
    for (int pt = threadIdx.x; pt < np; pt += blockDim.x) {
      const int sig = base ? pt / Q2 : nb[1], t = pt % Q2, i = t % Q, j = t / Q;
      const T *r1 = L.row(base, sig & 1, i), *r2 = L.row(base, sig >> 1, j);
      const T *o1 = L.row(!base, sig & 1, i), *o2 = L.row(!base, sig >> 1, j);
      const T *F = oth + (base ? sig : 0) * 4 * N2;
      T nA[3];
      hang_normal<T, N, Q, CURVED>(P1, ncell0, H.cell, f, base, nb, pt, L.w, nA);
      const T km = P.gfac * trace<T, N>(own, r1, r2), kp = P.gfac * trace<T, N>(F, o1, o2);
      const T vm = trace<T, N>(own + N2, r1, r2) * nA[0] + trace<T, N>(own + 2 * N2, r1, r2) * nA[1] +
                   trace<T, N>(own + 3 * N2, r1, r2) * nA[2];
      const T vp = trace<T, N>(F + N2, o1, o2) * nA[0] + trace<T, N>(F + 2 * N2, o1, o2) * nA[1] +
                   trace<T, N>(F + 3 * N2, o1, o2) * nA[2];
      coef[pt] = P.alpha * T(0.5) * (km * vm + kp * vp);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < N2; t += blockDim.x) {
      const int t1 = t % N, t2 = t / N;
      T acc = T(0);
      for (int pt = 0; pt < np; ++pt) {
        const int sig = base ? pt / Q2 : nb[1], q = pt % Q2;
        acc += coef[pt] * L.row(base, sig & 1, q % Q)[t1] * L.row(base, sig >> 1, q / Q)[t2];
      }
      g[face_node<N>(k, s ? N - 1 : 0, t1, t2)] += acc;
    }
    __syncthreads();
  }
  const long long o = (long long)H.cell * N3;
  for (int i = threadIdx.x; i < N3; i += blockDim.x) y[o + i] -= g[i];
}

template <int N, bool CURVED>
__global__ void __launch_bounds__(128) k_hang_expl(const OpP<double> P0, const OpP<double> P1,
                                                   const HangCell *__restrict__ hc, const double *__restrict__ htab,
                                                   const double *__restrict__ rho, const double *__restrict__ u,
                                                   double *__restrict__ Er, double *__restrict__ Em,
                                                   double *__restrict__ Ee, long long Ntot, long long ncell0) {
  using T = double;
  constexpr int Q = 2 * N - 1, N2 = N * N, N3 = N * N * N, Q2 = Q * Q;
  constexpr int HT = (hang_tab_size(N, Q) + 1) & ~1;
  __shared__ __align__(16) T ht[HT];
  __shared__ T own[4 * N2], oth[4 * 4 * N2], coef[5 * 4 * Q2], g[5 * N3];
  __shared__ HangCell H;
  if (threadIdx.x == 0) H = hc[blockIdx.x];
  for (int i = threadIdx.x; i < hang_tab_size(N, Q); i += blockDim.x) ht[i] = htab[i];
  for (int i = threadIdx.x; i < 5 * N3; i += blockDim.x) g[i] = T(0);
  __syncthreads();
  const HangTabs<T, N, Q> L(ht);
  const bool base = H.cell < ncell0;
  const T *fields[4] = {rho, u, u + Ntot, u + 2 * Ntot};
  for (int hf = 0; hf < H.nface; ++hf) {
    const int f = H.f[hf], k = f >> 1, s = f & 1;
    const int *nb = H.nb[hf];
    load_faces<T, N>(4, fields, Ntot, H.cell, f, base, nb, own, oth);
    __syncthreads();
    const int np = base ? 4 * Q2 : Q2;
    for (int pt = threadIdx.x; pt < np; pt += blockDim.x) {
      const int sig = base ? pt / Q2 : nb[1], t = pt % Q2, i = t % Q, j = t / Q;
      const T *r1 = L.row(base, sig & 1, i), *r2 = L.row(base, sig >> 1, j);
      const T *o1 = L.row(!base, sig & 1, i), *o2 = L.row(!base, sig >> 1, j);
      const T *F = oth + (base ? sig : 0) * 4 * N2;
      T nA[3];
      hang_normal<T, N, Q, CURVED>(P1, ncell0, H.cell, f, base, nb, pt, L.w, nA);  // includes the weights
      const T rm = trace<T, N>(own, r1, r2), rp = trace<T, N>(F, o1, o2);
      const T vm0 = trace<T, N>(own + N2, r1, r2), vm1 = trace<T, N>(own + 2 * N2, r1, r2),
              vm2 = trace<T, N>(own + 3 * N2, r1, r2);
      const T vp0 = trace<T, N>(F + N2, o1, o2), vp1 = trace<T, N>(F + 2 * N2, o1, o2),
              vp2 = trace<T, N>(F + 3 * N2, o1, o2);
      const T unm = vm0 * nA[0] + vm1 * nA[1] + vm2 * nA[2];
      const T unp = vp0 * nA[0] + vp1 * nA[1] + vp2 * nA[2];
      const T lam = fmax(fabs(unm), fabs(unp));  // lambda |nA| (weights included)
      const T km = T(0.5) * (vm0 * vm0 + vm1 * vm1 + vm2 * vm2), kp = T(0.5) * (vp0 * vp0 + vp1 * vp1 + vp2 * vp2);
      const T qm[5] = {rm, rm * vm0, rm * vm1, rm * vm2, rm * km};
      const T qp[5] = {rp, rp * vp0, rp * vp1, rp * vp2, rp * kp};
#pragma unroll
      for (int c = 0; c < 5; ++c) coef[c * 4 * Q2 + pt] = -(T(0.5) * (qm[c] * unm + qp[c] * unp) + T(0.5) * lam * (qm[c] - qp[c]));
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 5 * N2; idx += blockDim.x) {
      const int c = idx / N2, t = idx % N2, t1 = t % N, t2 = t / N;
      T acc = T(0);
      for (int pt = 0; pt < np; ++pt) {
        const int sig = base ? pt / Q2 : nb[1], q = pt % Q2;
        acc += coef[c * 4 * Q2 + pt] * L.row(base, sig & 1, q % Q)[t1] * L.row(base, sig >> 1, q / Q)[t2];
      }
      g[c * N3 + face_node<N>(k, s ? N - 1 : 0, t1, t2)] += acc;
    }
    __syncthreads();
  }
  const long long o = (long long)H.cell * N3;
  for (int i = threadIdx.x; i < N3; i += blockDim.x) {
    Er[o + i] += g[i];
    Em[o + i] += g[N3 + i];
    Em[Ntot + o + i] += g[2 * N3 + i];
    Em[2 * Ntot + o + i] += g[3 * N3 + i];
    Ee[o + i] += g[4 * N3 + i];
  }
}

template <typename T>
__global__ void k_fill_dead(T *x, const T *src, int nf, T v, long long Ntot, int nx, int ny, int n3, int4 lo, int4 ext,
                            long long nd) {
  const long long total = nd * n3 * nf;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int node = (int)(i % n3);
    const long long dc = (i / n3) % nd;
    const int fld = (int)(i / (n3 * nd));
    const int bx = (int)(dc % ext.x), by = (int)((dc / ext.x) % ext.y), bz = (int)(dc / ((long long)ext.x * ext.y));
    const long long cell = (lo.x + bx) + (long long)nx * ((lo.y + by) + (long long)ny * (lo.z + bz));
    const long long i0 = fld * Ntot + cell * n3 + node;
    x[i0] = src ? src[i0] : v;
  }
}

template <typename T>
const T *hang_tab(const dgx_ctx *c) {
  if constexpr (sizeof(T) == 8) return reinterpret_cast<const T *>(c->hang64);
  else return reinterpret_cast<const T *>(c->hang32);
}

template <typename T, int N, bool CURVED>
int hang_grad_impl(dgx_ctx *c, const T *p, const T *rho, T *V, cudaStream_t s, bool inv, double alpha) {
  OpP<T> P0 = make_params<T>(c, 0), P1 = make_params<T>(c, 1);
  if (alpha >= 0.0) P0.alpha = P1.alpha = (T)alpha;
  const HangCell *hc = reinterpret_cast<const HangCell *>(c->hcells);
  count_launch();
  if (inv)
    k_hang_grad<T, N, CURVED, true><<<c->nhcell, 128, 0, s>>>(P0, P1, hc, hang_tab<T>(c), p, rho, V, c->N, c->ncell0);
  else
    k_hang_grad<T, N, CURVED, false><<<c->nhcell, 128, 0, s>>>(P0, P1, hc, hang_tab<T>(c), p, rho, V, c->N, c->ncell0);
  return check_cuda(c, cudaGetLastError(), "k_hang_grad launch");
}

template <typename T, int N, bool CURVED>
int hang_div_impl(dgx_ctx *c, const T *V, const T *pk, T *y, cudaStream_t s, double alpha) {
  OpP<T> P0 = make_params<T>(c, 0), P1 = make_params<T>(c, 1);
  if (alpha >= 0.0) P0.alpha = P1.alpha = (T)alpha;
  count_launch();
  k_hang_div<T, N, CURVED><<<c->nhcell, 128, 0, s>>>(P0, P1, reinterpret_cast<const HangCell *>(c->hcells),
                                                     hang_tab<T>(c), V, pk, y, c->N, c->ncell0);
  return check_cuda(c, cudaGetLastError(), "k_hang_div launch");
}

template <int N, bool CURVED>
int hang_expl_impl(dgx_ctx *c, const double *rho, const double *u, double *Er, double *Em, double *Ee, cudaStream_t s) {
  count_launch();
  k_hang_expl<N, CURVED><<<c->nhcell, 128, 0, s>>>(make_params<double>(c, 0), make_params<double>(c, 1),
                                                   reinterpret_cast<const HangCell *>(c->hcells), c->hang64, rho, u,
                                                   Er, Em, Ee, c->N, c->ncell0);
  return check_cuda(c, cudaGetLastError(), "k_hang_expl launch");
}

#define DGX_NC_DISPATCH(CALL)                                                      \
  switch (c->n) {                                                                  \
    case 2: return c->curved ? CALL(2, true) : CALL(2, false);                     \
    case 3: return c->curved ? CALL(3, true) : CALL(3, false);                     \
    case 4: return c->curved ? CALL(4, true) : CALL(4, false);                     \
    case 5: return c->curved ? CALL(5, true) : CALL(5, false);                     \
    case 6: return c->curved ? CALL(6, true) : CALL(6, false);                     \
    default: return set_error(c, DGX_ERR_ARG, "non-conforming meshes: degree %d above 5", c->n - 1); \
  }

}  // namespace

template <typename T>
int launch_hang_grad(dgx_ctx *c, const T *p, const T *rho, T *V, cudaStream_t s, bool inv, double alpha) {
  if (c->nhcell == 0) return 0;
#define CALL_HG(NN, CC) hang_grad_impl<T, NN, CC>(c, p, rho, V, s, inv, alpha)
  DGX_NC_DISPATCH(CALL_HG)
#undef CALL_HG
}
template int launch_hang_grad<double>(dgx_ctx *, const double *, const double *, double *, cudaStream_t, bool, double);
template int launch_hang_grad<float>(dgx_ctx *, const float *, const float *, float *, cudaStream_t, bool, double);

template <typename T>
int launch_hang_div(dgx_ctx *c, const T *V, const T *pk, T *y, cudaStream_t s, double alpha) {
  if (c->nhcell == 0) return 0;
#define CALL_HD(NN, CC) hang_div_impl<T, NN, CC>(c, V, pk, y, s, alpha)
  DGX_NC_DISPATCH(CALL_HD)
#undef CALL_HD
}
template int launch_hang_div<double>(dgx_ctx *, const double *, const double *, double *, cudaStream_t, double);
template int launch_hang_div<float>(dgx_ctx *, const float *, const float *, float *, cudaStream_t, double);

int launch_hang_explicit(dgx_ctx *c, const double *rho, const double *u, double *Er, double *Em, double *Ee,
                         cudaStream_t s) {
  if (c->nhcell == 0) return 0;
#define CALL_HE(NN, CC) hang_expl_impl<NN, CC>(c, rho, u, Er, Em, Ee, s)
  DGX_NC_DISPATCH(CALL_HE)
#undef CALL_HE
}

template <typename T>
int fill_dead(dgx_ctx *c, T *x, int nf, double v, cudaStream_t s, const T *src) {
  if (!c->nc) return 0;
  const int *rf = c->mesh.refine;
  const int4 lo = make_int4(rf[0], rf[2], rf[4], 0), ext = make_int4(rf[1] - rf[0], rf[3] - rf[2], rf[5] - rf[4], 0);
  const long long nd = (long long)ext.x * ext.y * ext.z, n3 = (long long)c->n * c->n * c->n;
  const long long blocks = std::min<long long>((nd * n3 * nf + 255) / 256, 4 * 152);
  count_launch();
  k_fill_dead<T><<<(unsigned)std::max<long long>(blocks, 1), 256, 0, s>>>(x, src, nf, (T)v, c->N, c->mesh.nx,
                                                                        c->mesh.ny, (int)n3, lo, ext, nd);
  return check_cuda(c, cudaGetLastError(), "k_fill_dead launch");
}
template int fill_dead<double>(dgx_ctx *, double *, int, double, cudaStream_t, const double *);
template int fill_dead<float>(dgx_ctx *, float *, int, double, cudaStream_t, const float *);

// Hanging-face work list: every live base cell whose face neighbour lies in
// the box, and every child on the block's surface whose face leaves the block
// into the base mesh (not the domain boundary); their 1D tables.
int nonconf_setup(dgx_ctx *c) {
  if (int e = upload_const_tables(c)) return e;  // this translation unit's copy (fast inverse)
  const dgx_mesh_desc &m = c->mesh;
  const int *rf = m.refine;
  const int ext[3] = {m.nx, m.ny, m.nz}, *fd = c->fine;
  auto in_box = [&](const int x[3]) {
    for (int d = 0; d < 3; ++d)
      if (x[d] < rf[2 * d] || x[d] >= rf[2 * d + 1]) return false;
    return true;
  };
  auto base_index = [&](const int x[3]) { return x[0] + m.nx * (x[1] + m.ny * x[2]); };
  auto fine_index = [&](const int x[3]) { return (int)c->ncell0 + x[0] + fd[0] * (x[1] + fd[1] * x[2]); };
  std::vector<HangCell> list;
  for (int z = 0; z < m.nz; ++z)
    for (int y = 0; y < m.ny; ++y)
      for (int x = 0; x < m.nx; ++x) {
        const int cc[3] = {x, y, z};
        if (in_box(cc)) continue;
        HangCell h{};
        h.cell = base_index(cc);
        for (int f = 0; f < 6; ++f) {
          const int k = f >> 1, s = f & 1, t1 = k == 0 ? 1 : 0, t2 = k == 2 ? 1 : 2;
          int nc[3] = {x, y, z};
          nc[k] += s ? 1 : -1;
          if (nc[k] < 0 || nc[k] >= ext[k]) continue;  // domain boundary (the box stays clear of periodic faces)
          if (!in_box(nc)) continue;
          for (int sg = 0; sg < 4; ++sg) {
            int fc[3];
            fc[k] = 2 * (nc[k] - rf[2 * k]) + (s ? 0 : 1);
            fc[t1] = 2 * (cc[t1] - rf[2 * t1]) + (sg & 1);
            fc[t2] = 2 * (cc[t2] - rf[2 * t2]) + (sg >> 1);
            h.nb[h.nface][sg] = fine_index(fc);
          }
          h.f[h.nface++] = f;
        }
        if (h.nface) list.push_back(h);
      }
  for (int z = 0; z < fd[2]; ++z)
    for (int y = 0; y < fd[1]; ++y)
      for (int x = 0; x < fd[0]; ++x) {
        const int fc[3] = {x, y, z};
        HangCell h{};
        h.cell = fine_index(fc);
        for (int f = 0; f < 6; ++f) {
          const int k = f >> 1, s = f & 1, t1 = k == 0 ? 1 : 0, t2 = k == 2 ? 1 : 2;
          const int nk = fc[k] + (s ? 1 : -1);
          if (nk >= 0 && nk < fd[k]) continue;  // inside the block
          int bc[3] = {rf[0] + x / 2, rf[2] + y / 2, rf[4] + z / 2};
          bc[k] += s ? 1 : -1;
          if (bc[k] < 0 || bc[k] >= ext[k]) continue;  // domain boundary
          h.nb[h.nface][0] = base_index(bc);
          h.nb[h.nface][1] = (fc[t1] & 1) + 2 * (fc[t2] & 1);
          h.f[h.nface++] = f;
        }
        if (h.nface) list.push_back(h);
      }
  c->nhcell = (int)list.size();
  // tables: I, L0, L1 and the Gauss weights
  const int N = c->n, Q = c->q;
  std::vector<double> x, w, g, gw;
  rule_gll(N, x, w);
  rule_gauss(Q, g, gw);
  std::vector<double> t((size_t)hang_tab_size(N, Q));
  for (int q = 0; q < Q; ++q)
    for (int sg = -1; sg < 2; ++sg) {
      const double at = sg < 0 ? g[q] : 0.5 * (sg + g[q]);
      for (int a = 0; a < N; ++a) {
        double l = 1.0;
        for (int b = 0; b < N; ++b)
          if (b != a) l *= (at - x[b]) / (x[a] - x[b]);
        t[(size_t)(sg + 1) * Q * N + q * N + a] = l;
      }
    }
  for (int q = 0; q < Q; ++q) t[3 * Q * N + q] = gw[q];
  std::vector<float> t32(t.begin(), t.end());
  void *p64 = nullptr, *p32 = nullptr, *ph = nullptr;
  if (int e = check_cuda(c, cudaMalloc(&p64, t.size() * sizeof(double)), "cudaMalloc")) return e;
  c->owned.push_back(p64);
  if (int e = check_cuda(c, cudaMalloc(&p32, t32.size() * sizeof(float)), "cudaMalloc")) return e;
  c->owned.push_back(p32);
  if (int e = check_cuda(c, cudaMalloc(&ph, std::max<size_t>(1, list.size()) * sizeof(HangCell)), "cudaMalloc"))
    return e;
  c->owned.push_back(ph);
  cudaMemcpy(p64, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(p32, t32.data(), t32.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (!list.empty()) cudaMemcpy(ph, list.data(), list.size() * sizeof(HangCell), cudaMemcpyHostToDevice);
  c->hang64 = reinterpret_cast<double *>(p64);
  c->hang32 = reinterpret_cast<float *>(p32);
  c->hcells = ph;
  return check_cuda(c, cudaGetLastError(), "non-conforming set-up");
}

}  // namespace dgx
