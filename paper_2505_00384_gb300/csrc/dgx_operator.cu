// Matrix-free pressure (Schur) operator of the IMEX-DG scheme, sm_103a.
//
// arXiv:2505.00384, Sec. 2: the fixed-point pressure equation
//   D P + C A^-1 (F - B P) = G,   i.e. S P = (D - C A^-1 B) P,
// with A the density-weighted velocity mass (Eq. for A^(l)), B the weak
// pressure gradient, C the weak divergence of the enthalpy flux and D the
// internal-energy mass.  Sec. 3.3: every integral uses Q = 2r+1 Gauss points
// per direction; A^-1 = S^-T J^-1 S^-1 with r+1 Gauss points.
//
// Kernels (one hexahedral cell per CTA, sum factorisation in shared memory):
//   k_grad  V = A^-1 B P   (volume weak gradient + central {p} face term +
//                           fast inverse of the density-weighted mass)
//   k_div   y = D P - C V  (volume weak divergence of kappa V + central face
//                           flux + internal-energy mass), kappa = gamma p_k/(gamma-1)
//   k_minv  out = A^-1 in  (the fast inverse alone)
//   k_diag  Helmholtz and internal-energy diagonals of Sec. 3.1
// Readings of the paper's open points (shared with the CPU oracle by
// definition, not by code): central fluxes (also across periodic faces);
// p_hat = p- on slip walls and 0 (the background) on far-field faces; zero
// normal flux of kappa V on slip walls, transmissive on far-field faces;
// Gal-Chen terrain-following map z = zeta + h(x,y) (1 - zeta/H).
#include <cmath>
#include <cstdio>
#include <mutex>
#include <set>
#include <utility>

#include "dgx_common.cuh"
#include "dgx_sweep.cuh"

namespace dgx {
namespace {

constexpr int cmax(int a, int b) { return a > b ? a : b; }

// ------------------------------------------------------------------ k_grad
template <int N, int Q, bool CURVED>
struct GradL {
  static constexpr int N2 = N * N, N3 = N * N * N, Q2 = Q * Q, Q3 = Q * Q * Q;
  static constexpr int NFV = CURVED ? 5 : 3;   // volume flux fields f_{jd}
  static constexpr int NFP = CURVED ? 10 : 6;  // (face, component) products
  static constexpr int TAB = (tab_size(N, Q) + 1) & ~1;
  static constexpr int oP = TAB, oRho = oP + N3, oRq = oRho + N3, oOut = oRq + N3;
  static constexpr int oW = oOut + 3 * N3;
  // R1, R2: interpolation temporaries and the fast-inverse ping buffer
  static constexpr int szR1 = cmax(N2 * Q, 3 * N3), szR2 = cmax(N * Q2, N3);
  static constexpr int oR1 = oW, oR2 = oR1 + szR1, oVol = oR2 + szR2;
  static constexpr int szVol = NFV * Q3, szZ = NFV * Q2 * N, szY = NFV * Q * N2, szX = NFV * N3;
  // Wy reuses Wv (dead after the z sweep), Wx reuses Wz (dead after the y sweep);
  // the face stage reuses everything from oVol on (after the combine barrier).
  static constexpr int oZ = oVol + szVol, oY = oVol, oX = oZ, oFace = oVol;
  static constexpr int szFace = 6 * N2 + 6 * N * Q + 6 * Q2 + NFP * Q2 + NFP * N * Q + NFP * N2;
  static_assert(szY <= szVol && szX <= szZ, "layout");
  static constexpr int total = cmax(oZ + szZ, oFace + szFace);
};

// FP64 at r <= 4: ask for <= 85 registers so that three 256-thread CTAs fit on an SM.
template <typename T, int N>
constexpr int min_ctas() { return (sizeof(T) == 8 && N <= 5) ? 3 : 1; }

// INV = true: V = A^-1 (B p); INV = false: the dual vector B p itself.
// One cell per CTA; `sm` is the CTA's dynamic shared memory (GradL layout).
template <typename T, int N, int Q, bool CURVED, bool INV>
__device__ __forceinline__ void grad_body(const OpP<T> &P, const long long cell, const T *__restrict__ p,
                                          const T *__restrict__ rho, T *__restrict__ V, long long Ntot, T *sm) {
  using L = GradL<N, Q, CURVED>;
  constexpr int N2 = L::N2, N3 = L::N3, Q2 = L::Q2, Q3 = L::Q3, NFV = L::NFV, NFP = L::NFP;
  T *tab = sm;
  T *s_p = sm + L::oP, *s_rho = sm + L::oRho, *s_rq = sm + L::oRq, *s_out = sm + L::oOut;
  T *R1 = sm + L::oR1, *R2 = sm + L::oR2, *Wv = sm + L::oVol, *Wz = sm + L::oZ, *Wy = sm + L::oY,
    *Wx = sm + L::oX, *Wf = sm + L::oFace;

  const CellPos cp = cell_pos(P, cell);
  __shared__ long long s_nb[6];  // the six face neighbours (-1: boundary, -2: skipped), read after the first barrier
  if (threadIdx.x < 6) s_nb[threadIdx.x] = neighbour(P, cp, threadIdx.x);
  const T *colp = CURVED ? P.col + (long long)(cp.cx + P.nx * cp.cy) * col_size(N, Q) : nullptr;
  const T zeta0 = T(cp.cz) * P.dz;

  load_tables<T, N, Q>(P.tab, tab);
  for (int i = threadIdx.x; i < N3; i += blockDim.x) {
    s_p[i] = p[cell * N3 + i];
    s_rho[i] = rho[cell * N3 + i];
  }
  __syncthreads();
  const T *I = tab + tab_off_I(N, Q), *IT = tab + tab_off_IT(N, Q), *DT = tab + tab_off_DT(N, Q);
  const T *wq = tab + tab_off_wq(N, Q), *gq = tab + tab_off_gq(N, Q);

  // p at the Q^3 Gauss points; rho at the fast-rule points
  sweep<T, N, 0, Q, N, N, N, N, M_I, M_I, M_I>(1, 0u, s_p, R1);
  __syncthreads();
  sweep<T, N, 1, Q, N, Q, N, N, M_I, M_I, M_I>(1, 0u, R1, R2);
  __syncthreads();
  sweep<T, N, 2, Q, N, Q, Q, N, M_I, M_I, M_I>(1, 0u, R2, Wv);
  __syncthreads();
  rho_fast<T, N, Q>(tab, s_rho, R1, R2, s_rq);

  // volume fluxes f_{jd} = -alpha w p adj(J)_{jd}  (weak gradient, Sec. 2)
  for (int idx = threadIdx.x; idx < Q3; idx += blockDim.x) {
    const int i = idx % Q, j = (idx / Q) % Q, k = idx / Q2;
    if (CURVED) {  // weighted metric products from the column table
      const int t = i + Q * j;
      const T a = -P.alpha * Wv[idx];
      const T aw = a * wq[k], af = aw * (T(1) - (zeta0 + P.dz * gq[k]) * P.invH);
      Wv[0 * Q3 + idx] = aw * colp[col_off_w(N, Q, 0) + t];  // j=0, d=0
      Wv[1 * Q3 + idx] = af * colp[col_off_w(N, Q, 3) + t];  // j=2, d=0
      Wv[2 * Q3 + idx] = aw * colp[col_off_w(N, Q, 1) + t];  // j=1, d=1
      Wv[3 * Q3 + idx] = af * colp[col_off_w(N, Q, 4) + t];  // j=2, d=1
      Wv[4 * Q3 + idx] = aw * colp[col_off_w(N, Q, 2) + t];  // j=2, d=2
    } else {
      const T c = -P.alpha * wq[i] * wq[j] * wq[k] * Wv[idx];
      Wv[0 * Q3 + idx] = c * P.dy * P.dz;
      Wv[1 * Q3 + idx] = c * P.dx * P.dz;
      Wv[2 * Q3 + idx] = c * P.dx * P.dy;
    }
  }
  __syncthreads();
  // test with grad: z, y, x sweeps; D^T in the field's reference direction j
  if (CURVED) {
    sweep<T, N, 2, N, Q, Q, Q, Q, M_IT, M_DT, M_DT>(NFV, (1u << 2) | (1u << 6) | (1u << 8), Wv, Wz);
    __syncthreads();
    sweep<T, N, 1, N, Q, Q, Q, N, M_IT, M_DT, M_DT>(NFV, (1u << 4), Wz, Wy);
    __syncthreads();
    sweep<T, N, 0, N, Q, Q, N, N, M_IT, M_DT, M_DT>(NFV, (1u << 0), Wy, Wx);
  } else {
    sweep<T, N, 2, N, Q, Q, Q, Q, M_IT, M_DT, M_DT>(NFV, (1u << 4), Wv, Wz);
    __syncthreads();
    sweep<T, N, 1, N, Q, Q, Q, N, M_IT, M_DT, M_DT>(NFV, (1u << 2), Wz, Wy);
    __syncthreads();
    sweep<T, N, 0, N, Q, Q, N, N, M_IT, M_DT, M_DT>(NFV, (1u << 0), Wy, Wx);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < 3 * N3; idx += blockDim.x) {
    const int d = idx / N3, node = idx % N3;
    T v;
    if (CURVED) v = d == 0 ? Wx[node] + Wx[N3 + node] : (d == 1 ? Wx[2 * N3 + node] + Wx[3 * N3 + node] : Wx[4 * N3 + node]);
    else v = Wx[d * N3 + node];
    s_out[idx] = v;
  }
  __syncthreads();

  // faces: alpha int p_hat psi n_d, p_hat = {p} inside, p- on slip walls, and
  // the far-field datum p_hat = 0 (background pressure) on far-field faces
  T *Fg = Wf, *F1 = Fg + 6 * N2, *F2 = F1 + 6 * N * Q, *Fp = F2 + 6 * Q2, *Fb1 = Fp + NFP * Q2, *Fb2 = Fb1 + NFP * N * Q;
  for (int idx = threadIdx.x; idx < 6 * N2; idx += blockDim.x) {
    const int f = idx / N2, t = idx % N2, t1 = t % N, t2 = t / N;
    const int k = f >> 1, s = f & 1;
    const T own = s_p[face_node<N>(k, s ? N - 1 : 0, t1, t2)];
    const long long nb = s_nb[f];
    T ph = own;
    if (nb >= 0) ph = T(0.5) * (own + p[nb * N3 + face_node<N>(k, s ? 0 : N - 1, t1, t2)]);
    else if (nb == -2 || (k < 2 && P.bc_lat == 1)) ph = T(0);
    Fg[idx] = ph;
  }
  __syncthreads();
  sweep<T, N, 0, Q, N, N, N, 1, M_I, M_I, M_I>(6, 0u, Fg, F1);
  __syncthreads();
  sweep<T, N, 1, Q, N, Q, N, 1, M_I, M_I, M_I>(6, 0u, F1, F2);
  __syncthreads();
  for (int idx = threadIdx.x; idx < NFP * Q2; idx += blockDim.x) {
    const int sl = idx / Q2, t = idx % Q2, i = t % Q, j = t / Q;
    int f, d;
    if (CURVED) {
      f = sl < 4 ? sl : (sl < 7 ? 4 : 5);
      d = sl < 4 ? (sl >> 1) : (sl < 7 ? sl - 4 : sl - 7);
    } else {
      f = sl;
      d = sl >> 1;
    }
    T nA[3];
    face_normal<T, N, Q, CURVED>(P, colp, zeta0, f, i, j, nA);
    Fp[idx] = P.alpha * wq[i] * wq[j] * nA[d] * F2[f * Q2 + t];
  }
  __syncthreads();
  sweep<T, N, 0, N, Q, Q, Q, 1, M_IT, M_IT, M_IT>(NFP, 0u, Fp, Fb1);
  __syncthreads();
  sweep<T, N, 1, N, Q, N, Q, 1, M_IT, M_IT, M_IT>(NFP, 0u, Fb1, Fb2);
  __syncthreads();
  for (int idx = threadIdx.x; idx < 3 * N3; idx += blockDim.x) {
    const int d = idx / N3, node = idx % N3;
    const int a = node % N, b = (node / N) % N, c = node / N2;
    T acc = s_out[idx];
#pragma unroll
    for (int sl = 0; sl < NFP; ++sl) {
      int f, dd;
      if (CURVED) {
        f = sl < 4 ? sl : (sl < 7 ? 4 : 5);
        dd = sl < 4 ? (sl >> 1) : (sl < 7 ? sl - 4 : sl - 7);
      } else {
        f = sl;
        dd = sl >> 1;
      }
      if (dd != d) continue;
      const int k = f >> 1, e = (f & 1) ? N - 1 : 0;
      if (k == 0 && a == e) acc += Fb2[sl * N2 + b + N * c];
      if (k == 1 && b == e) acc += Fb2[sl * N2 + a + N * c];
      if (k == 2 && c == e) acc += Fb2[sl * N2 + a + N * b];
    }
    s_out[idx] = acc;
  }
  __syncthreads();

  // V = A^-1 (B P), per component
  if (INV) fast_inverse<T, N, Q, CURVED>(P, tab, colp, s_rq, 3, s_out, R1);
  for (int idx = threadIdx.x; idx < 3 * N3; idx += blockDim.x) {
    const int d = idx / N3, node = idx % N3;
    V[d * Ntot + cell * N3 + node] = s_out[idx];
  }
}

template <typename T, int N, int Q, bool CURVED, bool INV = true>
__global__ void __launch_bounds__(256, min_ctas<T, N>()) k_grad(const OpP<T> P, const T *__restrict__ p,
                                                                const T *__restrict__ rho, T *__restrict__ V,
                                                                long long Ntot) {
  extern __shared__ __align__(16) unsigned char smraw[];
  grad_body<T, N, Q, CURVED, INV>(P, blockIdx.x, p, rho, V, Ntot, reinterpret_cast<T *>(smraw));
}

// Several meshes of the same degree in one launch: CTA b belongs to the member
// whose cell range [cell_off, cell_off + ncell) holds b; vectors are the
// members' DoF blocks concatenated (member m starts at dof_off).
template <typename T>
__device__ __forceinline__ int member_of(const EnsMember<T> *mem, int nmem, long long b) {
  int m = 0;
  while (m + 1 < nmem && mem[m + 1].cell_off <= b) ++m;
  return m;
}

template <typename T, int N, int Q, bool CURVED>
__global__ void __launch_bounds__(256, min_ctas<T, N>()) k_grad_multi(const EnsMember<T> *__restrict__ mem, int nmem,
                                                                      const T *__restrict__ p_all) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int m = member_of(mem, nmem, blockIdx.x);
  const EnsMember<T> M = mem[m];
  grad_body<T, N, Q, CURVED, true>(M.P, blockIdx.x - M.cell_off, p_all + M.dof_off, M.rho, M.V, M.N,
                                   reinterpret_cast<T *>(smraw));
}

// ------------------------------------------------------------------ k_div
template <int N, int Q, bool CURVED>
struct DivL {
  static constexpr int N2 = N * N, N3 = N * N * N, Q2 = Q * Q, Q3 = Q * Q * Q;
  static constexpr int NSL = CURVED ? 32 : 24;  // face trace slots
  static constexpr int TAB = (tab_size(N, Q) + 1) & ~1;
  static constexpr int oIn = TAB, oY = oIn + 5 * N3, oW = oY + N3;
  // R1 (x sweep) and R3 (values at Q^3) share oW: R1 is dead when R3 is written.
  // Wz reuses R2, Wy reuses R3; the face region starts at oW; Wx lies beyond all.
  static constexpr int oR1 = oW, oR3 = oW, oR2 = oW + 5 * Q3, oZ = oR2, oYs = oW;
  static constexpr int szFace = cmax(NSL * N2, NSL * Q2) + NSL * N * Q + 6 * (Q2 + N * Q + N2);
  static constexpr int oFace = oW;
  static constexpr int oX = oW + cmax(5 * Q3 + 5 * N * Q2, szFace);
  static_assert(5 * N2 * Q <= 5 * Q3 && 4 * Q2 * N <= 5 * N * Q2 && 4 * Q * N2 <= 5 * Q3, "layout");
  static constexpr int total = oX + 4 * N3;
};

template <typename T, int N, int Q, bool CURVED>
__device__ __forceinline__ void div_body(const OpP<T> &P, const long long cell, const T *__restrict__ V,
                                         const T *__restrict__ p, const T *__restrict__ pk, T *__restrict__ y,
                                         long long Ntot, T *sm, const T *__restrict__ kq = nullptr) {
  using L = DivL<N, Q, CURVED>;
  constexpr int N2 = L::N2, N3 = L::N3, Q2 = L::Q2, Q3 = L::Q3, NSL = L::NSL;
  T *tab = sm;
  T *s_in = sm + L::oIn, *s_y = sm + L::oY;
  T *R1 = sm + L::oR1, *R2 = sm + L::oR2, *R3 = sm + L::oR3, *Wz = sm + L::oZ, *Wy = sm + L::oYs, *Wx = sm + L::oX;
  // gather (Fg) and second interpolation (F2) share a region: Fg is dead when F2 is written
  T *Fg = sm + L::oFace, *F2 = Fg, *F1 = Fg + cmax(NSL * N2, NSL * Q2), *Ff = F1 + NSL * N * Q, *Fb1 = Ff + 6 * Q2,
    *Fb2 = Fb1 + 6 * N * Q;

  const CellPos cp = cell_pos(P, cell);
  __shared__ long long s_nb[6];  // the six face neighbours (-1: boundary, -2: skipped), read after the first barrier
  if (threadIdx.x < 6) s_nb[threadIdx.x] = neighbour(P, cp, threadIdx.x);
  const T *colp = CURVED ? P.col + (long long)(cp.cx + P.nx * cp.cy) * col_size(N, Q) : nullptr;
  const T zeta0 = T(cp.cz) * P.dz;

  load_tables<T, N, Q>(P.tab, tab);
  // with kq (alpha gamma/(gamma-1) p_k at the Q^3 points of this coefficient set)
  // the p_k interpolation is skipped: fields V0, V1, V2, p, p_k instead of V0, V1, V2, p_k, p
  const bool pre = kq != nullptr;
  const int ip = pre ? 3 : 4, ik = pre ? 4 : 3;
  for (int i = threadIdx.x; i < N3; i += blockDim.x) {
    s_in[0 * N3 + i] = V[0 * Ntot + cell * N3 + i];
    s_in[1 * N3 + i] = V[1 * Ntot + cell * N3 + i];
    s_in[2 * N3 + i] = V[2 * Ntot + cell * N3 + i];
    s_in[ik * N3 + i] = pk[cell * N3 + i];
    s_in[ip * N3 + i] = p[cell * N3 + i];
  }
  __syncthreads();
  const T *I = tab + tab_off_I(N, Q), *IT = tab + tab_off_IT(N, Q), *DT = tab + tab_off_DT(N, Q);
  const T *wq = tab + tab_off_wq(N, Q), *gq = tab + tab_off_gq(N, Q);

  const int nfi = pre ? 4 : 5;
  sweep<T, N, 0, Q, N, N, N, N, M_I, M_I, M_I>(nfi, 0u, s_in, R1);
  __syncthreads();
  sweep<T, N, 1, Q, N, Q, N, N, M_I, M_I, M_I>(nfi, 0u, R1, R2);
  __syncthreads();
  sweep<T, N, 2, Q, N, Q, Q, N, M_I, M_I, M_I>(nfi, 0u, R2, R3);
  __syncthreads();

  // -C V volume part: + alpha int kappa V . grad psi  -> F_j = alpha kappa w sum_d adj_{jd} V_d
  //  D P: w det J p / (gamma - 1)
  for (int idx = threadIdx.x; idx < Q3; idx += blockDim.x) {
    const int i = idx % Q, j = (idx / Q) % Q, k = idx / Q2;
    const T v0 = R3[idx], v1 = R3[Q3 + idx], v2 = R3[2 * Q3 + idx], pq = R3[ip * Q3 + idx];
    const T c0 = pre ? kq[cell * Q3 + idx] : P.alpha * P.gfac * R3[3 * Q3 + idx];
    if (CURVED) {  // weighted metric products from the column table
      const int t = i + Q * j;
      const T ck = c0 * wq[k], cf = ck * (T(1) - (zeta0 + P.dz * gq[k]) * P.invH);
      R3[idx] = ck * colp[col_off_w(N, Q, 0) + t] * v0;
      R3[Q3 + idx] = ck * colp[col_off_w(N, Q, 1) + t] * v1;
      R3[2 * Q3 + idx] = ck * colp[col_off_w(N, Q, 2) + t] * v2 +
                         cf * (colp[col_off_w(N, Q, 3) + t] * v0 + colp[col_off_w(N, Q, 4) + t] * v1);
      R3[3 * Q3 + idx] = (wq[k] * P.igm1) * colp[col_off_w(N, Q, 5) + t] * pq;
    } else {
      const T w = wq[i] * wq[j] * wq[k];
      const T c = c0 * w;
      R3[idx] = c * P.dy * P.dz * v0;
      R3[Q3 + idx] = c * P.dx * P.dz * v1;
      R3[2 * Q3 + idx] = c * P.dx * P.dy * v2;
      R3[3 * Q3 + idx] = w * P.dx * P.dy * P.dz * pq * P.igm1;
    }
  }
  __syncthreads();
  sweep<T, N, 2, N, Q, Q, Q, Q, M_IT, M_DT, M_DT>(4, (1u << 4), R3, Wz);
  __syncthreads();
  sweep<T, N, 1, N, Q, Q, Q, N, M_IT, M_DT, M_DT>(4, (1u << 2), Wz, Wy);
  __syncthreads();
  sweep<T, N, 0, N, Q, Q, N, N, M_IT, M_DT, M_DT>(4, (1u << 0), Wy, Wx);
  __syncthreads();

  // faces: - alpha int (kappa V)^ . n psi
  for (int idx = threadIdx.x; idx < N3; idx += blockDim.x)
    s_y[idx] = Wx[idx] + Wx[N3 + idx] + Wx[2 * N3 + idx] + Wx[3 * N3 + idx];
  for (int idx = threadIdx.x; idx < NSL * N2; idx += blockDim.x) {
    const int sl = idx / N2, t = idx % N2, t1 = t % N, t2 = t / N;
    int f, side, field;
    div_slot<CURVED>(sl, f, side, field);
    const int k = f >> 1, s = f & 1;
    const long long nb = s_nb[f];
    T v;
    if (side == 0 || nb < 0) {
      const int node = face_node<N>(k, s ? N - 1 : 0, t1, t2);
      v = field == 0 ? P.gfac * s_in[ik * N3 + node] : s_in[(field - 1) * N3 + node];
      // slip wall: no normal flux (all traces of this face set to zero)
      if (nb == -2 || (nb < 0 && (k == 2 || P.bc_lat == 0))) v = T(0);
    } else {
      const long long node = nb * N3 + face_node<N>(k, s ? 0 : N - 1, t1, t2);
      v = field == 0 ? P.gfac * pk[node] : V[(field - 1) * Ntot + node];
    }
    Fg[idx] = v;
  }
  __syncthreads();
  sweep<T, N, 0, Q, N, N, N, 1, M_I, M_I, M_I>(NSL, 0u, Fg, F1);
  __syncthreads();
  sweep<T, N, 1, Q, N, Q, N, 1, M_I, M_I, M_I>(NSL, 0u, F1, F2);
  __syncthreads();
  for (int idx = threadIdx.x; idx < 6 * Q2; idx += blockDim.x) {
    const int f = idx / Q2, t = idx % Q2, i = t % Q, j = t / Q;
    T nA[3];
    face_normal<T, N, Q, CURVED>(P, colp, zeta0, f, i, j, nA);
    const T *S = F2 + div_slot_base<CURVED>(f) * Q2 + t;
    T flux;
    if (f < 4 || !CURVED) {
      const int k = f >> 1;
      // slots: kappa-, V-, kappa+, V+
      flux = T(0.5) * nA[k] * (S[0] * S[Q2] + S[2 * Q2] * S[3 * Q2]);
    } else {
      const T vm = S[Q2] * nA[0] + S[2 * Q2] * nA[1] + S[3 * Q2] * nA[2];
      const T vp = S[5 * Q2] * nA[0] + S[6 * Q2] * nA[1] + S[7 * Q2] * nA[2];
      flux = T(0.5) * (S[0] * vm + S[4 * Q2] * vp);
    }
    Ff[idx] = -P.alpha * wq[i] * wq[j] * flux;
  }
  __syncthreads();
  sweep<T, N, 0, N, Q, Q, Q, 1, M_IT, M_IT, M_IT>(6, 0u, Ff, Fb1);
  __syncthreads();
  sweep<T, N, 1, N, Q, N, Q, 1, M_IT, M_IT, M_IT>(6, 0u, Fb1, Fb2);
  __syncthreads();
  for (int idx = threadIdx.x; idx < N3; idx += blockDim.x) {
    const int a = idx % N, b = (idx / N) % N, c = idx / N2;
    T acc = s_y[idx];
    if (a == 0) acc += Fb2[0 * N2 + b + N * c];
    if (a == N - 1) acc += Fb2[1 * N2 + b + N * c];
    if (b == 0) acc += Fb2[2 * N2 + a + N * c];
    if (b == N - 1) acc += Fb2[3 * N2 + a + N * c];
    if (c == 0) acc += Fb2[4 * N2 + a + N * b];
    if (c == N - 1) acc += Fb2[5 * N2 + a + N * b];
    y[cell * N3 + idx] = acc;
  }
}

template <typename T, int N, int Q, bool CURVED>
__global__ void __launch_bounds__(256, min_ctas<T, N>()) k_div(const OpP<T> P, const T *__restrict__ V,
                                                               const T *__restrict__ p, const T *__restrict__ pk,
                                                               T *__restrict__ y, long long Ntot,
                                                               const T *__restrict__ kq) {
  extern __shared__ __align__(16) unsigned char smraw[];
  div_body<T, N, Q, CURVED>(P, blockIdx.x, V, p, pk, y, Ntot, reinterpret_cast<T *>(smraw), kq);
}

// kq = alpha gamma/(gamma-1) p_k at the Q^3 Gauss points of every cell (the
// coefficient part of k_div's volume term, once per coefficient set)
template <typename T, int N, int Q>
__global__ void __launch_bounds__(128) k_kappa(const OpP<T> P, const T *__restrict__ pk, T *__restrict__ kq) {
  constexpr int N2 = N * N, N3 = N * N * N, Q3 = Q * Q * Q;
  constexpr int TAB = (tab_size(N, Q) + 1) & ~1;
  extern __shared__ __align__(16) unsigned char smraw[];
  T *sm = reinterpret_cast<T *>(smraw);
  T *tab = sm, *s_in = sm + TAB, *R1 = s_in + N3, *R2 = R1 + N2 * Q, *R3 = R2 + N * Q * Q;
  const long long cell = blockIdx.x;
  load_tables<T, N, Q>(P.tab, tab);
  for (int i = threadIdx.x; i < N3; i += blockDim.x) s_in[i] = pk[cell * N3 + i];
  __syncthreads();
  sweep<T, N, 0, Q, N, N, N, N, M_I, M_I, M_I>(1, 0u, s_in, R1);
  __syncthreads();
  sweep<T, N, 1, Q, N, Q, N, N, M_I, M_I, M_I>(1, 0u, R1, R2);
  __syncthreads();
  sweep<T, N, 2, Q, N, Q, Q, N, M_I, M_I, M_I>(1, 0u, R2, R3);
  __syncthreads();
  for (int idx = threadIdx.x; idx < Q3; idx += blockDim.x) kq[cell * Q3 + idx] = P.alpha * P.gfac * R3[idx];
}

template <typename T, int N, int Q, bool CURVED>
__global__ void __launch_bounds__(256, min_ctas<T, N>()) k_div_multi(const EnsMember<T> *__restrict__ mem, int nmem,
                                                                     const T *__restrict__ p_all, T *__restrict__ y_all) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int m = member_of(mem, nmem, blockIdx.x);
  const EnsMember<T> M = mem[m];
  div_body<T, N, Q, CURVED>(M.P, blockIdx.x - M.cell_off, M.V, p_all + M.dof_off, M.pk, y_all + M.dof_off, M.N,
                            reinterpret_cast<T *>(smraw));
}

// ------------------------------------------------------------------ k_minv
template <int N, int Q>
struct MinvL {
  static constexpr int N3 = N * N * N;
  static constexpr int TAB = (tab_size(N, Q) + 1) & ~1;
  static constexpr int oRho = TAB, oRq = oRho + N3, oA = oRq + N3, oB = oA + 3 * N3, total = oB + 3 * N3;
};

template <typename T, int N, int Q, bool CURVED>
__global__ void __launch_bounds__(128) k_minv(const OpP<T> P, const T *__restrict__ in, const T *__restrict__ rho,
                                              T *__restrict__ out, long long Ntot, int nf) {
  using L = MinvL<N, Q>;
  constexpr int N3 = L::N3;
  extern __shared__ __align__(16) unsigned char smraw[];
  T *sm = reinterpret_cast<T *>(smraw);
  T *tab = sm, *s_rho = sm + L::oRho, *s_rq = sm + L::oRq, *A = sm + L::oA, *B = sm + L::oB;
  const long long cell = blockIdx.x;
  const CellPos cp = cell_pos(P, cell);
  const T *colp = CURVED ? P.col + (long long)(cp.cx + P.nx * cp.cy) * col_size(N, Q) : nullptr;
  load_tables<T, N, Q>(P.tab, tab);
  for (int i = threadIdx.x; i < nf * N3; i += blockDim.x) {
    const int d = i / N3, node = i % N3;
    A[i] = in[d * Ntot + cell * N3 + node];
    if (d == 0) s_rho[node] = rho[cell * N3 + node];
  }
  __syncthreads();
  rho_fast<T, N, Q>(tab, s_rho, B, B + N3, s_rq);
  fast_inverse<T, N, Q, CURVED>(P, tab, colp, s_rq, nf, A, B);
  for (int i = threadIdx.x; i < nf * N3; i += blockDim.x) {
    const int d = i / N3, node = i % N3;
    out[d * Ntot + cell * N3 + node] = A[i];
  }
}

// ------------------------------------------------------------------ k_diag
template <int N, int Q, bool CURVED>
struct DiagL {
  static constexpr int N2 = N * N, N3 = N * N * N, Q2 = Q * Q, Q3 = Q * Q * Q;
  static constexpr int NF = CURVED ? 6 : 4;
  static constexpr int TAB = (tab_size(N, Q) + 1) & ~1;
  // R3 (rho, p_k at Q^3) first; R1, R2 after it; the coefficient fields F reuse
  // R1/R2 (dead after the z interpolation); Wy reuses F, Wx reuses Wz.
  static constexpr int oIn = TAB, oR3 = oIn + 2 * N3, oR1 = oR3 + 2 * Q3, oR2 = oR1 + 2 * N2 * Q;
  static constexpr int oF = oR1, oZ = oF + NF * Q3, oY = oF, oX = oZ;
  static_assert(NF * Q * N2 <= NF * Q3 && NF * N3 <= NF * Q2 * N, "layout");
  static constexpr int total = cmax(oR2 + 2 * N * Q2, oZ + NF * Q2 * N);
};

// Sec. 3.1: S~_ii = int psi_i^2/(gamma-1) + alpha^2 int h |grad psi_i|^2, h = gamma p_k/((gamma-1) rho)
// |grad psi|^2 det J = sum_{j,j'} d_j psi d_j' psi (adj adj^T)_{jj'} / det J.
template <typename T, int N, int Q, bool CURVED>
__global__ void __launch_bounds__(256) k_diag(const OpP<T> P, const T *__restrict__ rho, const T *__restrict__ pk,
                                              T *__restrict__ dh, T *__restrict__ die) {
  using L = DiagL<N, Q, CURVED>;
  constexpr int N3 = L::N3, Q2 = L::Q2, Q3 = L::Q3, NF = L::NF;
  extern __shared__ __align__(16) unsigned char smraw[];
  T *sm = reinterpret_cast<T *>(smraw);
  T *tab = sm, *s_in = sm + L::oIn, *R1 = sm + L::oR1, *R2 = sm + L::oR2, *R3 = sm + L::oR3, *F = sm + L::oF,
    *Wz = sm + L::oZ, *Wy = sm + L::oY, *Wx = sm + L::oX;
  const long long cell = blockIdx.x;
  const CellPos cp = cell_pos(P, cell);
  const T *colp = CURVED ? P.col + (long long)(cp.cx + P.nx * cp.cy) * col_size(N, Q) : nullptr;
  const T zeta0 = T(cp.cz) * P.dz;
  load_tables<T, N, Q>(P.tab, tab);
  for (int i = threadIdx.x; i < N3; i += blockDim.x) {
    s_in[i] = rho[cell * N3 + i];
    s_in[N3 + i] = pk[cell * N3 + i];
  }
  __syncthreads();
  const T *I = tab + tab_off_I(N, Q), *IIT = tab + tab_off_IIT(N, Q), *DDT = tab + tab_off_DDT(N, Q),
          *IDT = tab + tab_off_IDT(N, Q), *wq = tab + tab_off_wq(N, Q), *gq = tab + tab_off_gq(N, Q);
  sweep<T, N, 0, Q, N, N, N, N, M_I, M_I, M_I>(2, 0u, s_in, R1);
  __syncthreads();
  sweep<T, N, 1, Q, N, Q, N, N, M_I, M_I, M_I>(2, 0u, R1, R2);
  __syncthreads();
  sweep<T, N, 2, Q, N, Q, Q, N, M_I, M_I, M_I>(2, 0u, R2, R3);
  __syncthreads();
  const T a2 = P.alpha * P.alpha;
  for (int idx = threadIdx.x; idx < Q3; idx += blockDim.x) {
    const int i = idx % Q, j = (idx / Q) % Q, k = idx / Q2;
    const T w = wq[i] * wq[j] * wq[k];
    const T h = P.gfac * R3[Q3 + idx] / R3[idx];
    T z1 = 0, z2 = 0, z3 = P.dz;
    if (CURVED) {
      const T hh = colp[col_off_hq(N, Q) + i + Q * j];
      const T fac = T(1) - (zeta0 + P.dz * gq[k]) * P.invH;
      z1 = colp[col_off_h1q(N, Q) + i + Q * j] * fac;
      z2 = colp[col_off_h2q(N, Q) + i + Q * j] * fac;
      z3 = P.dz * (T(1) - hh * P.invH);
    }
    const T det = P.dx * P.dy * z3;
    const T A00 = P.dy * z3, A11 = P.dx * z3, A20 = -P.dy * z1, A21 = -P.dx * z2, A22 = P.dx * P.dy;
    const T c = a2 * h * w / det;
    F[0 * Q3 + idx] = w * det * P.igm1;
    F[1 * Q3 + idx] = c * A00 * A00;
    F[2 * Q3 + idx] = c * A11 * A11;
    F[3 * Q3 + idx] = c * (A20 * A20 + A21 * A21 + A22 * A22);
    if (CURVED) {
      F[4 * Q3 + idx] = T(2) * c * A00 * A20;
      F[5 * Q3 + idx] = T(2) * c * A11 * A21;
    }
  }
  __syncthreads();
  // matrices: 0 = (I o I)^T, 1 = (D o D)^T, 2 = (I o D)^T
  const unsigned selz = (1u << 6) | (CURVED ? ((2u << 8) | (2u << 10)) : 0u);
  const unsigned sely = (1u << 4) | (CURVED ? (2u << 10) : 0u);
  const unsigned selx = (1u << 2) | (CURVED ? (2u << 8) : 0u);
  sweep<T, N, 2, N, Q, Q, Q, Q, M_IIT, M_DDT, M_IDT>(NF, selz, F, Wz);
  __syncthreads();
  sweep<T, N, 1, N, Q, Q, Q, N, M_IIT, M_DDT, M_IDT>(NF, sely, Wz, Wy);
  __syncthreads();
  sweep<T, N, 0, N, Q, Q, N, N, M_IIT, M_DDT, M_IDT>(NF, selx, Wy, Wx);
  __syncthreads();
  for (int idx = threadIdx.x; idx < N3; idx += blockDim.x) {
    T s = 0;
#pragma unroll
    for (int f = 0; f < NF; ++f) s += Wx[f * N3 + idx];
    dh[cell * N3 + idx] = s;
    die[cell * N3 + idx] = Wx[idx];
  }
}

// Kernel attributes (dynamic shared memory above 48 KB, maximum carveout), set
// once per kernel and device, so that later launches -- also inside CUDA-graph
// capture -- make no attribute calls.
template <typename Kern>
int prep(dgx_ctx *c, Kern k, size_t smem) {
  static std::mutex mu;
  static std::set<std::pair<int, const void *>> done;  // (device, kernel)
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
  return check_cuda(c, e, "cudaFuncSetAttribute");
}

int threads_for(int N) { return N <= 3 ? 128 : 256; }

constexpr int kLegacyThreads[3] = {128, 192, 256};

// variant in use for precision T: the chosen one, else the default of the degree
template <typename T>
int op_variant(const dgx_ctx *c) {
  return c->op_variant[sizeof(T) == 8 ? 0 : 1];
}

template <typename T>
int op_threads(const dgx_ctx *c, int N) {
  const int v = op_variant<T>(c);
  return (v >= 0 && v < 3) ? kLegacyThreads[v] : threads_for(N);
}

template <typename T, int N, bool CURVED>
int grad_main(dgx_ctx *c, const T *p, const T *rho, T *V, cudaStream_t s, bool inv, double alpha) {
  constexpr int Q = 2 * N - 1;
  const size_t smem = sizeof(T) * GradL<N, Q, CURVED>::total;
  if constexpr (sizeof(T) == 8)
    if (op_variant<T>(c) >= 5) return fused_grad<df64, N, CURVED>(c, p, rho, V, s, inv, alpha, op_variant<T>(c) - 5);
  if (op_variant<T>(c) >= 3) return fused_grad<T, N, CURVED>(c, p, rho, V, s, inv, alpha, op_variant<T>(c) - 3);
  auto k = inv ? k_grad<T, N, Q, CURVED, true> : k_grad<T, N, Q, CURVED, false>;
  if (int e = prep(c, k, smem)) return e;
  for (int pi = 0; pi < num_patches(c); ++pi) {
    OpP<T> P = make_params<T>(c, pi);
    if (alpha >= 0.0) P.alpha = (T)alpha;
    const long long o = patch_cell0(c, pi) * N * N * N;
    count_launch();
    k<<<(unsigned)patch_ncell(c, pi), op_threads<T>(c, N), smem, s>>>(P, p + o, rho + o, V + o, c->N);
  }
  return check_cuda(c, cudaGetLastError(), "k_grad launch");
}

template <typename T, int N, bool CURVED>
int grad_impl(dgx_ctx *c, const T *p, const T *rho, T *V, cudaStream_t s, bool inv, double alpha) {
  if (int e = grad_main<T, N, CURVED>(c, p, rho, V, s, inv, alpha)) return e;
  return c->nc ? launch_hang_grad<T>(c, p, rho, V, s, inv, alpha) : 0;
}

template <typename T, int N, bool CURVED>
int div_impl(dgx_ctx *c, const T *V, const T *p, const T *pk, T *y, cudaStream_t s, double alpha) {
  constexpr int Q = 2 * N - 1;
  // the precomputed kappa applies to the context's own p_k and alpha only, and
  // to FP64 (FP32 interpolates p_k faster than it loads the Q^3 values)
  const T *kq = nullptr;
  if constexpr (sizeof(T) == 8)
    if (alpha < 0.0 && pk == c->pk64 && c->kq64_version == c->coef_version) kq = reinterpret_cast<const T *>(c->kq64);
  int e = 0;
  if constexpr (sizeof(T) == 8)
    if (op_variant<T>(c) >= 5) {
      if ((e = fused_div<df64, N, CURVED>(c, V, p, pk, y, s, alpha, kq, op_variant<T>(c) - 5))) return e;
      return c->nc ? launch_hang_div<T>(c, V, pk, y, s, alpha) : 0;
    }
  if (op_variant<T>(c) >= 3) {
    if ((e = fused_div<T, N, CURVED>(c, V, p, pk, y, s, alpha, kq, op_variant<T>(c) - 3))) return e;
    return c->nc ? launch_hang_div<T>(c, V, pk, y, s, alpha) : 0;
  }
  const size_t smem = sizeof(T) * DivL<N, Q, CURVED>::total;
  auto k = k_div<T, N, Q, CURVED>;
  if ((e = prep(c, k, smem))) return e;
  for (int pi = 0; pi < num_patches(c); ++pi) {
    OpP<T> P = make_params<T>(c, pi);
    if (alpha >= 0.0) P.alpha = (T)alpha;
    const long long o = patch_cell0(c, pi) * N * N * N, oq = patch_cell0(c, pi) * Q * Q * Q;
    count_launch();
    k<<<(unsigned)patch_ncell(c, pi), op_threads<T>(c, N), smem, s>>>(P, V + o, p + o, pk + o, y + o, c->N,
                                                                      kq ? kq + oq : nullptr);
  }
  if ((e = check_cuda(c, cudaGetLastError(), "k_div launch"))) return e;
  return c->nc ? launch_hang_div<T>(c, V, pk, y, s, alpha) : 0;
}

template <typename T, int N, bool CURVED>
int kappa_impl(dgx_ctx *c, const T *pk, T *kq, cudaStream_t s) {
  constexpr int Q = 2 * N - 1;
  const size_t smem = sizeof(T) * (((tab_size(N, Q) + 1) & ~1) + N * N * N + N * N * Q + N * Q * Q + Q * Q * Q);
  auto k = k_kappa<T, N, Q>;
  if (int e = prep(c, k, smem)) return e;
  count_launch();
  k<<<(unsigned)c->ncell, 128, smem, s>>>(make_params<T>(c), pk, kq);
  return check_cuda(c, cudaGetLastError(), "k_kappa launch");
}

template <typename T, int N, bool CURVED>
int minv_impl(dgx_ctx *c, const T *in, const T *rho, T *out, cudaStream_t s, int nf) {
  constexpr int Q = 2 * N - 1;
  const size_t smem = sizeof(T) * MinvL<N, Q>::total;
  auto k = k_minv<T, N, Q, CURVED>;
  if (int e = prep(c, k, smem)) return e;
  for (int pi = 0; pi < num_patches(c); ++pi) {
    const long long o = patch_cell0(c, pi) * N * N * N;
    count_launch();
    k<<<(unsigned)patch_ncell(c, pi), 128, smem, s>>>(make_params<T>(c, pi), in + o, rho + o, out + o, c->N, nf);
  }
  return check_cuda(c, cudaGetLastError(), "k_minv launch");
}

template <typename T, int N, bool CURVED>
int diag_impl(dgx_ctx *c, const T *rho, const T *pk, T *dh, T *die, cudaStream_t s) {
  constexpr int Q = 2 * N - 1;
  const size_t smem = sizeof(T) * DiagL<N, Q, CURVED>::total;
  auto k = k_diag<T, N, Q, CURVED>;
  if (int e = prep(c, k, smem)) return e;
  for (int pi = 0; pi < num_patches(c); ++pi) {
    const long long o = patch_cell0(c, pi) * N * N * N;
    count_launch();
    k<<<(unsigned)patch_ncell(c, pi), threads_for(N), smem, s>>>(make_params<T>(c, pi), rho + o, pk + o, dh + o,
                                                                 die + o);
  }
  return check_cuda(c, cudaGetLastError(), "k_diag launch");
}

template <typename T, int N, bool CURVED>
int opmulti_impl(dgx_ctx *c, const EnsMember<T> *mem, int nmem, long long ncell, const T *x, T *y, cudaStream_t s,
                 int threads) {
  constexpr int Q = 2 * N - 1;
  const size_t sg = sizeof(T) * GradL<N, Q, CURVED>::total, sd = sizeof(T) * DivL<N, Q, CURVED>::total;
  auto kg = k_grad_multi<T, N, Q, CURVED>;
  auto kd = k_div_multi<T, N, Q, CURVED>;
  if (int e = prep(c, kg, sg)) return e;
  if (int e = prep(c, kd, sd)) return e;
  count_launch(2);
  kg<<<(unsigned)ncell, threads, sg, s>>>(mem, nmem, x);
  kd<<<(unsigned)ncell, threads, sd, s>>>(mem, nmem, x, y);
  return check_cuda(c, cudaGetLastError(), "multi-mesh operator launch");
}

#define DGX_DISPATCH(CALL)                                                         \
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

int ensure_const_tables(dgx_ctx *c) { return upload_const_tables(c); }

// Integer and geometric parameters of a patch, shared by every precision: the
// children block of a non-conforming mesh has half the base cell sizes and,
// relative to its own bottom zeta_0, the map z - zeta_0 = zeta' + h' (1 -
// zeta'/H') with H' = Lz - zeta_0 and h' = h (1 - zeta_0/Lz) (the same points
// as the base map; its terrain tables hold h').
struct PatchGeo {
  int nx, ny, nz, hole[6], iface;
  double dx, dy, dz, H;
  long long col_off;
};
static PatchGeo patch_geo(const dgx_ctx *c, int patch) {
  const dgx_mesh_desc &m = c->mesh;
  PatchGeo g{};
  g.dx = m.Lx / m.nx;
  g.dy = m.Ly / m.ny;
  g.dz = m.Lz / m.nz;
  g.H = m.Lz;
  if (patch == 0) {
    g.nx = m.nx;
    g.ny = m.ny;
    g.nz = m.nz;
    if (c->nc)
      for (int i = 0; i < 6; ++i) g.hole[i] = m.refine[i];
    return g;
  }
  g.nx = c->fine[0];
  g.ny = c->fine[1];
  g.nz = c->fine[2];
  g.dx *= 0.5;
  g.dy *= 0.5;
  g.dz *= 0.5;
  g.H = m.Lz - c->zoff;
  g.col_off = c->col1_off * col_size(c->n, c->q);
  const int ext[3] = {m.nx, m.ny, m.nz};
  for (int k = 0; k < 3; ++k) {
    if (m.refine[2 * k] > 0) g.iface |= 1 << (2 * k);
    if (m.refine[2 * k + 1] < ext[k]) g.iface |= 1 << (2 * k + 1);
  }
  return g;
}

template <typename T>
OpP<T> make_params(const dgx_ctx *c, int patch) {
  const PatchGeo g = patch_geo(c, patch);
  OpP<T> P;
  P.nx = g.nx;
  P.ny = g.ny;
  P.nz = g.nz;
  P.bc_lat = c->mesh.bc_lateral;
  for (int i = 0; i < 6; ++i) P.hole[i] = g.hole[i];
  P.iface = g.iface;
  P.pad_ = 0;
  P.dx = (T)g.dx;
  P.dy = (T)g.dy;
  P.dz = (T)g.dz;
  P.H = (T)g.H;
  P.invH = (T)(1.0 / g.H);
  P.alpha = (T)c->alpha;
  P.gfac = (T)(c->gamma / (c->gamma - 1.0));
  P.igm1 = (T)(1.0 / (c->gamma - 1.0));
  if constexpr (sizeof(T) == 8) {
    P.tab = reinterpret_cast<const T *>(c->tab64);
    P.col = c->col64 ? reinterpret_cast<const T *>(c->col64 + g.col_off) : nullptr;
  } else {
    P.tab = reinterpret_cast<const T *>(c->tab32);
    P.col = c->col32 ? reinterpret_cast<const T *>(c->col32 + g.col_off) : nullptr;
  }
  return P;
}
template OpP<double> make_params<double>(const dgx_ctx *, int);
template OpP<float> make_params<float>(const dgx_ctx *, int);
// double-word parameters: every scalar split from its double; the terrain
// columns as double-words; the 1D tables live in constant memory only
template <>
OpP<df64> make_params<df64>(const dgx_ctx *c, int patch) {
  const PatchGeo g = patch_geo(c, patch);
  OpP<df64> P;
  P.nx = g.nx;
  P.ny = g.ny;
  P.nz = g.nz;
  P.bc_lat = c->mesh.bc_lateral;
  for (int i = 0; i < 6; ++i) P.hole[i] = g.hole[i];
  P.iface = g.iface;
  P.pad_ = 0;
  P.dx = df64(g.dx);
  P.dy = df64(g.dy);
  P.dz = df64(g.dz);
  P.H = df64(g.H);
  P.invH = df64(1.0 / g.H);
  P.alpha = df64(c->alpha);
  P.gfac = df64(c->gamma / (c->gamma - 1.0));
  P.igm1 = df64(1.0 / (c->gamma - 1.0));
  P.tab = nullptr;
  P.col = c->coldf ? reinterpret_cast<const df64 *>(c->coldf + 2 * g.col_off) : nullptr;
  return P;
}

template <typename T>
bool op_variant_ok(const dgx_ctx *c, int v) {
  if (v < 0 || v >= kOpVariants) return false;
  if (v < 3) return true;
  if (v >= 5 && sizeof(T) != 8) return false;  // double-word kernels: FP64 arrays only
  size_t smem = 0;
#define FSM(NN)                                                                                                  \
  (v >= 5 ? (c->curved ? fused_smem<df64, NN, true>(v - 5) : fused_smem<df64, NN, false>(v - 5))                  \
          : (c->curved ? fused_smem<T, NN, true>(v - 3) : fused_smem<T, NN, false>(v - 3)))
  switch (c->n) {
    case 2: smem = FSM(2); break;
    case 3: smem = FSM(3); break;
    case 4: smem = FSM(4); break;
    case 5: smem = FSM(5); break;
    case 6: smem = FSM(6); break;
    case 7: smem = FSM(7); break;
    default: return false;
  }
#undef FSM
  return smem <= kFusedMaxSmem;
}
template bool op_variant_ok<double>(const dgx_ctx *, int);
template bool op_variant_ok<float>(const dgx_ctx *, int);

int op_variant_threads(const dgx_ctx *c, int v) {
  if (v >= 0 && v < 3) return kLegacyThreads[v];
  if (v >= 3 && v < 5) return fused_nt(c->n, v - 3);
  if (v >= 5 && v < kOpVariants) return fused_nt(c->n, v - 5);
  return threads_for(c->n);
}

template <typename T>
int launch_grad(dgx_ctx *c, const T *p, const T *rho, T *V, cudaStream_t s, bool inv, double alpha) {
#define CALL_GRAD(NN, CC) grad_impl<T, NN, CC>(c, p, rho, V, s, inv, alpha)
  DGX_DISPATCH(CALL_GRAD)
#undef CALL_GRAD
}

template <typename T>
int launch_div(dgx_ctx *c, const T *V, const T *p, const T *pk, T *y, cudaStream_t s, double alpha) {
#define CALL_DIV(NN, CC) div_impl<T, NN, CC>(c, V, p, pk, y, s, alpha)
  DGX_DISPATCH(CALL_DIV)
#undef CALL_DIV
}

template <typename T>
int launch_mass_inverse(dgx_ctx *c, const T *in, const T *rho, T *out, cudaStream_t s, int nf) {
#define CALL_MINV(NN, CC) minv_impl<T, NN, CC>(c, in, rho, out, s, nf)
  DGX_DISPATCH(CALL_MINV)
#undef CALL_MINV
}

template <typename T>
int launch_kappa(dgx_ctx *c, const T *pk, T *kq, cudaStream_t s) {
#define CALL_KAPPA(NN, CC) kappa_impl<T, NN, CC>(c, pk, kq, s)
  DGX_DISPATCH(CALL_KAPPA)
#undef CALL_KAPPA
}
template int launch_kappa<double>(dgx_ctx *, const double *, double *, cudaStream_t);

template <typename T>
int launch_diag(dgx_ctx *c, const T *rho, const T *pk, T *dh, T *die, cudaStream_t s) {
#define CALL_DIAG(NN, CC) diag_impl<T, NN, CC>(c, rho, pk, dh, die, s)
  DGX_DISPATCH(CALL_DIAG)
#undef CALL_DIAG
}
template int launch_diag<double>(dgx_ctx *, const double *, const double *, double *, double *, cudaStream_t);
template int launch_diag<float>(dgx_ctx *, const float *, const float *, float *, float *, cudaStream_t);

template <typename T>
int launch_operator_multi(dgx_ctx *c, int n, bool curved, const EnsMember<T> *mem, int nmem, long long ncell,
                          const T *x, T *y, cudaStream_t s, int threads) {
  if (threads < 32 || threads > 256 || threads % 32) return set_error(c, DGX_ERR_ARG, "threads %d", threads);
  switch (n) {
    case 2: return curved ? opmulti_impl<T, 2, true>(c, mem, nmem, ncell, x, y, s, threads) : opmulti_impl<T, 2, false>(c, mem, nmem, ncell, x, y, s, threads);
    case 3: return curved ? opmulti_impl<T, 3, true>(c, mem, nmem, ncell, x, y, s, threads) : opmulti_impl<T, 3, false>(c, mem, nmem, ncell, x, y, s, threads);
    case 4: return curved ? opmulti_impl<T, 4, true>(c, mem, nmem, ncell, x, y, s, threads) : opmulti_impl<T, 4, false>(c, mem, nmem, ncell, x, y, s, threads);
    case 5: return curved ? opmulti_impl<T, 5, true>(c, mem, nmem, ncell, x, y, s, threads) : opmulti_impl<T, 5, false>(c, mem, nmem, ncell, x, y, s, threads);
    case 6: return curved ? opmulti_impl<T, 6, true>(c, mem, nmem, ncell, x, y, s, threads) : opmulti_impl<T, 6, false>(c, mem, nmem, ncell, x, y, s, threads);
    case 7: return curved ? opmulti_impl<T, 7, true>(c, mem, nmem, ncell, x, y, s, threads) : opmulti_impl<T, 7, false>(c, mem, nmem, ncell, x, y, s, threads);
    default: return set_error(c, DGX_ERR_ARG, "unsupported degree %d", n - 1);
  }
}
template int launch_operator_multi<double>(dgx_ctx *, int, bool, const EnsMember<double> *, int, long long,
                                           const double *, double *, cudaStream_t, int);
template int launch_operator_multi<float>(dgx_ctx *, int, bool, const EnsMember<float> *, int, long long,
                                          const float *, float *, cudaStream_t, int);

template int launch_grad<double>(dgx_ctx *, const double *, const double *, double *, cudaStream_t, bool, double);
template int launch_grad<float>(dgx_ctx *, const float *, const float *, float *, cudaStream_t, bool, double);
template int launch_div<double>(dgx_ctx *, const double *, const double *, const double *, double *, cudaStream_t,
                                double);
template int launch_div<float>(dgx_ctx *, const float *, const float *, const float *, float *, cudaStream_t, double);
template int launch_mass_inverse<double>(dgx_ctx *, const double *, const double *, double *, cudaStream_t, int);
template int launch_mass_inverse<float>(dgx_ctx *, const float *, const float *, float *, cudaStream_t, int);

}  // namespace dgx
