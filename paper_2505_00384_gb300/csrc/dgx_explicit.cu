// Explicit part of the IMEX step (arXiv:2505.00384, Sec. 2, stage equations):
// DG weak forms of -div(rho u), -div(rho u_d u), -div(rho k u) with a local
// Lax-Friedrichs flux, the explicit gravity work rho g.u, and the mass-type
// terms that assemble the stage right-hand sides.  FP64, one cell per CTA,
// sum factorisation through shared memory (the sweep machinery of
// dgx_sweep.cuh), the consistent 2r+1 Gauss rule.
//
// Readings of the open points (the CPU oracle implements the same
// definitions independently): Lax-Friedrichs speed max(|u-.n|, |u+.n|) (the
// acoustic part is implicit); slip walls by the mirror state rho+ = rho-,
// u+ = u- - 2 (u-.n) n; far-field faces with rho+ = rho_bar, u+ = (u_bar, 0, 0).
#include "dgx_common.cuh"
#include "dgx_fused.cuh"  // the double-word tables and line product (dgx_sweep.cuh's sweeps in double-words)

namespace dgx {
namespace {

constexpr int cmax2(int a, int b) { return a > b ? a : b; }

// T: the arithmetic, double (FP64 pipe) or df64 (double-words on the FP32
// pipes); the arrays are FP64 either way.
template <typename T>
struct ExP {
  OpP<T> P;
  T g, ubar;
  const double *tab64;  // the 1D tables in FP64 (double-words convert them while staging)
};

template <int N, int Q>
struct ExL {
  static constexpr int N2 = N * N, N3 = N * N * N, Q2 = Q * Q, Q3 = Q * Q * Q;
  static constexpr int TAB = (tab_size(N, Q) + 1) & ~1;
  static constexpr int oIn = TAB, oOut = oIn + 5 * N3;
  static constexpr int oR1 = oOut + 5 * N3;          // x sweep of 4 fields; later Wy (3 fields)
  static constexpr int oR2 = oR1 + 4 * N2 * Q;       // y sweep of 4 fields; later Wz (3 fields)
  static constexpr int oVQ = oR2 + 4 * N * Q2;       // rho, u0, u1, u2 at the Q^3 points
  static constexpr int oFL = oVQ + 4 * Q3;           // three flux fields of one quantity
  static constexpr int oWx = oFL + 3 * Q3;           // x sweep output (3 fields)
  static constexpr int oU = oWx + 3 * N3;            // w adj(J) u (contravariant velocity times weight)
  static constexpr int oEnd = oU + 3 * Q3;
  // faces reuse everything from oR1 on (volume finished)
  static constexpr int szFace = 8 * cmax2(N2, Q2) + 8 * N * Q + 5 * Q2 + 5 * N * Q + 5 * N2;
  static constexpr int total = cmax2(oEnd, oR1 + szFace);
  static_assert(3 * Q * N2 <= 4 * N2 * Q && 3 * Q2 * N <= 4 * N * Q2, "layout");
};

template <typename T, int N, int Q, bool CURVED>
__global__ void __launch_bounds__(256) k_explicit(const ExP<T> X, const double *__restrict__ rho,
                                                  const double *__restrict__ u, const double *__restrict__ rho_bar,
                                                  double *__restrict__ Erho, double *__restrict__ Em,
                                                  double *__restrict__ Ee, long long Ntot) {
  using L = ExL<N, Q>;
  constexpr int N2 = L::N2, N3 = L::N3, Q2 = L::Q2, Q3 = L::Q3;
  const OpP<T> &P = X.P;
  extern __shared__ __align__(16) unsigned char smraw[];
  T *sm = reinterpret_cast<T *>(smraw);
  T *tab = sm, *s_in = sm + L::oIn, *s_out = sm + L::oOut, *R1 = sm + L::oR1, *R2 = sm + L::oR2, *VQ = sm + L::oVQ,
    *FL = sm + L::oFL, *Wx = sm + L::oWx, *U = sm + L::oU;
  T *Wy = R1, *Wz = R2;
  const long long cell = blockIdx.x;
  const CellPos cp = cell_pos(P, cell);
  __shared__ long long s_nb[6];  // the six face neighbours (-1: boundary, -2: skipped), read after the first barrier
  if (threadIdx.x < 6) s_nb[threadIdx.x] = neighbour(P, cp, threadIdx.x);
  const T *colp = CURVED ? P.col + (long long)(cp.cx + P.nx * cp.cy) * col_size(N, Q) : nullptr;
  const T zeta0 = T(cp.cz) * P.dz;

  if constexpr (std::is_same<T, df64>::value) {
    for (int i = threadIdx.x; i < tab_size(N, Q); i += blockDim.x) tab[i] = T(X.tab64[i]);
  } else {
    load_tables<T, N, Q>(P.tab, tab);
  }
  for (int i = threadIdx.x; i < N3; i += blockDim.x) {
    s_in[i] = rho[cell * N3 + i];
    s_in[N3 + i] = u[cell * N3 + i];
    s_in[2 * N3 + i] = u[Ntot + cell * N3 + i];
    s_in[3 * N3 + i] = u[2 * Ntot + cell * N3 + i];
    s_in[4 * N3 + i] = rho_bar[cell * N3 + i];
  }
  for (int i = threadIdx.x; i < 5 * N3; i += blockDim.x) s_out[i] = T(0);
  __syncthreads();
  const T *wq = tab + tab_off_wq(N, Q), *gq = tab + tab_off_gq(N, Q);

  sweep<T, N, 0, Q, N, N, N, N, M_I, M_I, M_I>(4, 0u, s_in, R1);
  __syncthreads();
  sweep<T, N, 1, Q, N, Q, N, N, M_I, M_I, M_I>(4, 0u, R1, R2);
  __syncthreads();
  sweep<T, N, 2, Q, N, Q, Q, N, M_I, M_I, M_I>(4, 0u, R2, VQ);
  __syncthreads();

  // volume: int q_c u . grad psi = sum_j D_j^T (q_c U_j), U_j = w sum_d adj_{jd} u_d the same for
  // every quantity q_c (weighted metric products from the column table); pass 5 = gravity work
  for (int idx = threadIdx.x; idx < Q3; idx += blockDim.x) {
    const int i = idx % Q, j = (idx / Q) % Q, k = idx / Q2;
    const T v0 = VQ[Q3 + idx], v1 = VQ[2 * Q3 + idx], v2 = VQ[3 * Q3 + idx];
    if (CURVED) {
      const int t = i + Q * j;
      const T wk = wq[k], wf = wk * (T(1) - (zeta0 + P.dz * gq[k]) * P.invH);
      U[idx] = wk * colp[col_off_w(N, Q, 0) + t] * v0;
      U[Q3 + idx] = wk * colp[col_off_w(N, Q, 1) + t] * v1;
      U[2 * Q3 + idx] =
          wk * colp[col_off_w(N, Q, 2) + t] * v2 + wf * (colp[col_off_w(N, Q, 3) + t] * v0 + colp[col_off_w(N, Q, 4) + t] * v1);
    } else {
      const T w = wq[i] * wq[j] * wq[k];
      U[idx] = w * P.dy * P.dz * v0;
      U[Q3 + idx] = w * P.dx * P.dz * v1;
      U[2 * Q3 + idx] = w * P.dx * P.dy * v2;
    }
  }
  __syncthreads();
  for (int c = 0; c < 6; ++c) {
    for (int idx = threadIdx.x; idx < Q3; idx += blockDim.x) {
      const T r = VQ[idx], v0 = VQ[Q3 + idx], v1 = VQ[2 * Q3 + idx], v2 = VQ[3 * Q3 + idx];
      if (c < 5) {
        const T q = c == 0 ? r : (c == 1 ? r * v0 : (c == 2 ? r * v1 : (c == 3 ? r * v2 : T(0.5) * r * (v0 * v0 + v1 * v1 + v2 * v2))));
        FL[idx] = q * U[idx];
        FL[Q3 + idx] = q * U[Q3 + idx];
        FL[2 * Q3 + idx] = q * U[2 * Q3 + idx];
      } else {
        const int i = idx % Q, j = (idx / Q) % Q, k = idx / Q2;
        const T wdet = CURVED ? wq[k] * colp[col_off_w(N, Q, 5) + i + Q * j] : wq[i] * wq[j] * wq[k] * P.dx * P.dy * P.dz;
        FL[idx] = -X.g * r * v2 * wdet;
      }
    }
    __syncthreads();
    const int nf = c < 5 ? 3 : 1;
    const unsigned sz = c < 5 ? (1u << 4) : 0u, sy = c < 5 ? (1u << 2) : 0u, sx = c < 5 ? 1u : 0u;
    sweep<T, N, 2, N, Q, Q, Q, Q, M_IT, M_DT, M_DT>(nf, sz, FL, Wz);
    __syncthreads();
    sweep<T, N, 1, N, Q, Q, Q, N, M_IT, M_DT, M_DT>(nf, sy, Wz, Wy);
    __syncthreads();
    sweep<T, N, 0, N, Q, Q, N, N, M_IT, M_DT, M_DT>(nf, sx, Wy, Wx);
    __syncthreads();
    const int co = c < 5 ? c : 4;
    for (int idx = threadIdx.x; idx < N3; idx += blockDim.x) {
      T acc = s_out[co * N3 + idx];
      for (int f = 0; f < nf; ++f) acc += Wx[f * N3 + idx];
      s_out[co * N3 + idx] = acc;
    }
    __syncthreads();
  }

  // faces, one at a time: - int F^ psi with the local Lax-Friedrichs flux
  T *G = sm + L::oR1, *F2 = G, *F1 = G + cmax2(8 * N2, 8 * Q2), *Ff = F1 + 8 * N * Q, *Fb1 = Ff + 5 * Q2,
    *Fb2 = Fb1 + 5 * N * Q;
  for (int f = 0; f < 6; ++f) {
    const int kd = f >> 1, s = f & 1;
    const long long nb = s_nb[f];
    if (nb == -2) continue;  // non-conforming meshes: the hanging-face kernel's (uniform per CTA)
    const bool wall = nb < 0 && (kd == 2 || P.bc_lat == 0);
    const bool far = nb < 0 && !wall;
    for (int idx = threadIdx.x; idx < 8 * N2; idx += blockDim.x) {
      const int sl = idx / N2, t = idx % N2, t1 = t % N, t2 = t / N;
      const int fld = sl & 3;  // 0 rho, 1..3 u
      const int own = face_node<N>(kd, s ? N - 1 : 0, t1, t2);
      T v;
      if (sl < 4 || wall) {
        v = s_in[fld * N3 + own];
      } else if (far) {
        v = fld == 0 ? s_in[4 * N3 + own] : (fld == 1 ? X.ubar : T(0));
      } else {
        const long long nn = nb * N3 + face_node<N>(kd, s ? 0 : N - 1, t1, t2);
        v = fld == 0 ? rho[nn] : u[(long long)(fld - 1) * Ntot + nn];
      }
      G[idx] = v;
    }
    __syncthreads();
    sweep<T, N, 0, Q, N, N, N, 1, M_I, M_I, M_I>(8, 0u, G, F1);
    __syncthreads();
    sweep<T, N, 1, Q, N, Q, N, 1, M_I, M_I, M_I>(8, 0u, F1, F2);
    __syncthreads();
    for (int idx = threadIdx.x; idx < Q2; idx += blockDim.x) {
      const int i = idx % Q, j = idx / Q;
      T nA[3];
      face_normal<T, N, Q, CURVED>(P, colp, zeta0, f, i, j, nA);
      const T rm = F2[idx], vm0 = F2[Q2 + idx], vm1 = F2[2 * Q2 + idx], vm2 = F2[3 * Q2 + idx];
      T rp = F2[4 * Q2 + idx], vp0 = F2[5 * Q2 + idx], vp1 = F2[6 * Q2 + idx], vp2 = F2[7 * Q2 + idx];
      if (wall) {  // mirror state: u+ = u- - 2 (u-.n) n with n = nA / |nA|
        const T un = (vm0 * nA[0] + vm1 * nA[1] + vm2 * nA[2]) / (nA[0] * nA[0] + nA[1] * nA[1] + nA[2] * nA[2]);
        rp = rm;
        vp0 = vm0 - T(2) * un * nA[0];
        vp1 = vm1 - T(2) * un * nA[1];
        vp2 = vm2 - T(2) * un * nA[2];
      }
      const T unm = vm0 * nA[0] + vm1 * nA[1] + vm2 * nA[2];
      const T unp = vp0 * nA[0] + vp1 * nA[1] + vp2 * nA[2];
      const T lam = tmax(tabs(unm), tabs(unp));  // lambda |nA|
      const T km = T(0.5) * (vm0 * vm0 + vm1 * vm1 + vm2 * vm2), kp = T(0.5) * (vp0 * vp0 + vp1 * vp1 + vp2 * vp2);
      const T qm[5] = {rm, rm * vm0, rm * vm1, rm * vm2, rm * km};
      const T qp[5] = {rp, rp * vp0, rp * vp1, rp * vp2, rp * kp};
      const T w = wq[i] * wq[j];
#pragma unroll
      for (int c = 0; c < 5; ++c)
        Ff[c * Q2 + idx] = -w * (T(0.5) * (qm[c] * unm + qp[c] * unp) + T(0.5) * lam * (qm[c] - qp[c]));
    }
    __syncthreads();
    sweep<T, N, 0, N, Q, Q, Q, 1, M_IT, M_IT, M_IT>(5, 0u, Ff, Fb1);
    __syncthreads();
    sweep<T, N, 1, N, Q, N, Q, 1, M_IT, M_IT, M_IT>(5, 0u, Fb1, Fb2);
    __syncthreads();
    for (int idx = threadIdx.x; idx < 5 * N2; idx += blockDim.x) {
      const int c = idx / N2, t = idx % N2, t1 = t % N, t2 = t / N;
      s_out[c * N3 + face_node<N>(kd, s ? N - 1 : 0, t1, t2)] += Fb2[idx];
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < N3; i += blockDim.x) {
    Erho[cell * N3 + i] = static_cast<double>(s_out[i]);
    Em[cell * N3 + i] = static_cast<double>(s_out[N3 + i]);
    Em[Ntot + cell * N3 + i] = static_cast<double>(s_out[2 * N3 + i]);
    Em[2 * Ntot + cell * N3 + i] = static_cast<double>(s_out[3 * N3 + i]);
    Ee[cell * N3 + i] = static_cast<double>(s_out[4 * N3 + i]);
  }
}

// Consistent-rule mass of a pointwise expression:
//   MODE 0: out_i = scale int f0 psi_i;   MODE 1: out_i = scale int f0 |(f1,f2,f3)|^2 / 2 psi_i.
template <int N, int Q>
struct CmL {
  static constexpr int N2 = N * N, N3 = N * N * N, Q2 = Q * Q, Q3 = Q * Q * Q;
  static constexpr int TAB = (tab_size(N, Q) + 1) & ~1;
  static constexpr int oIn = TAB, oR1 = oIn + 4 * N3, oR2 = oR1 + 4 * N2 * Q, oR3 = oR2 + 4 * N * Q2,
                       oZ = oR3 + 4 * Q3, oY = oZ + Q2 * N, oX = oY + Q * N2, total = oX + N3;
};

template <typename T, int N, int Q, bool CURVED, int MODE>
__global__ void __launch_bounds__(256) k_cmass(const OpP<T> P, T scale, const double *__restrict__ tab64,
                                               const double *__restrict__ f0, const double *__restrict__ fv,
                                               double *__restrict__ out, long long Ntot) {
  using L = CmL<N, Q>;
  constexpr int N3 = L::N3, Q2 = L::Q2, Q3 = L::Q3;
  constexpr int NF = MODE == 0 ? 1 : 4;
  extern __shared__ __align__(16) unsigned char smraw[];
  T *sm = reinterpret_cast<T *>(smraw);
  T *tab = sm, *s_in = sm + L::oIn, *R1 = sm + L::oR1, *R2 = sm + L::oR2, *R3 = sm + L::oR3, *Wz = sm + L::oZ,
    *Wy = sm + L::oY, *Wx = sm + L::oX;
  const long long cell = blockIdx.x;
  const CellPos cp = cell_pos(P, cell);
  const T *colp = CURVED ? P.col + (long long)(cp.cx + P.nx * cp.cy) * col_size(N, Q) : nullptr;
  if constexpr (std::is_same<T, df64>::value) {
    for (int i = threadIdx.x; i < tab_size(N, Q); i += blockDim.x) tab[i] = T(tab64[i]);
  } else {
    load_tables<T, N, Q>(P.tab, tab);
  }
  for (int i = threadIdx.x; i < N3; i += blockDim.x) {
    s_in[i] = f0[cell * N3 + i];
    if (MODE == 1) {
      s_in[N3 + i] = fv[cell * N3 + i];
      s_in[2 * N3 + i] = fv[Ntot + cell * N3 + i];
      s_in[3 * N3 + i] = fv[2 * Ntot + cell * N3 + i];
    }
  }
  __syncthreads();
  const T *wq = tab + tab_off_wq(N, Q);
  sweep<T, N, 0, Q, N, N, N, N, M_I, M_I, M_I>(NF, 0u, s_in, R1);
  __syncthreads();
  sweep<T, N, 1, Q, N, Q, N, N, M_I, M_I, M_I>(NF, 0u, R1, R2);
  __syncthreads();
  sweep<T, N, 2, Q, N, Q, Q, N, M_I, M_I, M_I>(NF, 0u, R2, R3);
  __syncthreads();
  for (int idx = threadIdx.x; idx < Q3; idx += blockDim.x) {
    const int i = idx % Q, j = (idx / Q) % Q;
    T det = P.dx * P.dy * P.dz;
    if (CURVED) det *= T(1) - colp[col_off_hq(N, Q) + i + Q * j] * P.invH;
    const int k = idx / Q2;
    T v = R3[idx];
    if (MODE == 1) v *= T(0.5) * (R3[Q3 + idx] * R3[Q3 + idx] + R3[2 * Q3 + idx] * R3[2 * Q3 + idx] +
                                  R3[3 * Q3 + idx] * R3[3 * Q3 + idx]);
    R3[idx] = scale * v * wq[i] * wq[j] * wq[k] * det;
  }
  __syncthreads();
  sweep<T, N, 2, N, Q, Q, Q, Q, M_IT, M_IT, M_IT>(1, 0u, R3, Wz);
  __syncthreads();
  sweep<T, N, 1, N, Q, Q, Q, N, M_IT, M_IT, M_IT>(1, 0u, Wz, Wy);
  __syncthreads();
  sweep<T, N, 0, N, Q, Q, N, N, M_IT, M_IT, M_IT>(1, 0u, Wy, Wx);
  __syncthreads();
  for (int i = threadIdx.x; i < N3; i += blockDim.x) out[cell * N3 + i] = static_cast<double>(Wx[i]);
}

// Forward fast density-weighted mass A(rho) v = Ia^T J Ia v (r+1 Gauss points,
// J = rho(x_q) w_q det J(x_q)), 3 components (Sec. 3.3).
template <int N, int Q>
struct MfL {
  static constexpr int N3 = N * N * N;
  static constexpr int TAB = (tab_size(N, Q) + 1) & ~1;
  static constexpr int oA = TAB, oB = oA + 4 * N3, total = oB + 4 * N3;
};

template <int N, int Q, bool CURVED>
__global__ void __launch_bounds__(128) k_mass_fwd(const OpP<double> P, const double *__restrict__ rho,
                                                  const double *__restrict__ v, double *__restrict__ out,
                                                  long long Ntot) {
  using T = double;
  using L = MfL<N, Q>;
  constexpr int N3 = L::N3;
  extern __shared__ __align__(16) unsigned char smraw[];
  T *sm = reinterpret_cast<T *>(smraw);
  T *tab = sm, *A = sm + L::oA, *B = sm + L::oB;
  const long long cell = blockIdx.x;
  const CellPos cp = cell_pos(P, cell);
  const T *colp = CURVED ? P.col + (long long)(cp.cx + P.nx * cp.cy) * col_size(N, Q) : nullptr;
  load_tables<T, N, Q>(P.tab, tab);
  for (int i = threadIdx.x; i < 4 * N3; i += blockDim.x) {
    const int d = i / N3, node = i % N3;
    A[i] = d < 3 ? v[(long long)d * Ntot + cell * N3 + node] : rho[cell * N3 + node];
  }
  __syncthreads();
  sweep<T, N, 0, N, N, N, N, N, M_IA, M_IA, M_IA>(4, 0u, A, B);
  __syncthreads();
  sweep<T, N, 1, N, N, N, N, N, M_IA, M_IA, M_IA>(4, 0u, B, A);
  __syncthreads();
  sweep<T, N, 2, N, N, N, N, N, M_IA, M_IA, M_IA>(4, 0u, A, B);
  __syncthreads();
  const T *wa = tab + tab_off_wa(N, Q);
  for (int idx = threadIdx.x; idx < 3 * N3; idx += blockDim.x) {
    const int node = idx % N3;
    const int i = node % N, j = (node / N) % N, k = node / (N * N);
    T det = P.dx * P.dy * P.dz;
    if (CURVED) det *= T(1) - colp[col_off_hqa(N, Q) + i + N * j] * P.invH;
    B[idx] *= B[3 * N3 + node] * wa[i] * wa[j] * wa[k] * det;
  }
  __syncthreads();
  sweep<T, N, 0, N, N, N, N, N, M_IAT, M_IAT, M_IAT>(3, 0u, B, A);
  __syncthreads();
  sweep<T, N, 1, N, N, N, N, N, M_IAT, M_IAT, M_IAT>(3, 0u, A, B);
  __syncthreads();
  sweep<T, N, 2, N, N, N, N, N, M_IAT, M_IAT, M_IAT>(3, 0u, B, A);
  __syncthreads();
  for (int i = threadIdx.x; i < 3 * N3; i += blockDim.x) {
    const int d = i / N3, node = i % N3;
    out[(long long)d * Ntot + cell * N3 + node] = A[i];
  }
}

template <typename Kern>
int prep2(dgx_ctx *c, Kern k, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  return check_cuda(c, e, "cudaFuncSetAttribute");
}

template <typename T, int N, bool CURVED>
int explicit_go(dgx_ctx *c, const double *rho, const double *u, const double *rho_bar, double *Er, double *Em,
                double *Ee, cudaStream_t s) {
  constexpr int Q = 2 * N - 1;
  const size_t smem = sizeof(T) * ExL<N, Q>::total;
  auto k = k_explicit<T, N, Q, CURVED>;
  if (int e = prep2(c, k, smem)) return e;
  for (int pi = 0; pi < num_patches(c); ++pi) {
    ExP<T> X{make_params<T>(c, pi), T(c->bg.g), T(c->bg.u_bar), c->tab64};
    const long long o = patch_cell0(c, pi) * N * N * N;
    count_launch();
    k<<<(unsigned)patch_ncell(c, pi), 256, smem, s>>>(X, rho + o, u + o, rho_bar + o, Er + o, Em + o, Ee + o, c->N);
  }
  return 0;
}

// The explicit fluxes in double-words (c->explicit_variant 1, degrees up to 4)
// or on the FP64 pipe.
template <int N, bool CURVED>
int explicit_impl(dgx_ctx *c, const double *rho, const double *u, const double *rho_bar, double *Er, double *Em,
                  double *Ee, cudaStream_t s) {
  int e;
  if constexpr (N <= 5) {
    if (c->explicit_variant == 1) {
      if ((e = upload_fused_tables(c))) return e;
      e = explicit_go<df64, N, CURVED>(c, rho, u, rho_bar, Er, Em, Ee, s);
    } else {
      e = explicit_go<double, N, CURVED>(c, rho, u, rho_bar, Er, Em, Ee, s);
    }
  } else {
    e = explicit_go<double, N, CURVED>(c, rho, u, rho_bar, Er, Em, Ee, s);
  }
  if (e) return e;
  if ((e = check_cuda(c, cudaGetLastError(), "k_explicit launch"))) return e;
  return c->nc ? launch_hang_explicit(c, rho, u, Er, Em, Ee, s) : 0;
}

template <int N, bool CURVED>
int cmass_impl(dgx_ctx *c, int mode, double scale, const double *f0, const double *fv, double *out, cudaStream_t s) {
  constexpr int Q = 2 * N - 1;
  auto go = [&](auto tag) -> int {
    using T = decltype(tag);
    const size_t smem = sizeof(T) * CmL<N, Q>::total;
    auto k = mode == 0 ? k_cmass<T, N, Q, CURVED, 0> : k_cmass<T, N, Q, CURVED, 1>;
    if (int e = prep2(c, k, smem)) return e;
    for (int pi = 0; pi < num_patches(c); ++pi) {
      const long long o = patch_cell0(c, pi) * N * N * N;
      count_launch();
      k<<<(unsigned)patch_ncell(c, pi), 128, smem, s>>>(make_params<T>(c, pi), T(scale), c->tab64, f0 + o,
                                                        fv ? fv + o : nullptr, out + o, c->N);
    }
    return check_cuda(c, cudaGetLastError(), "k_cmass launch");
  };
  if constexpr (N <= 5) {  // the explicit side's arithmetic (dgx_set_explicit_variant)
    if (c->explicit_variant == 1) {
      if (int e = upload_fused_tables(c)) return e;
      return go(df64{});
    }
  }
  return go(double{});
}

template <int N, bool CURVED>
int massfwd_impl(dgx_ctx *c, const double *rho, const double *v, double *out, cudaStream_t s) {
  constexpr int Q = 2 * N - 1;
  const size_t smem = sizeof(double) * MfL<N, Q>::total;
  auto k = k_mass_fwd<N, Q, CURVED>;
  if (int e = prep2(c, k, smem)) return e;
  for (int pi = 0; pi < num_patches(c); ++pi) {
    const long long o = patch_cell0(c, pi) * N * N * N;
    count_launch();
    k<<<(unsigned)patch_ncell(c, pi), 128, smem, s>>>(make_params<double>(c, pi), rho + o, v + o, out + o, c->N);
  }
  return check_cuda(c, cudaGetLastError(), "k_mass_fwd launch");
}

#define DGX_DISPATCH2(CALL)                                                        \
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

int ensure_const_tables_explicit(dgx_ctx *c) { return upload_const_tables(c); }

int launch_explicit(dgx_ctx *c, const double *rho, const double *u, const double *rho_bar, double *Er, double *Em,
                    double *Ee, cudaStream_t s) {
  if (int e = ensure_const_tables_explicit(c)) return e;
#define CALL_EX(NN, CC) explicit_impl<NN, CC>(c, rho, u, rho_bar, Er, Em, Ee, s)
  DGX_DISPATCH2(CALL_EX)
#undef CALL_EX
}

int launch_cmass(dgx_ctx *c, int mode, double scale, const double *f0, const double *fv, double *out,
                 cudaStream_t s) {
  if (int e = ensure_const_tables_explicit(c)) return e;
#define CALL_CM(NN, CC) cmass_impl<NN, CC>(c, mode, scale, f0, fv, out, s)
  DGX_DISPATCH2(CALL_CM)
#undef CALL_CM
}

int launch_mass_fwd(dgx_ctx *c, const double *rho, const double *v, double *out, cudaStream_t s) {
  if (int e = ensure_const_tables_explicit(c)) return e;
#define CALL_MF(NN, CC) massfwd_impl<NN, CC>(c, rho, v, out, s)
  DGX_DISPATCH2(CALL_MF)
#undef CALL_MF
}

}  // namespace dgx
