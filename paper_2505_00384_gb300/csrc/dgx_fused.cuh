// Fused, multi-cell kernels of the pressure (Schur) operator (arXiv:2505.00384,
// Sec. 2 and Sec. 3.3): the same two halves as k_grad / k_div,
//   kf_grad  V = A^-1 B P   (or the dual B P alone)
//   kf_div   y = D P - C V
// computed with a different schedule:
//  * CPB consecutive cells per CTA and NT threads, every stage a compile-time
//    list of 1D lines (cells x lines per cell) dealt out to the threads, so
//    that the short line counts of one cell fill the warps and a barrier
//    serves CPB cells;
//  * the last interpolation direction (z), the pointwise flux at the Q^3 Gauss
//    points and the first test direction (z again) are one pass in registers:
//    a thread owns one (x, y) column of Gauss points, so the Q^3 field is never
//    stored;
//  * the fast inverse S^-T J^-1 S^-1 of the density-weighted mass is folded
//    into the test: the test matrices times the inverse's first factor are
//    applied as one product per direction, J^-1 and the x factor of the
//    second where the x test ends;
//  * the face terms are gathered and interpolated straight from global memory
//    and added to the x-test lines that own the face nodes (no combine pass);
//  * quadrature weights and points live in constant memory next to the
//    even-odd 1D matrices, indexed at compile time.
// The arithmetic per line is that of the even-odd line products of
// dgx_sweep.cuh; only the order of the line products and where their results
// are kept differ, so the result equals k_grad / k_div to rounding.
#pragma once

#include <type_traits>

#include "dgx_sweep.cuh"

namespace dgx {
namespace {

// ---------------------------------------------------------- constant tables
// Gauss weights wq and points gq of the 2r+1 point rule and the weights wa of
// the r+1 point (fast-inverse) rule of every degree, on [0, 1], by N = r+1.
static __constant__ double c_wq64[kMaxDegree + 2][2 * kMaxDegree + 1];
static __constant__ double c_gq64[kMaxDegree + 2][2 * kMaxDegree + 1];
static __constant__ double c_wa64[kMaxDegree + 2][kMaxDegree + 1];
static __constant__ float c_wq32[kMaxDegree + 2][2 * kMaxDegree + 1];
static __constant__ float c_gq32[kMaxDegree + 2][2 * kMaxDegree + 1];
static __constant__ float c_wa32[kMaxDegree + 2][kMaxDegree + 1];
// the same rules and the even-odd 1D matrices as double-words (hi, lo)
static __constant__ float2 c_wqdf[kMaxDegree + 2][2 * kMaxDegree + 1];
static __constant__ float2 c_gqdf[kMaxDegree + 2][2 * kMaxDegree + 1];
static __constant__ float2 c_wadf[kMaxDegree + 2][kMaxDegree + 1];
static __constant__ float2 c_eodf[kEoTotal];

template <>
__device__ __forceinline__ df64 ceo<df64>(int i) {
  return df64(c_eodf[i].x, c_eodf[i].y);
}

template <typename T, int N>
__device__ __forceinline__ T cwq(int k) {
  if constexpr (std::is_same<T, df64>::value) return df64(c_wqdf[N][k].x, c_wqdf[N][k].y);
  else if constexpr (sizeof(T) == 8) return c_wq64[N][k];
  else return c_wq32[N][k];
}
template <typename T, int N>
__device__ __forceinline__ T cgq(int k) {
  if constexpr (std::is_same<T, df64>::value) return df64(c_gqdf[N][k].x, c_gqdf[N][k].y);
  else if constexpr (sizeof(T) == 8) return c_gq64[N][k];
  else return c_gq32[N][k];
}
template <typename T, int N>
__device__ __forceinline__ T cwa(int k) {
  if constexpr (std::is_same<T, df64>::value) return df64(c_wadf[N][k].x, c_wadf[N][k].y);
  else if constexpr (sizeof(T) == 8) return c_wa64[N][k];
  else return c_wa32[N][k];
}

// double-word split of a host double: hi = RN(v), lo = RN(v - hi)
static inline float2 dw_split(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

// Upload the even-odd matrices (dgx_sweep.cuh) and the rule tables into this
// translation unit's constant memory on the context's device (once per device).
static int upload_fused_tables(dgx_ctx *c) {
  if (int e = upload_const_tables(c)) return e;
  static std::mutex mu;
  static bool done[64] = {};
  std::lock_guard<std::mutex> lk(mu);
  if (done[c->device]) return 0;
  double wq[kMaxDegree + 2][2 * kMaxDegree + 1] = {}, gq[kMaxDegree + 2][2 * kMaxDegree + 1] = {};
  double wa[kMaxDegree + 2][kMaxDegree + 1] = {};
  for (int r = 1; r <= kMaxDegree; ++r) {
    const int N = r + 1, Q = 2 * r + 1;
    std::vector<double> tab;
    if (!build_table_block(r, tab)) return set_error(c, DGX_ERR_ARG, "table construction failed (r=%d)", r);
    for (int k = 0; k < Q; ++k) {
      wq[N][k] = tab[tab_off_wq(N, Q) + k];
      gq[N][k] = tab[tab_off_gq(N, Q) + k];
    }
    for (int k = 0; k < N; ++k) wa[N][k] = tab[tab_off_wa(N, Q) + k];
  }
  float wq32[kMaxDegree + 2][2 * kMaxDegree + 1], gq32[kMaxDegree + 2][2 * kMaxDegree + 1];
  float wa32[kMaxDegree + 2][kMaxDegree + 1];
  static float2 wqdf[kMaxDegree + 2][2 * kMaxDegree + 1], gqdf[kMaxDegree + 2][2 * kMaxDegree + 1];
  static float2 wadf[kMaxDegree + 2][kMaxDegree + 1];
  for (int n = 0; n < kMaxDegree + 2; ++n) {
    for (int k = 0; k < 2 * kMaxDegree + 1; ++k) {
      wq32[n][k] = (float)wq[n][k];
      gq32[n][k] = (float)gq[n][k];
      wqdf[n][k] = dw_split(wq[n][k]);
      gqdf[n][k] = dw_split(gq[n][k]);
    }
    for (int k = 0; k < kMaxDegree + 1; ++k) {
      wa32[n][k] = (float)wa[n][k];
      wadf[n][k] = dw_split(wa[n][k]);
    }
  }
  // even-odd matrices as double-words, from this translation unit's FP64 copy
  std::vector<double> eo(kEoTotal);
  std::vector<float2> eodf(kEoTotal);
  if (int err = check_cuda(c, cudaMemcpyFromSymbol(eo.data(), c_eo64, kEoTotal * sizeof(double)), "constant tables"))
    return err;
  for (int k = 0; k < kEoTotal; ++k) eodf[k] = dw_split(eo[k]);
  cudaError_t e = cudaMemcpyToSymbol(c_wq64, wq, sizeof(wq));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_gq64, gq, sizeof(gq));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_wa64, wa, sizeof(wa));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_wq32, wq32, sizeof(wq32));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_gq32, gq32, sizeof(gq32));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_wa32, wa32, sizeof(wa32));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_wqdf, wqdf, sizeof(wqdf));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_gqdf, gqdf, sizeof(gqdf));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_wadf, wadf, sizeof(wadf));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_eodf, eodf.data(), kEoTotal * sizeof(float2));
  if (int err = check_cuda(c, e, "constant rule tables")) return err;
  done[c->device] = true;
  return 0;
}

// ------------------------------------------------------------ line helpers
// Double-word line product (same even-odd scheme as line_eo): the pair sums
// e_m, d_m are kept unnormalised (TwoSum of the high parts, low parts added),
// and each output is a compensated dot product (Ogita, Rump and Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 26 (2005), Dot2):
// products of the high parts split exactly by FMA, their running sum by
// TwoSum, all low-order terms gathered in one FP32 accumulator, one
// normalisation at the end.
__device__ __forceinline__ void dot2_term(float &sh, float &sl, bool first, float ch, float cl, float xh, float xl) {
  const float p = __fmul_rn(ch, xh);
  float lo = __fmaf_rn(ch, xh, -p);
  lo = __fmaf_rn(ch, xl, lo);
  lo = __fmaf_rn(cl, xh, lo);
  if (first) {
    sh = p;
    sl = lo;
  } else {
    const df64 t = two_sum(sh, p);
    sh = t.hi;
    sl = __fadd_rn(sl, __fadd_rn(t.lo, lo));
  }
}

template <int NN, int MAT, int MO, int MI>
__device__ __forceinline__ void line_dw(const df64 *x, df64 *y) {
  constexpr int HO = (MO + 1) / 2, HI = MI / 2;
  constexpr int base = eo_mat_off(NN, MAT);
  constexpr bool odd_in = (MI & 1) != 0;
  constexpr int par = mat_parity(MAT);
  float eh[HI > 0 ? HI : 1], el[HI > 0 ? HI : 1], dh[HI > 0 ? HI : 1], dl[HI > 0 ? HI : 1];
#pragma unroll
  for (int m = 0; m < HI; ++m) {
    const df64 u = x[m], v = x[MI - 1 - m];
    const df64 sp = two_sum(u.hi, v.hi), sm = two_sum(u.hi, -v.hi);
    eh[m] = sp.hi;
    el[m] = __fadd_rn(sp.lo, __fadd_rn(u.lo, v.lo));
    dh[m] = sm.hi;
    dl[m] = __fadd_rn(sm.lo, __fsub_rn(u.lo, v.lo));
  }
#pragma unroll
  for (int o = 0; o < HO; ++o) {
    float ah = 0.f, al = 0.f, bh = 0.f, bl = 0.f;
    bool afirst = true;
    if (odd_in) {
      const float2 cm = c_eodf[base + 2 * HO * HI + o];
      dot2_term(ah, al, true, cm.x, cm.y, x[HI].hi, x[HI].lo);
      afirst = false;
    }
#pragma unroll
    for (int m = 0; m < HI; ++m) {
      const float2 ce = c_eodf[base + o * HI + m], cd = c_eodf[base + HO * HI + o * HI + m];
      dot2_term(ah, al, afirst && m == 0, ce.x, ce.y, eh[m], el[m]);
      dot2_term(bh, bl, m == 0, cd.x, cd.y, dh[m], dl[m]);
    }
    const df64 a = fast_two_sum(ah, al), b = fast_two_sum(bh, bl);
    y[o] = a + b;
    if (o != MO - 1 - o) y[MO - 1 - o] = par > 0 ? a - b : b - a;
  }
}

// y = M x for register arrays (M: even-odd matrix MAT of degree NN, MO x MI).
template <typename T, int NN, int MAT, int MO, int MI>
__device__ __forceinline__ void mv(const T *x, T *y) {
  if constexpr (std::is_same<T, df64>::value) line_dw<NN, MAT, MO, MI>(x, y);
  else line_eo<T, NN, MAT, MO, MI>(x, 1, y, 1);
}
// y += M x
template <typename T, int NN, int MAT, int MO, int MI>
__device__ __forceinline__ void mv_acc(const T *x, T *y) {
  T t[MO];
  mv<T, NN, MAT, MO, MI>(x, t);
#pragma unroll
  for (int o = 0; o < MO; ++o) y[o] += t[o];
}
// M values of stride S into / out of registers; U is the memory type (the
// storage type for global arrays, converted to and from the compute type T)
template <typename T, int M, int S, typename U>
__device__ __forceinline__ void lds(const U *p, T *r) {
#pragma unroll
  for (int m = 0; m < M; ++m) r[m] = static_cast<T>(p[m * S]);
}
template <typename T, int M, int S, typename U>
__device__ __forceinline__ void sts(U *p, const T *r) {
#pragma unroll
  for (int m = 0; m < M; ++m) p[m * S] = static_cast<U>(r[m]);
}

// Neighbour across face f (2k+s) of cell `cell` (32-bit index arithmetic), -1 on
// the boundary; x and y wrap around with periodic lateral faces; -2 for a face
// the kernel skips (non-conforming meshes: dead cells, the patch interface).
template <typename T>
__device__ __forceinline__ bool hole32(const OpP<T> &P, int x, int y, int z) {
  return x >= P.hole[0] && x < P.hole[1] && y >= P.hole[2] && y < P.hole[3] && z >= P.hole[4] && z < P.hole[5];
}
template <typename T>
__device__ __forceinline__ int nb32(const OpP<T> &P, int cx, int cy, int cz, int f) {
  const int k = f >> 1, s = f & 1;
  int x = cx, y = cy, z = cz;
  if (hole32(P, x, y, z)) return -2;
  if (k == 0) {
    x += s ? 1 : -1;
    if (x < 0 || x >= P.nx) {
      if (P.iface & (1 << f)) return -2;
      if (P.bc_lat != 2) return -1;
      x = x < 0 ? P.nx - 1 : 0;
    }
  } else if (k == 1) {
    y += s ? 1 : -1;
    if (y < 0 || y >= P.ny) {
      if (P.iface & (1 << f)) return -2;
      if (P.bc_lat != 2) return -1;
      y = y < 0 ? P.ny - 1 : 0;
    }
  } else {
    z += s ? 1 : -1;
    if (z < 0 || z >= P.nz) return (P.iface & (1 << f)) ? -2 : -1;
  }
  if (hole32(P, x, y, z)) return -2;
  return x + P.nx * (y + P.ny * z);
}

// Per-cell data every stage reads: the six neighbours, the terrain column and
// the layer index, set by the first stage of a kernel.
template <int CPB>
struct CellInfo {
  int nb[CPB][6];
  int col[CPB];
  int cz[CPB];
};

template <typename T, int N, int CPB, int NT>
__device__ __forceinline__ void cell_info(const OpP<T> &P, int cell0, int ncell, CellInfo<CPB> &ci) {
  for (int t = threadIdx.x; t < CPB; t += NT) {
    const int cell = cell0 + t;
    if (cell < ncell) {
      const unsigned u = (unsigned)cell, nx = (unsigned)P.nx, ny = (unsigned)P.ny;
      const unsigned q1 = u / nx, cx = u - q1 * nx, cz = q1 / ny, cy = q1 - cz * ny;
      ci.col[t] = (int)(cx + nx * cy);
      ci.cz[t] = (int)cz;
#pragma unroll
      for (int f = 0; f < 6; ++f) ci.nb[t][f] = nb32(P, (int)cx, (int)cy, (int)cz, f);
    } else {
      ci.col[t] = 0;
      ci.cz[t] = 0;
#pragma unroll
      for (int f = 0; f < 6; ++f) ci.nb[t][f] = -1;
    }
  }
}

// Outward normal times area element of face f at face Gauss point (i, j)
// (unweighted), with the tangential order of face_node: x face (y, z), y face
// (x, z), z face (x, y).  Same expressions as face_normal in dgx_sweep.cuh.
template <typename T, int N, bool CURVED>
__device__ __forceinline__ T fnormal(const OpP<T> &P, const T *colp, T zeta0, int f, int i, int j, int d) {
  constexpr int Q = 2 * N - 1;
  const int k = f >> 1, s = f & 1;
  const T sg = s ? T(1) : T(-1);
  if (k == 0) {
    if (d != 0) return T(0);
    T z3 = P.dz;
    if (CURVED) z3 = P.dz * (T(1) - colp[col_off_hx(N, Q, s) + i] * P.invH);
    return sg * P.dy * z3;
  }
  if (k == 1) {
    if (d != 1) return T(0);
    T z3 = P.dz;
    if (CURVED) z3 = P.dz * (T(1) - colp[col_off_hy(N, Q, s) + i] * P.invH);
    return sg * P.dx * z3;
  }
  if (d == 2) return sg * P.dx * P.dy;
  if (!CURVED) return T(0);
  const T fac = T(1) - (zeta0 + T(s) * P.dz) * P.invH;
  if (d == 0) return -sg * P.dy * colp[col_off_h1q(N, Q) + i + Q * j] * fac;
  return -sg * P.dx * colp[col_off_h2q(N, Q) + i + Q * j] * fac;
}

constexpr int fmax3(int a, int b, int c) { return a > b ? (a > c ? a : c) : (b > c ? b : c); }
// Minimum resident CTAs asked of the compiler: FP32 kernels up to degree 4
// are held to 64 registers per thread (they are latency bound, so occupancy
// pays; higher degrees would spill), double-word kernels to 224; FP64 kernels
// are left free (bound by the FP64 pipe).
template <typename T, int N, int NT>
constexpr int fused_min_blocks() {
  if (sizeof(T) == 4 && N <= 5) return 65536 / (NT * 64) > 0 ? 65536 / (NT * 64) : 1;
  // double-word kernels are latency bound at ~250 registers: ask for 224 (one more CTA at r = 4)
  if (std::is_same<T, df64>::value && N <= 5) return 65536 / (NT * 224) > 0 ? 65536 / (NT * 224) : 1;
  return 1;
}
constexpr int fmax2(int a, int b) { return a > b ? a : b; }

// ------------------------------------------------------------------ kf_grad
// With INV the fast inverse A^-1 = P^3 J^-1 (P^T)^3 is folded into the test:
// the z, y and x tests use the products P^T I^T and P^T D^T (M_PIT, M_PDT),
// so the tested arrays are already at the fast-rule points; the face terms are
// tested with P^T I^T along both tangential directions and spread along the
// normal direction with the column P^T[q][e] of the face layer e.  The x-test
// lines then scale by J^-1 and apply P_x; P_y and P_z follow.  Without INV
// the plain I^T, D^T give the dual vector B p at the nodes.
//
// Per-cell shared-memory plan (elements of T), two arenas written by
// alternate stages:
//   lo: S1 A1 (x-interp of p), R1 (Ia_x rho), F2 (face traces, t1-interp)
//       S3 F4 (faces tested), JI (J^-1 at the fast points), C3 (z pass output)
//       S5 X5 (x test, J^-1, P_x) over C3
//   hi: S2 B2 (y-interp), R2 (Ia_y Ia_x rho), F3 (faces, t2 pass)
//       S4 D4 (y test)   S6 Y6 (P_y)
template <int N, bool CURVED>
struct FGradL {
  static constexpr int Q = 2 * N - 1, N2 = N * N, N3 = N2 * N, Q2 = Q * Q;
  static constexpr int NFV = CURVED ? 5 : 3;   // volume flux fields (j, d)
  static constexpr int NG = CURVED ? 4 : 3;    // fields after the y test
  static constexpr int NFP = CURVED ? 10 : 6;  // face (face, component) slots
  static constexpr int oA1 = 0, oR1 = Q * N2, oF2 = oR1 + N3;
  static constexpr int oF4 = 0, oJI = NFP * N2, oC3 = oJI + N3, oX5 = oC3;
  static constexpr int LO = fmax3(oF2 + 6 * Q * N, oC3 + NFV * Q2 * N, oX5 + 3 * N3);
  static constexpr int oB2 = LO, oR2 = LO + Q2 * N, oF3 = oR2 + N3, oD4 = LO, oY6 = LO;
  static constexpr int HI = fmax3(Q2 * N + N3 + NFP * N * Q, NG * Q * N2, 3 * N3);
  static constexpr int per_cell = ((LO + HI) + 3) & ~3;
};

// One CTA's work: cells cell0 .. cell0 + CPB - 1 (those below ncell) of the mesh of P.
template <typename T, int N, bool CURVED, bool INV, int CPB, int NT>
__device__ __forceinline__ void kf_grad_body(const OpP<T> &P, const store_t<T> *__restrict__ p,
                                             const store_t<T> *__restrict__ rho, store_t<T> *__restrict__ V,
                                             long long Ntot, int ncell, int cell0) {
  using L = FGradL<N, CURVED>;
  constexpr int Q = L::Q, N2 = L::N2, N3 = L::N3, Q2 = L::Q2, NFP = L::NFP, NG = L::NG, PC = L::per_cell;
  constexpr int MIT = INV ? M_PIT : M_IT, MDT = INV ? M_PDT : M_DT;  // test matrices
  extern __shared__ __align__(16) unsigned char smraw[];
  T *sm = reinterpret_cast<T *>(smraw);
  __shared__ CellInfo<CPB> ci;
  __shared__ T s_wq[Q], s_wa[N], s_pte[2][N];
  cell_info<T, N, CPB, NT>(P, cell0, ncell, ci);
  for (int t = threadIdx.x; t < Q; t += NT) s_wq[t] = cwq<T, N>(t);
  for (int t = threadIdx.x; t < N; t += NT) s_wa[t] = cwa<T, N>(t);
  if (INV && threadIdx.x < 2 * N) {  // columns e = 0 and N-1 of P^T: PT[q][e] = M_PIT applied to a unit trace
    const int e = threadIdx.x / N, q = threadIdx.x - e * N;
    T u[N], o[N];
#pragma unroll
    for (int a = 0; a < N; ++a) u[a] = T(0);
    u[e ? N - 1 : 0] = T(1);
    mv<T, N, M_PT, N, N>(u, o);
#pragma unroll
    for (int a = 0; a < N; ++a)
      if (a == q) s_pte[e][q] = o[a];
  }
  __syncthreads();

  // S1: x-interpolation of p, Ia_x rho, face traces p^ interpolated along t1
  {
    constexpr int W1 = N2, W2 = INV ? N2 : 0, W3 = 6 * N, WC = W1 + W2 + W3;
    for (int w = threadIdx.x; w < CPB * WC; w += NT) {
      // heavy face lines first, so that the last round holds light lines
      const int cl = w / WC, cell = cell0 + cl;
      int l = w - cl * WC + (W1 + W2);
      if (l >= WC) l -= WC;
      if (cell >= ncell) continue;
      T *cs = sm + cl * PC;
      if (l < W1) {
        T x[N], y[Q];
        lds<T, N, 1>(p + (long long)cell * N3 + N * l, x);
        mv<T, N, M_I, Q, N>(x, y);
        sts<T, Q, 1>(cs + L::oA1 + Q * l, y);
      } else if (l < W1 + W2) {
        const int m = l - W1;
        T x[N], y[N];
        lds<T, N, 1>(rho + (long long)cell * N3 + N * m, x);
        mv<T, N, M_IA, N, N>(x, y);
        sts<T, N, 1>(cs + L::oR1 + N * m, y);
      } else {
        const int m = l - W1 - W2, f = m / N, t2 = m - f * N, k = f >> 1, s = f & 1;
        const int nb = ci.nb[cl][f];
        T x[N], y[Q];
#pragma unroll
        for (int t1 = 0; t1 < N; ++t1) {
          const T own = p[(long long)cell * N3 + face_node<N>(k, s ? N - 1 : 0, t1, t2)];
          T ph = own;
          if (nb >= 0) ph = T(0.5) * (own + p[(long long)nb * N3 + face_node<N>(k, s ? 0 : N - 1, t1, t2)]);
          else if (nb == -2 || (k < 2 && P.bc_lat == 1)) ph = T(0);
          x[t1] = ph;
        }
        mv<T, N, M_I, Q, N>(x, y);
        sts<T, Q, 1>(cs + L::oF2 + f * Q * N + Q * t2, y);
      }
    }
  }
  __syncthreads();

  // S2: y-interpolation, Ia_y rho, faces: t2 interpolation, normal and weights, t2 test
  {
    constexpr int W1 = Q * N, W2 = INV ? N2 : 0, W3 = 6 * Q, WC = W1 + W2 + W3;
    for (int w = threadIdx.x; w < CPB * WC; w += NT) {
      // heavy face lines first, so that the last round holds light lines
      const int cl = w / WC, cell = cell0 + cl;
      int l = w - cl * WC + (W1 + W2);
      if (l >= WC) l -= WC;
      if (cell >= ncell) continue;
      T *cs = sm + cl * PC;
      if (l < W1) {
        const int i = l % Q, c = l / Q;
        T x[N], y[Q];
        lds<T, N, Q>(cs + L::oA1 + i + Q * N * c, x);
        mv<T, N, M_I, Q, N>(x, y);
        sts<T, Q, Q>(cs + L::oB2 + i + Q2 * c, y);
      } else if (l < W1 + W2) {
        const int m = l - W1, q = m % N, c = m / N;
        T x[N], y[N];
        lds<T, N, N>(cs + L::oR1 + q + N2 * c, x);
        mv<T, N, M_IA, N, N>(x, y);
        sts<T, N, N>(cs + L::oR2 + q + N2 * c, y);
      } else {
        const int m = l - W1 - W2, f = m / Q, i = m - f * Q, k = f >> 1;
        const T *colp = CURVED ? P.col + (long long)ci.col[cl] * col_size(N, Q) : nullptr;
        const T zeta0 = T(ci.cz[cl]) * P.dz;
        T x[N], ph[Q], v[Q], o[N];
        lds<T, N, Q>(cs + L::oF2 + f * Q * N + i, x);
        mv<T, N, M_I, Q, N>(x, ph);
        const T wi = P.alpha * s_wq[i];
        if (k < 2 || !CURVED) {  // one component (d = k), normal constant along the line
          const T nk = wi * fnormal<T, N, CURVED>(P, colp, zeta0, f, i, 0, k);
#pragma unroll
          for (int j = 0; j < Q; ++j) v[j] = nk * cwq<T, N>(j) * ph[j];
          mv<T, N, MIT, N, Q>(v, o);
          sts<T, N, Q>(cs + L::oF3 + f * N * Q + i, o);
        } else {  // curved z face: three components, slots 4 + 3 (f - 4) + d
#pragma unroll 1
          for (int d = 0; d < 3; ++d) {
#pragma unroll
            for (int j = 0; j < Q; ++j) v[j] = wi * cwq<T, N>(j) * fnormal<T, N, CURVED>(P, colp, zeta0, f, i, j, d) * ph[j];
            mv<T, N, MIT, N, Q>(v, o);
            sts<T, N, Q>(cs + L::oF3 + (4 + 3 * (f - 4) + d) * N * Q + i, o);
          }
        }
      }
    }
  }
  __syncthreads();

  // S3: z pass (interpolate, weak-gradient fluxes, z test), faces tested along t1,
  // and (INV) J^-1 at the fast points from rho (Ia_z)
  {
    constexpr int W1 = Q2, W2 = NFP * N, W3 = INV ? N2 : 0, WC = W1 + W2 + W3;
    for (int w = threadIdx.x; w < CPB * WC; w += NT) {
      const int cl = w / WC, l = w - cl * WC, cell = cell0 + cl;
      if (cell >= ncell) continue;
      T *cs = sm + cl * PC;
      if (l < W1) {
        const int i = l % Q, j = l / Q;
        T x[N], pz[Q];
        lds<T, N, Q2>(cs + L::oB2 + i + Q * j, x);
        mv<T, N, M_I, Q, N>(x, pz);
        T *out = cs + L::oC3 + i + Q * j;
        constexpr int FS = Q2 * N;  // field stride of C3
        T v[Q], o[N];
        if (CURVED) {
          const T *colp = P.col + (long long)ci.col[cl] * col_size(N, Q);
          const T wA = colp[col_off_w(N, Q, 0) + l], wB = colp[col_off_w(N, Q, 1) + l],
                  wC = colp[col_off_w(N, Q, 2) + l], wE = colp[col_off_w(N, Q, 3) + l],
                  wF = colp[col_off_w(N, Q, 4) + l];
          const T zeta0 = T(ci.cz[cl]) * P.dz;
          T aw[Q], af[Q];
#pragma unroll
          for (int k = 0; k < Q; ++k) {
            aw[k] = -P.alpha * pz[k] * cwq<T, N>(k);
            af[k] = aw[k] * (T(1) - (zeta0 + P.dz * cgq<T, N>(k)) * P.invH);
          }
          // field order: (j0,d0) I, (j2,d0) D, (j1,d1) I, (j2,d1) D, (j2,d2) D in z
#pragma unroll
          for (int k = 0; k < Q; ++k) v[k] = aw[k] * wA;
          mv<T, N, MIT, N, Q>(v, o);
          sts<T, N, Q2>(out + 0 * FS, o);
#pragma unroll
          for (int k = 0; k < Q; ++k) v[k] = af[k] * wE;
          mv<T, N, MDT, N, Q>(v, o);
          sts<T, N, Q2>(out + 1 * FS, o);
#pragma unroll
          for (int k = 0; k < Q; ++k) v[k] = aw[k] * wB;
          mv<T, N, MIT, N, Q>(v, o);
          sts<T, N, Q2>(out + 2 * FS, o);
#pragma unroll
          for (int k = 0; k < Q; ++k) v[k] = af[k] * wF;
          mv<T, N, MDT, N, Q>(v, o);
          sts<T, N, Q2>(out + 3 * FS, o);
#pragma unroll
          for (int k = 0; k < Q; ++k) v[k] = aw[k] * wC;
          mv<T, N, MDT, N, Q>(v, o);
          sts<T, N, Q2>(out + 4 * FS, o);
        } else {
          const T wij = -P.alpha * s_wq[i] * s_wq[j];
          T c[Q];
#pragma unroll
          for (int k = 0; k < Q; ++k) c[k] = wij * cwq<T, N>(k) * pz[k];
          // field order: (j0,d0) I, (j1,d1) I, (j2,d2) D in z
#pragma unroll
          for (int k = 0; k < Q; ++k) v[k] = c[k] * (P.dy * P.dz);
          mv<T, N, MIT, N, Q>(v, o);
          sts<T, N, Q2>(out + 0 * FS, o);
#pragma unroll
          for (int k = 0; k < Q; ++k) v[k] = c[k] * (P.dx * P.dz);
          mv<T, N, MIT, N, Q>(v, o);
          sts<T, N, Q2>(out + 1 * FS, o);
#pragma unroll
          for (int k = 0; k < Q; ++k) v[k] = c[k] * (P.dx * P.dy);
          mv<T, N, MDT, N, Q>(v, o);
          sts<T, N, Q2>(out + 2 * FS, o);
        }
      } else if (l < W1 + W2) {
        const int m = l - W1, sl = m / N, t2 = m - sl * N;
        T x[Q], o[N];
        lds<T, Q, 1>(cs + L::oF3 + sl * N * Q + Q * t2, x);
        mv<T, N, MIT, N, Q>(x, o);
        sts<T, N, 1>(cs + L::oF4 + sl * N2 + N * t2, o);
      } else {
        const int m = l - W1 - W2, qx = m % N, qy = m / N;
        T x[N], rq[N];
        lds<T, N, N2>(cs + L::oR2 + m, x);
        mv<T, N, M_IA, N, N>(x, rq);
        T det = P.dx * P.dy * P.dz;
        if (CURVED) {
          const T *colp = P.col + (long long)ci.col[cl] * col_size(N, Q);
          det *= T(1) - colp[col_off_hqa(N, Q) + m] * P.invH;
        }
        const T wxy = s_wa[qx] * s_wa[qy] * det;
#pragma unroll
        for (int k = 0; k < N; ++k) cs[L::oJI + m + N2 * k] = T(1) / (rq[k] * wxy * cwa<T, N>(k));
      }
    }
  }
  __syncthreads();

  // S4: y test (merging the fields that share the x test)
  {
    constexpr int WC = NG * Q * N, FS = Q2 * N;
    for (int w = threadIdx.x; w < CPB * WC; w += NT) {
      const int cl = w / WC, l = w - cl * WC, cell = cell0 + cl;
      if (cell >= ncell) continue;
      T *cs = sm + cl * PC;
      const int g = l / (Q * N), m = l - g * (Q * N), i = m % Q, c = m / Q;
      const T *in = cs + L::oC3 + i + Q2 * c;
      T x[Q], o[N];
      if (CURVED) {
        // g0 = I C0 (-> D_x), g1 = I C1 (-> I_x), g2 = D C2 + I C3 (-> I_x), g3 = I C4 (-> I_x)
        if (g == 0) {
          lds<T, Q, Q>(in, x);
          mv<T, N, MIT, N, Q>(x, o);
        } else if (g == 1) {
          lds<T, Q, Q>(in + FS, x);
          mv<T, N, MIT, N, Q>(x, o);
        } else if (g == 2) {
          lds<T, Q, Q>(in + 2 * FS, x);
          mv<T, N, MDT, N, Q>(x, o);
          lds<T, Q, Q>(in + 3 * FS, x);
          mv_acc<T, N, MIT, N, Q>(x, o);
        } else {
          lds<T, Q, Q>(in + 4 * FS, x);
          mv<T, N, MIT, N, Q>(x, o);
        }
      } else {
        // g0 = I C0 (-> D_x), g1 = D C1 (-> I_x), g2 = I C2 (-> I_x)
        lds<T, Q, Q>(in + g * FS, x);
        if (g == 1) mv<T, N, MDT, N, Q>(x, o);
        else mv<T, N, MIT, N, Q>(x, o);
      }
      sts<T, N, Q>(cs + L::oD4 + g * Q * N2 + i + Q * N * c, o);
    }
  }
  __syncthreads();

  // S5: x test and the face terms of the line; INV: J^-1 and P_x, else the dual vector out
  {
    constexpr int WC = 3 * N2, GS = Q * N2;
    for (int w = threadIdx.x; w < CPB * WC; w += NT) {
      const int cl = w / WC, l = w - cl * WC, cell = cell0 + cl;
      if (cell >= ncell) continue;
      T *cs = sm + cl * PC;
      const int d = l / N2, m = l - d * N2, b = m % N, c = m / N;  // (b, c): nodes, or fast points with INV
      const T *in = cs + L::oD4 + Q * m;
      T x[Q], X[N];
      if (CURVED) {
        if (d == 0) {
          lds<T, Q, 1>(in, x);
          mv<T, N, MDT, N, Q>(x, X);
          lds<T, Q, 1>(in + GS, x);
          mv_acc<T, N, MIT, N, Q>(x, X);
        } else {
          lds<T, Q, 1>(in + (d + 1) * GS, x);
          mv<T, N, MIT, N, Q>(x, X);
        }
      } else {
        lds<T, Q, 1>(in + d * GS, x);
        if (d == 0) mv<T, N, MDT, N, Q>(x, X);
        else mv<T, N, MIT, N, Q>(x, X);
      }
      const T *F4 = cs + L::oF4;
      const int s0 = CURVED ? 4 + d : 4, s1 = CURVED ? 7 + d : 5;  // z-face slots of component d
      if (!INV) {  // face terms at the face nodes
        if (d == 0) {  // x faces (t1 = y, t2 = z)
          X[0] += F4[0 * N2 + b + N * c];
          X[N - 1] += F4[1 * N2 + b + N * c];
        }
        if (d == 1) {  // y faces (t1 = x, t2 = z)
          if (b == 0) {
#pragma unroll
            for (int a = 0; a < N; ++a) X[a] += F4[2 * N2 + a + N * c];
          }
          if (b == N - 1) {
#pragma unroll
            for (int a = 0; a < N; ++a) X[a] += F4[3 * N2 + a + N * c];
          }
        }
        if (CURVED || d == 2) {  // z faces (t1 = x, t2 = y)
          if (c == 0) {
#pragma unroll
            for (int a = 0; a < N; ++a) X[a] += F4[s0 * N2 + a + N * b];
          }
          if (c == N - 1) {
#pragma unroll
            for (int a = 0; a < N; ++a) X[a] += F4[s1 * N2 + a + N * b];
          }
        }
        sts<T, N, 1>(V + d * Ntot + (long long)cell * N3 + N * m, X);
      } else {  // face terms spread along the normal with P^T[q][e]; then J^-1 and P_x
        if (d == 0) {
          const T f0 = F4[0 * N2 + m], f1 = F4[1 * N2 + m];
#pragma unroll
          for (int a = 0; a < N; ++a) X[a] += s_pte[0][a] * f0 + s_pte[1][a] * f1;
        }
        if (d == 1) {
          const T e0 = s_pte[0][b], e1 = s_pte[1][b];
#pragma unroll
          for (int a = 0; a < N; ++a) X[a] += e0 * F4[2 * N2 + a + N * c] + e1 * F4[3 * N2 + a + N * c];
        }
        if (CURVED || d == 2) {
          const T e0 = s_pte[0][c], e1 = s_pte[1][c];
#pragma unroll
          for (int a = 0; a < N; ++a) X[a] += e0 * F4[s0 * N2 + a + N * b] + e1 * F4[s1 * N2 + a + N * b];
        }
        const T *ji = cs + L::oJI + N * m;
#pragma unroll
        for (int a = 0; a < N; ++a) X[a] *= ji[a];
        T y[N];
        mv<T, N, M_P, N, N>(X, y);
        sts<T, N, 1>(cs + L::oX5 + d * N3 + N * m, y);
      }
    }
  }
  if (!INV) return;
  __syncthreads();

  // S6: P_y
  {
    constexpr int WC = 3 * N2;
    for (int w = threadIdx.x; w < CPB * WC; w += NT) {
      const int cl = w / WC, l = w - cl * WC, cell = cell0 + cl;
      if (cell >= ncell) continue;
      T *cs = sm + cl * PC;
      const int d = l / N2, m = l - d * N2, a = m % N, c = m / N;
      T x[N], y[N];
      lds<T, N, N>(cs + L::oX5 + d * N3 + a + N2 * c, x);
      mv<T, N, M_P, N, N>(x, y);
      sts<T, N, N>(cs + L::oY6 + d * N3 + a + N2 * c, y);
    }
  }
  __syncthreads();

  // S7: P_z, written to V
  {
    constexpr int WC = 3 * N2;
    for (int w = threadIdx.x; w < CPB * WC; w += NT) {
      const int cl = w / WC, l = w - cl * WC, cell = cell0 + cl;
      if (cell >= ncell) continue;
      T *cs = sm + cl * PC;
      const int d = l / N2, m = l - d * N2;
      T x[N], y[N];
      lds<T, N, N2>(cs + L::oY6 + d * N3 + m, x);
      mv<T, N, M_P, N, N>(x, y);
      sts<T, N, N2>(V + d * Ntot + (long long)cell * N3 + m, y);
    }
  }
}

// ------------------------------------------------------------------ kf_div
// Per-cell plan: lo: S1 A1 (x-interp of NFI fields), F2 (face slots, t1-interp)
//                    S3 F4 (faces tested back), C3 (z pass output, 3 fields)
//                hi: S2 B2 (y-interp), F3 (faces, t2 pass)   S4 D4 (y test, 2 fields)
template <int N, bool CURVED, bool KQ>
struct FDivL {
  static constexpr int Q = 2 * N - 1, N2 = N * N, N3 = N2 * N, Q2 = Q * Q;
  static constexpr int NFI = KQ ? 4 : 5;        // V0, V1, V2, [p_k,] p
  static constexpr int NSL = CURVED ? 32 : 24;  // face trace slots
  static constexpr int oA1 = 0, oF2 = NFI * Q * N2;
  static constexpr int oF4 = 0, oC3 = 6 * N2;
  static constexpr int LO = fmax2(oF2 + NSL * Q * N, oC3 + 3 * Q2 * N);
  static constexpr int oB2 = LO, oF3 = LO + NFI * Q2 * N, oD4 = LO;
  static constexpr int HI = fmax2(NFI * Q2 * N + 6 * N * Q, 2 * Q * N2);
  static constexpr int per_cell = (LO + HI + 3) & ~3;
};

template <typename T, int N, bool CURVED, bool KQ, int CPB, int NT>
__device__ __forceinline__ void kf_div_body(const OpP<T> &P, const store_t<T> *__restrict__ V,
                                            const store_t<T> *__restrict__ p, const store_t<T> *__restrict__ pk,
                                            store_t<T> *__restrict__ y, long long Ntot, int ncell,
                                            const store_t<T> *__restrict__ kq, int cell0) {
  using L = FDivL<N, CURVED, KQ>;
  constexpr int Q = L::Q, N2 = L::N2, N3 = L::N3, Q2 = L::Q2, NFI = L::NFI, NSL = L::NSL, PC = L::per_cell;
  constexpr int IP = KQ ? 3 : 4;  // field index of p (p_k is field 3 without KQ)
  extern __shared__ __align__(16) unsigned char smraw[];
  T *sm = reinterpret_cast<T *>(smraw);
  __shared__ CellInfo<CPB> ci;
  __shared__ T s_wq[Q];
  cell_info<T, N, CPB, NT>(P, cell0, ncell, ci);
  for (int t = threadIdx.x; t < Q; t += NT) s_wq[t] = cwq<T, N>(t);
  __syncthreads();

  // S1: x-interpolation of the cell's fields; face traces interpolated along t1
  {
    constexpr int W1 = NFI * N2, W2 = NSL * N, WC = W1 + W2;
    for (int w = threadIdx.x; w < CPB * WC; w += NT) {
      // heavy face lines first, so that the last round holds light lines
      const int cl = w / WC, cell = cell0 + cl;
      int l = w - cl * WC + (W1);
      if (l >= WC) l -= WC;
      if (cell >= ncell) continue;
      T *cs = sm + cl * PC;
      if (l < W1) {
        const int f = l / N2, m = l - f * N2;
        const long long off = (long long)cell * N3 + N * m;
        const store_t<T> *src = f < 3 ? V + f * Ntot + off : (f == IP ? p + off : pk + off);
        T x[N], o[Q];
        lds<T, N, 1>(src, x);
        mv<T, N, M_I, Q, N>(x, o);
        sts<T, Q, 1>(cs + L::oA1 + f * Q * N2 + Q * m, o);
      } else {
        const int m = l - W1, sl = m / N, t2 = m - sl * N;
        int f, side, field;
        div_slot<CURVED>(sl, f, side, field);
        const int k = f >> 1, s = f & 1, nb = ci.nb[cl][f];
        T x[N], o[Q];
        if (side == 0 || nb < 0) {
          const bool wall = nb == -2 || (nb < 0 && (k == 2 || P.bc_lat == 0));
#pragma unroll
          for (int t1 = 0; t1 < N; ++t1) {
            const long long node = (long long)cell * N3 + face_node<N>(k, s ? N - 1 : 0, t1, t2);
            const T v = field == 0 ? P.gfac * pk[node] : V[(field - 1) * Ntot + node];
            x[t1] = wall ? T(0) : v;
          }
        } else {
#pragma unroll
          for (int t1 = 0; t1 < N; ++t1) {
            const long long node = (long long)nb * N3 + face_node<N>(k, s ? 0 : N - 1, t1, t2);
            x[t1] = field == 0 ? P.gfac * pk[node] : V[(field - 1) * Ntot + node];
          }
        }
        mv<T, N, M_I, Q, N>(x, o);
        sts<T, Q, 1>(cs + L::oF2 + sl * Q * N + Q * t2, o);
      }
    }
  }
  __syncthreads();

  // S2: y-interpolation; faces: t2 interpolation, central flux, weights, t2 test
  {
    constexpr int W1 = NFI * Q * N, W2 = 6 * Q, WC = W1 + W2;
    for (int w = threadIdx.x; w < CPB * WC; w += NT) {
      // heavy face lines first, so that the last round holds light lines
      const int cl = w / WC, cell = cell0 + cl;
      int l = w - cl * WC + (W1);
      if (l >= WC) l -= WC;
      if (cell >= ncell) continue;
      T *cs = sm + cl * PC;
      if (l < W1) {
        const int f = l / (Q * N), m = l - f * (Q * N), i = m % Q, c = m / Q;
        T x[N], o[Q];
        lds<T, N, Q>(cs + L::oA1 + f * Q * N2 + i + Q * N * c, x);
        mv<T, N, M_I, Q, N>(x, o);
        sts<T, Q, Q>(cs + L::oB2 + f * Q2 * N + i + Q2 * c, o);
      } else {
        const int m = l - W1, f = m / Q, i = m - f * Q, k = f >> 1;
        const T *colp = CURVED ? P.col + (long long)ci.col[cl] * col_size(N, Q) : nullptr;
        const T zeta0 = T(ci.cz[cl]) * P.dz;
        const T *S = cs + L::oF2 + div_slot_base<CURVED>(f) * Q * N + i;
        T x[N], a[Q], b[Q], fl[Q];
        if (f < 4 || !CURVED) {
          // slots: kappa-, V_k-, kappa+, V_k+ ; flux = nA_k (kappa- V- + kappa+ V+) / 2,
          // nA_k constant along the line
          lds<T, N, Q>(S, x);
          mv<T, N, M_I, Q, N>(x, a);
          lds<T, N, Q>(S + Q * N, x);
          mv<T, N, M_I, Q, N>(x, b);
#pragma unroll
          for (int j = 0; j < Q; ++j) fl[j] = a[j] * b[j];
          lds<T, N, Q>(S + 2 * Q * N, x);
          mv<T, N, M_I, Q, N>(x, a);
          lds<T, N, Q>(S + 3 * Q * N, x);
          mv<T, N, M_I, Q, N>(x, b);
          const T hk = T(0.5) * fnormal<T, N, CURVED>(P, colp, zeta0, f, i, 0, k);
#pragma unroll
          for (int j = 0; j < Q; ++j) fl[j] = hk * (fl[j] + a[j] * b[j]);
        } else {
          // slots: kappa-, Vx-, Vy-, Vz-, kappa+, Vx+, Vy+, Vz+ ; flux = (kappa- V-.nA + kappa+ V+.nA) / 2
          const int s1 = f & 1;
          const T sg = s1 ? T(1) : T(-1);
          const T fac = T(1) - (zeta0 + T(s1) * P.dz) * P.invH;
          const T c0 = -sg * P.dy * fac, c1 = -sg * P.dx * fac, n2 = sg * P.dx * P.dy;
          T n0[Q], n1[Q];
#pragma unroll
          for (int j = 0; j < Q; ++j) {
            n0[j] = c0 * colp[col_off_h1q(N, Q) + i + Q * j];
            n1[j] = c1 * colp[col_off_h2q(N, Q) + i + Q * j];
            fl[j] = T(0);
          }
#pragma unroll
          for (int sd = 0; sd < 2; ++sd) {
            T vn[Q];
            lds<T, N, Q>(S + (4 * sd + 1) * Q * N, x);
            mv<T, N, M_I, Q, N>(x, b);
#pragma unroll
            for (int j = 0; j < Q; ++j) vn[j] = b[j] * n0[j];
            lds<T, N, Q>(S + (4 * sd + 2) * Q * N, x);
            mv<T, N, M_I, Q, N>(x, b);
#pragma unroll
            for (int j = 0; j < Q; ++j) vn[j] += b[j] * n1[j];
            lds<T, N, Q>(S + (4 * sd + 3) * Q * N, x);
            mv<T, N, M_I, Q, N>(x, b);
#pragma unroll
            for (int j = 0; j < Q; ++j) vn[j] += b[j] * n2;
            lds<T, N, Q>(S + 4 * sd * Q * N, x);
            mv<T, N, M_I, Q, N>(x, a);  // kappa
#pragma unroll
            for (int j = 0; j < Q; ++j) fl[j] += a[j] * vn[j];
          }
#pragma unroll
          for (int j = 0; j < Q; ++j) fl[j] *= T(0.5);
        }
        const T wi = -P.alpha * s_wq[i];
#pragma unroll
        for (int j = 0; j < Q; ++j) fl[j] *= wi * cwq<T, N>(j);
        T o[N];
        mv<T, N, M_IT, N, Q>(fl, o);
        sts<T, N, Q>(cs + L::oF3 + f * N * Q + i, o);
      }
    }
  }
  __syncthreads();

  // S3: z pass (interpolate, enthalpy flux and mass at the Gauss points, z test); faces along t1
  {
    constexpr int W1 = Q2, W2 = 6 * N, WC = W1 + W2, FS = Q2 * N;
    for (int w = threadIdx.x; w < CPB * WC; w += NT) {
      const int cl = w / WC, l = w - cl * WC, cell = cell0 + cl;
      if (cell >= ncell) continue;
      T *cs = sm + cl * PC;
      if (l < W1) {
        const int i = l % Q, j = l / Q;
        const T *in = cs + L::oB2 + i + Q * j;
        T x[N], v[Q], cq[Q], acc[Q], o[N], o2[N];
        if (KQ) {
#pragma unroll
          for (int k = 0; k < Q; ++k) cq[k] = kq[(long long)cell * (Q2 * Q) + l + Q2 * k];
        } else {
          lds<T, N, Q2>(in + 3 * FS, x);
          mv<T, N, M_I, Q, N>(x, cq);
#pragma unroll
          for (int k = 0; k < Q; ++k) cq[k] *= P.alpha * P.gfac;
        }
        T *out = cs + L::oC3 + i + Q * j;
        if (CURVED) {
          const T *colp = P.col + (long long)ci.col[cl] * col_size(N, Q);
          const T wA = colp[col_off_w(N, Q, 0) + l], wB = colp[col_off_w(N, Q, 1) + l],
                  wC = colp[col_off_w(N, Q, 2) + l], wE = colp[col_off_w(N, Q, 3) + l],
                  wF = colp[col_off_w(N, Q, 4) + l], wG = colp[col_off_w(N, Q, 5) + l];
          const T zeta0 = T(ci.cz[cl]) * P.dz;
          T cf[Q];
#pragma unroll
          for (int k = 0; k < Q; ++k) {
            cq[k] *= cwq<T, N>(k);  // ck
            cf[k] = cq[k] * (T(1) - (zeta0 + P.dz * cgq<T, N>(k)) * P.invH);
          }
          lds<T, N, Q2>(in, x);  // V0
          mv<T, N, M_I, Q, N>(x, v);
#pragma unroll
          for (int k = 0; k < Q; ++k) {
            acc[k] = cf[k] * wE * v[k];
            v[k] = cq[k] * wA * v[k];
          }
          mv<T, N, M_IT, N, Q>(v, o);
          sts<T, N, Q2>(out, o);
          lds<T, N, Q2>(in + FS, x);  // V1
          mv<T, N, M_I, Q, N>(x, v);
#pragma unroll
          for (int k = 0; k < Q; ++k) {
            acc[k] += cf[k] * wF * v[k];
            v[k] = cq[k] * wB * v[k];
          }
          mv<T, N, M_IT, N, Q>(v, o);
          sts<T, N, Q2>(out + FS, o);
          lds<T, N, Q2>(in + 2 * FS, x);  // V2
          mv<T, N, M_I, Q, N>(x, v);
#pragma unroll
          for (int k = 0; k < Q; ++k) acc[k] += cq[k] * wC * v[k];
          mv<T, N, M_DT, N, Q>(acc, o2);
          lds<T, N, Q2>(in + IP * FS, x);  // p: internal-energy mass
          mv<T, N, M_I, Q, N>(x, v);
#pragma unroll
          for (int k = 0; k < Q; ++k) v[k] = (cwq<T, N>(k) * P.igm1) * wG * v[k];
          mv_acc<T, N, M_IT, N, Q>(v, o2);
          sts<T, N, Q2>(out + 2 * FS, o2);
        } else {
          const T wij = s_wq[i] * s_wq[j];
#pragma unroll
          for (int k = 0; k < Q; ++k) cq[k] *= wij * cwq<T, N>(k);
          lds<T, N, Q2>(in, x);
          mv<T, N, M_I, Q, N>(x, v);
#pragma unroll
          for (int k = 0; k < Q; ++k) v[k] *= cq[k] * (P.dy * P.dz);
          mv<T, N, M_IT, N, Q>(v, o);
          sts<T, N, Q2>(out, o);
          lds<T, N, Q2>(in + FS, x);
          mv<T, N, M_I, Q, N>(x, v);
#pragma unroll
          for (int k = 0; k < Q; ++k) v[k] *= cq[k] * (P.dx * P.dz);
          mv<T, N, M_IT, N, Q>(v, o);
          sts<T, N, Q2>(out + FS, o);
          lds<T, N, Q2>(in + 2 * FS, x);
          mv<T, N, M_I, Q, N>(x, v);
#pragma unroll
          for (int k = 0; k < Q; ++k) v[k] *= cq[k] * (P.dx * P.dy);
          mv<T, N, M_DT, N, Q>(v, o2);
          lds<T, N, Q2>(in + IP * FS, x);
          mv<T, N, M_I, Q, N>(x, v);
          const T wm = wij * P.dx * P.dy * P.dz * P.igm1;
#pragma unroll
          for (int k = 0; k < Q; ++k) v[k] *= wm * cwq<T, N>(k);
          mv_acc<T, N, M_IT, N, Q>(v, o2);
          sts<T, N, Q2>(out + 2 * FS, o2);
        }
      } else {
        const int m = l - W1, f = m / N, t2 = m - f * N;
        T x[Q], o[N];
        lds<T, Q, 1>(cs + L::oF3 + f * N * Q + Q * t2, x);
        mv<T, N, M_IT, N, Q>(x, o);
        sts<T, N, 1>(cs + L::oF4 + f * N2 + N * t2, o);
      }
    }
  }
  __syncthreads();

  // S4: y test: g0 = I C0 (-> D_x), g1 = D C1 + I C2 (-> I_x)
  {
    constexpr int WC = 2 * Q * N, FS = Q2 * N;
    for (int w = threadIdx.x; w < CPB * WC; w += NT) {
      const int cl = w / WC, l = w - cl * WC, cell = cell0 + cl;
      if (cell >= ncell) continue;
      T *cs = sm + cl * PC;
      const int g = l / (Q * N), m = l - g * (Q * N), i = m % Q, c = m / Q;
      const T *in = cs + L::oC3 + i + Q2 * c;
      T x[Q], o[N];
      if (g == 0) {
        lds<T, Q, Q>(in, x);
        mv<T, N, M_IT, N, Q>(x, o);
      } else {
        lds<T, Q, Q>(in + FS, x);
        mv<T, N, M_DT, N, Q>(x, o);
        lds<T, Q, Q>(in + 2 * FS, x);
        mv_acc<T, N, M_IT, N, Q>(x, o);
      }
      sts<T, N, Q>(cs + L::oD4 + g * Q * N2 + i + Q * N * c, o);
    }
  }
  __syncthreads();

  // S5: x test and the face terms of the lines' nodes, written to y
  {
    constexpr int WC = N2, GS = Q * N2;
    for (int w = threadIdx.x; w < CPB * WC; w += NT) {
      const int cl = w / WC, m = w - cl * WC, cell = cell0 + cl;
      if (cell >= ncell) continue;
      const T *cs = sm + cl * PC;
      const int b = m % N, c = m / N;
      T x[Q], Y[N];
      lds<T, Q, 1>(cs + L::oD4 + Q * m, x);
      mv<T, N, M_DT, N, Q>(x, Y);
      lds<T, Q, 1>(cs + L::oD4 + GS + Q * m, x);
      mv_acc<T, N, M_IT, N, Q>(x, Y);
      const T *F4 = cs + L::oF4;
      Y[0] += F4[0 * N2 + b + N * c];
      Y[N - 1] += F4[1 * N2 + b + N * c];
      if (b == 0) {
#pragma unroll
        for (int a = 0; a < N; ++a) Y[a] += F4[2 * N2 + a + N * c];
      }
      if (b == N - 1) {
#pragma unroll
        for (int a = 0; a < N; ++a) Y[a] += F4[3 * N2 + a + N * c];
      }
      if (c == 0) {
#pragma unroll
        for (int a = 0; a < N; ++a) Y[a] += F4[4 * N2 + a + N * b];
      }
      if (c == N - 1) {
#pragma unroll
        for (int a = 0; a < N; ++a) Y[a] += F4[5 * N2 + a + N * b];
      }
      sts<T, N, 1>(y + (long long)cell * N3 + N * m, Y);
    }
  }
}

template <typename T, int N, bool CURVED, bool INV, int CPB, int NT>
__global__ void __launch_bounds__(NT, fused_min_blocks<T, N, NT>())
    kf_grad(const OpP<T> P, const store_t<T> *__restrict__ p, const store_t<T> *__restrict__ rho,
            store_t<T> *__restrict__ V, long long Ntot, int ncell) {
  kf_grad_body<T, N, CURVED, INV, CPB, NT>(P, p, rho, V, Ntot, ncell, blockIdx.x * CPB);
}

template <typename T, int N, bool CURVED, bool KQ, int CPB, int NT>
__global__ void __launch_bounds__(NT, fused_min_blocks<T, N, NT>())
    kf_div(const OpP<T> P, const store_t<T> *__restrict__ V, const store_t<T> *__restrict__ p,
           const store_t<T> *__restrict__ pk, store_t<T> *__restrict__ y, long long Ntot, int ncell,
           const store_t<T> *__restrict__ kq) {
  kf_div_body<T, N, CURVED, KQ, CPB, NT>(P, V, p, pk, y, Ntot, ncell, kq, blockIdx.x * CPB);
}

// Several meshes of one degree in one launch (ensembles): member m owns CTAs
// cta_off[m] .. cta_off[m+1] - 1, CPB of its cells each; vectors are the
// members' DoF blocks concatenated (member m starts at dof_off).
template <typename T>
__device__ __forceinline__ int member_of_cta(const int *cta_off, int nmem) {
  int m = 0;
  while (m + 1 < nmem && cta_off[m + 1] <= (int)blockIdx.x) ++m;
  return m;
}

template <typename T, int N, bool CURVED, int CPB, int NT>
__global__ void __launch_bounds__(NT, fused_min_blocks<T, N, NT>())
    kf_grad_multi(const EnsMember<T> *__restrict__ mem, int nmem, const int *__restrict__ cta_off,
                  const store_t<T> *__restrict__ p_all) {
  const int m = member_of_cta<T>(cta_off, nmem);
  const EnsMember<T> M = mem[m];
  kf_grad_body<T, N, CURVED, true, CPB, NT>(M.P, p_all + M.dof_off, M.rho, M.V, M.N,
                                            (int)(M.N / (N * N * N)), ((int)blockIdx.x - cta_off[m]) * CPB);
}

template <typename T, int N, bool CURVED, int CPB, int NT>
__global__ void __launch_bounds__(NT, fused_min_blocks<T, N, NT>())
    kf_div_multi(const EnsMember<T> *__restrict__ mem, int nmem, const int *__restrict__ cta_off,
                 const store_t<T> *__restrict__ p_all, store_t<T> *__restrict__ y_all) {
  const int m = member_of_cta<T>(cta_off, nmem);
  const EnsMember<T> M = mem[m];
  kf_div_body<T, N, CURVED, false, CPB, NT>(M.P, M.V, p_all + M.dof_off, M.pk, y_all + M.dof_off, M.N,
                                            (int)(M.N / (N * N * N)), nullptr, ((int)blockIdx.x - cta_off[m]) * CPB);
}

}  // namespace
}  // namespace dgx
