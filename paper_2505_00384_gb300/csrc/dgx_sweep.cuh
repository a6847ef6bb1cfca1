// Sum-factorisation machinery shared by the kernel translation units: the 1D
// matrices in __constant__ memory (one copy per translation unit, uploaded
// per device by upload_const_tables), the even-odd line kernel, the sweep over
// a cell's tensor-product array, cell and face helpers, and the fast inverse
// of the density-weighted mass (arXiv:2505.00384, Sec. 3.3).
#pragma once

#include <cmath>
#include <mutex>
#include <type_traits>
#include <vector>

#include "dgx_common.cuh"

namespace dgx {
namespace {

// ------------------------------------------------------------- 1D matrices
// The 1D matrices of every degree live in __constant__ memory in even-odd
// form.  All of them are centro-symmetric, M[R-1-o][C-1-m] = s M[o][m] with
// s = +1 (interpolation, mass-like) or -1 (derivative): the Gauss and
// Gauss-Lobatto point sets are symmetric about 1/2.  Writing
//   e_m = in[m] + in[C-1-m],  d_m = in[m] - in[C-1-m]   (m < C/2),
//   a_o = sum_m E[o][m] e_m + Mc[o] in[mid],  b_o = sum_m Od[o][m] d_m,
// with E = (M[o][m] + M[o][C-1-m])/2, Od = (M[o][m] - M[o][C-1-m])/2 and Mc the
// middle column (odd C), gives out[o] = a_o + b_o and out[R-1-o] = s (a_o - b_o)
// for o < (R+1)/2: half the multiply-adds of the plain product.  Unrolled with
// compile-time indices, every coefficient is an FMA operand read straight from
// the constant bank (no load instruction).
static __constant__ float c_eo32[kEoTotal];
static __constant__ double c_eo64[kEoTotal];

template <typename T>
__device__ __forceinline__ T ceo(int i);
template <>
__device__ __forceinline__ float ceo<float>(int i) { return c_eo32[i]; }
template <>
__device__ __forceinline__ double ceo<double>(int i) { return c_eo64[i]; }

// One line of length MI (stride ss in `src`) -> MO outputs (stride ds in `dst`).
template <typename T, int NN, int MAT, int MO, int MI>
__device__ __forceinline__ void line_eo(const T *src, int ss, T *dst, int ds) {
  constexpr int HO = (MO + 1) / 2, HI = MI / 2;
  constexpr int base = eo_mat_off(NN, MAT);
  constexpr bool odd_in = (MI & 1) != 0;
  constexpr int par = mat_parity(MAT);
  T e[HI > 0 ? HI : 1], d[HI > 0 ? HI : 1];
#pragma unroll
  for (int m = 0; m < HI; ++m) {
    const T x = src[m * ss], y = src[(MI - 1 - m) * ss];
    e[m] = x + y;
    d[m] = x - y;
  }
  const T c = odd_in ? src[HI * ss] : T(0);
#pragma unroll
  for (int o = 0; o < HO; ++o) {
    T a = odd_in ? ceo<T>(base + 2 * HO * HI + o) * c : T(0);
    T b = T(0);
#pragma unroll
    for (int m = 0; m < HI; ++m) {
      a += ceo<T>(base + o * HI + m) * e[m];
      b += ceo<T>(base + HO * HI + o * HI + m) * d[m];
    }
    dst[o * ds] = a + b;
    if (o != MO - 1 - o) dst[(MO - 1 - o) * ds] = par > 0 ? a - b : b - a;
  }
}

// Double-word line product (compensated dot products; defined with the fused
// kernels' double-word tables in dgx_fused.cuh, which a translation unit that
// sweeps double-words includes).
template <int NN, int MAT, int MO, int MI>
__device__ __forceinline__ void line_dw(const df64 *x, df64 *y);

// One line of a sweep: the even-odd product, or for double-words the line
// gathered into registers and multiplied by line_dw.
template <typename T, int NN, int MAT, int MO, int MI>
__device__ __forceinline__ void line_any(const T *src, int ss, T *dst, int ds) {
  if constexpr (std::is_same<T, df64>::value) {
    df64 x[MI], y[MO];
#pragma unroll
    for (int m = 0; m < MI; ++m) x[m] = src[m * ss];
    line_dw<NN, MAT, MO, MI>(x, y);
#pragma unroll
    for (int o = 0; o < MO; ++o) dst[o * ds] = y[o];
  } else {
    line_eo<T, NN, MAT, MO, MI>(src, ss, dst, ds);
  }
}

// One sum-factorisation sweep along direction DIR of `nf` fields stored back
// to back.  Input field shape (S0, S1, S2), x fastest, with S_DIR == MI; the
// output replaces that extent by MO.  One thread per 1D line; field f uses the
// matrix MAT0 / MAT1 / MAT2 selected by bits 2f..2f+1 of `sel`.  The lines are
// dealt out with the fields grouped by matrix (a permutation packed 4 bits per
// field, nf <= 16), so that the threads of a warp take the same branch except
// at the two group boundaries; each line's arithmetic does not depend on
// which thread computes it.
template <typename T, int NN, int DIR, int MO, int MI, int S0, int S1, int S2, int MAT0, int MAT1, int MAT2>
__device__ __forceinline__ void sweep(int nf, unsigned sel, const T *__restrict__ in, T *__restrict__ out) {
  constexpr int L0 = DIR == 0 ? S1 : S0;  // faster non-DIR extent
  constexpr int L1 = DIR == 2 ? S1 : S2;  // slower non-DIR extent
  constexpr int NL = L0 * L1;
  constexpr int IT = S0 * S1 * S2, OT = IT / MI * MO;
  constexpr int O0 = DIR == 0 ? MO : S0, O1 = DIR == 1 ? MO : S1;
  constexpr int ss = DIR == 0 ? 1 : (DIR == 1 ? S0 : S0 * S1);
  constexpr int ds = DIR == 0 ? 1 : (DIR == 1 ? O0 : O0 * O1);
  const int total = nf * NL;
  unsigned long long perm = 0;  // grouped position g -> field, 4 bits each
  int c0 = nf, c01 = nf;        // ends of the MAT0 and MAT1 groups
  if (sel) {
    int k = 0;
    for (int m = 0; m < 3; ++m) {
      for (int f = 0; f < nf; ++f)
        if (((sel >> (2 * f)) & 3u) == (unsigned)m) perm |= (unsigned long long)f << (4 * k++);
      if (m == 0) c0 = k;
      if (m == 1) c01 = k;
    }
  }
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int g = idx / NL, l = idx - g * NL;
    const int f = sel ? (int)((perm >> (4 * g)) & 15u) : g;
    const int l0 = l % L0, l1 = l / L0;
    int io, oo;
    if (DIR == 0) {
      io = (l1 * S1 + l0) * S0;
      oo = (l1 * O1 + l0) * O0;
    } else if (DIR == 1) {
      io = l0 + S0 * S1 * l1;
      oo = l0 + O0 * O1 * l1;
    } else {
      io = l0 + S0 * l1;
      oo = l0 + O0 * l1;
    }
    const T *src = in + f * IT + io;
    T *dst = out + f * OT + oo;
    if constexpr (MAT0 == MAT1 && MAT1 == MAT2) {  // one matrix: one copy of the line code
      line_any<T, NN, MAT0, MO, MI>(src, ss, dst, ds);
    } else if constexpr (MAT1 == MAT2) {
      if (g < c0) line_any<T, NN, MAT0, MO, MI>(src, ss, dst, ds);
      else line_any<T, NN, MAT1, MO, MI>(src, ss, dst, ds);
    } else {
      if (g < c0) line_any<T, NN, MAT0, MO, MI>(src, ss, dst, ds);
      else if (g < c01) line_any<T, NN, MAT1, MO, MI>(src, ss, dst, ds);
      else line_any<T, NN, MAT2, MO, MI>(src, ss, dst, ds);
    }
  }
}

// Node index of face-local point (t1, t2) on the face normal to direction k at
// layer e (0 or N-1).  Tangential order: x face (xi2, xi3), y face (xi1, xi3),
// z face (xi1, xi2).
template <int N>
__device__ __forceinline__ int face_node(int k, int e, int t1, int t2) {
  return k == 0 ? e + N * (t1 + N * t2) : (k == 1 ? t1 + N * (e + N * t2) : t1 + N * (t2 + N * e));
}

struct CellPos {
  long long cell;
  int cx, cy, cz;
};

template <typename T>
__device__ __forceinline__ CellPos cell_pos(const OpP<T> &P, long long cell) {
  CellPos c;
  c.cell = cell;
  c.cx = (int)(cell % P.nx);
  c.cy = (int)((cell / P.nx) % P.ny);
  c.cz = (int)(cell / ((long long)P.nx * P.ny));
  return c;
}

// Whether patch cell (x, y, z) lies in the patch's hole (dead cells of a
// non-conforming mesh's base patch).
template <typename T>
__device__ __forceinline__ bool in_hole(const OpP<T> &P, int x, int y, int z) {
  return x >= P.hole[0] && x < P.hole[1] && y >= P.hole[2] && y < P.hole[3] && z >= P.hole[4] && z < P.hole[5];
}

// Neighbour across face f = 2k+s, or -1 on the boundary (x and y wrap around
// with periodic lateral boundaries); -2 for a face whose terms this kernel
// skips (a face of a dead cell, a face to a dead cell, a face of the patch box
// that borders the other patch).
template <typename T>
__device__ __forceinline__ long long neighbour(const OpP<T> &P, const CellPos &c, int f) {
  const int k = f >> 1, s = f & 1;
  int x = c.cx, y = c.cy, z = c.cz;
  if (in_hole(P, x, y, z)) return -2;
  if (k == 0) {
    x += s ? 1 : -1;
    if (x < 0 || x >= P.nx) {
      if (P.iface & (1 << f)) return -2;
      if (P.bc_lat != 2) return -1;
      x = (x + P.nx) % P.nx;  // periodic lateral boundaries
    }
  } else if (k == 1) {
    y += s ? 1 : -1;
    if (y < 0 || y >= P.ny) {
      if (P.iface & (1 << f)) return -2;
      if (P.bc_lat != 2) return -1;
      y = (y + P.ny) % P.ny;
    }
  } else {
    z += s ? 1 : -1;
    if (z < 0 || z >= P.nz) return (P.iface & (1 << f)) ? -2 : -1;
  }
  if (in_hole(P, x, y, z)) return -2;
  return x + (long long)P.nx * (y + (long long)P.ny * z);
}

// Face trace slots of the divergence kernels (k_div, kf_div): slot -> (face,
// side, field), field 0 = kappa, 1..3 = V_x, V_y, V_z; x and y faces carry
// (kappa-, V_k-, kappa+, V_k+), curved z faces all three components per side.
template <bool CURVED>
__device__ __forceinline__ void div_slot(int sl, int &f, int &side, int &field) {
  if (sl < 16) {
    f = sl >> 2;
    const int w = sl & 3;  // kappa-, Vk-, kappa+, Vk+
    side = w >> 1;
    field = (w & 1) ? 1 + (f >> 1) : 0;
  } else if (CURVED) {
    f = 4 + ((sl - 16) >> 3);
    const int w = (sl - 16) & 7;  // kappa-, Vx-, Vy-, Vz-, kappa+, Vx+, Vy+, Vz+
    side = w >> 2;
    field = w & 3;
  } else {
    f = 4 + ((sl - 16) >> 2);
    const int w = (sl - 16) & 3;
    side = w >> 1;
    field = (w & 1) ? 3 : 0;
  }
}

template <bool CURVED>
__device__ __forceinline__ int div_slot_base(int f) {
  return f < 4 ? 4 * f : (CURVED ? 16 + 8 * (f - 4) : 16 + 4 * (f - 4));
}

template <typename T, int N, int Q>
__device__ __forceinline__ void load_tables(const T *__restrict__ g, T *s) {
  constexpr int TS = tab_size(N, Q);
  for (int i = threadIdx.x; i < TS; i += blockDim.x) s[i] = g[i];
}

// Outward normal times area element of face f at face Gauss point (i, j)
// (unweighted).  Curved z faces have all three components; x and y faces
// stay planar (normal +-e_x, +-e_y) under the Gal-Chen map.
template <typename T, int N, int Q, bool CURVED>
__device__ __forceinline__ void face_normal(const OpP<T> &P, const T *colp, T zeta0, int f, int i, int j,
                                            T nA[3]) {
  const int k = f >> 1, s = f & 1;
  const T sg = s ? T(1) : T(-1);
  nA[0] = nA[1] = nA[2] = T(0);
  if (k == 0) {
    T z3 = P.dz;
    if (CURVED) z3 = P.dz * (T(1) - colp[col_off_hx(N, Q, s) + i] * P.invH);
    nA[0] = sg * P.dy * z3;
  } else if (k == 1) {
    T z3 = P.dz;
    if (CURVED) z3 = P.dz * (T(1) - colp[col_off_hy(N, Q, s) + i] * P.invH);
    nA[1] = sg * P.dx * z3;
  } else {
    nA[2] = sg * P.dx * P.dy;
    if (CURVED) {
      const T fac = T(1) - (zeta0 + T(s) * P.dz) * P.invH;
      nA[0] = -sg * P.dy * colp[col_off_h1q(N, Q) + i + Q * j] * fac;
      nA[1] = -sg * P.dx * colp[col_off_h2q(N, Q) + i + Q * j] * fac;
    }
  }
}

// In-block fast inverse of the density-weighted mass for nf fields (N^3 each)
// in `a` (result left in `a`); rq = rho at the fast-rule points.
// A^-1 v = P^3 (J^-1 (P^T)^3 v), J_q = rho(x_q) w_q det J(x_q)   (Sec. 3.3).
template <typename T, int N, int Q, bool CURVED>
__device__ __forceinline__ void fast_inverse(const OpP<T> &P, const T *tab, const T *colp, const T *rq, int nf,
                                             T *a, T *b) {
  constexpr int N3 = N * N * N;
  const T *PT = tab + tab_off_PT(N, Q);
  const T *Pm = tab + tab_off_P(N, Q);
  const T *wa = tab + tab_off_wa(N, Q);
  sweep<T, N, 0, N, N, N, N, N, M_PT, M_PT, M_PT>(nf, 0u, a, b);
  __syncthreads();
  sweep<T, N, 1, N, N, N, N, N, M_PT, M_PT, M_PT>(nf, 0u, b, a);
  __syncthreads();
  sweep<T, N, 2, N, N, N, N, N, M_PT, M_PT, M_PT>(nf, 0u, a, b);
  __syncthreads();
  for (int node = threadIdx.x; node < N3; node += blockDim.x) {  // one division per node, all fields
    const int i = node % N, j = (node / N) % N, k = node / (N * N);
    T det = P.dx * P.dy * P.dz;
    if (CURVED) det *= (T(1) - colp[col_off_hqa(N, Q) + i + N * j] * P.invH);
    const T inv = T(1) / (rq[node] * wa[i] * wa[j] * wa[k] * det);
    for (int f = 0; f < nf; ++f) b[f * N3 + node] *= inv;
  }
  __syncthreads();
  sweep<T, N, 0, N, N, N, N, N, M_P, M_P, M_P>(nf, 0u, b, a);
  __syncthreads();
  sweep<T, N, 1, N, N, N, N, N, M_P, M_P, M_P>(nf, 0u, a, b);
  __syncthreads();
  sweep<T, N, 2, N, N, N, N, N, M_P, M_P, M_P>(nf, 0u, b, a);
  __syncthreads();
}

// rho at the fast-rule points: Ia^3 rho.
template <typename T, int N, int Q>
__device__ __forceinline__ void rho_fast(const T *tab, const T *rho, T *t1, T *t2, T *rq) {
  const T *Ia = tab + tab_off_Ia(N, Q);
  sweep<T, N, 0, N, N, N, N, N, M_IA, M_IA, M_IA>(1, 0u, rho, t1);
  __syncthreads();
  sweep<T, N, 1, N, N, N, N, N, M_IA, M_IA, M_IA>(1, 0u, t1, t2);
  __syncthreads();
  sweep<T, N, 2, N, N, N, N, N, M_IA, M_IA, M_IA>(1, 0u, t2, rq);
  __syncthreads();
}


}  // namespace

// Upload the even-odd matrices of all degrees into this translation unit's
// constant tables on the context's device (once per device).
static int upload_const_tables(dgx_ctx *c) {
  static std::mutex mu;
  static bool done[64] = {};
  if (c->device < 0 || c->device >= 64) return set_error(c, DGX_ERR_ARG, "device %d", c->device);
  std::lock_guard<std::mutex> lk(mu);
  if (done[c->device]) return 0;
  std::vector<double> eo(kEoTotal, 0.0);
  for (int r = 1; r <= kMaxDegree; ++r) {
    const int N = r + 1, Q = 2 * r + 1;
    std::vector<double> tab;
    if (!build_table_block(r, tab)) return set_error(c, DGX_ERR_ARG, "table construction failed (r=%d)", r);
    const int off[M_COUNT] = {tab_off_I(N, Q),  tab_off_D(N, Q),  tab_off_IT(N, Q),  tab_off_DT(N, Q),
                              tab_off_Ia(N, Q), tab_off_P(N, Q),  tab_off_PT(N, Q),  tab_off_IIT(N, Q),
                              tab_off_DDT(N, Q), tab_off_IDT(N, Q), tab_off_Ia(N, Q), tab_off_IT(N, Q),
                              tab_off_DT(N, Q)};
    for (int id = 0; id < M_COUNT; ++id) {
      const int R = mat_rows(id, N), C = mat_cols(id, N), HO = (R + 1) / 2, HI = C / 2;
      std::vector<double> Mv(R * C, 0.0);
      if (id == M_IAT) {  // transpose of Ia (forward fast mass: Ia^T J Ia)
        for (int a = 0; a < R; ++a)
          for (int q = 0; q < C; ++q) Mv[a * C + q] = tab[off[id] + q * N + a];
      } else if (id == M_PIT || id == M_PDT) {  // PT [q][a] times IT or DT [a][g]
        for (int q = 0; q < R; ++q)
          for (int g = 0; g < C; ++g) {
            double acc = 0.0;
            for (int a = 0; a < N; ++a) acc += tab[tab_off_PT(N, Q) + q * N + a] * tab[off[id] + a * Q + g];
            Mv[q * C + g] = acc;
          }
      } else {
        for (int k = 0; k < R * C; ++k) Mv[k] = tab[off[id] + k];
      }
      const double *M = Mv.data();
      const double s = mat_parity(id);
      double mx = 0.0, asym = 0.0;
      for (int o = 0; o < R; ++o)
        for (int m = 0; m < C; ++m) {
          mx = std::fmax(mx, std::fabs(M[o * C + m]));
          asym = std::fmax(asym, std::fabs(M[(R - 1 - o) * C + (C - 1 - m)] - s * M[o * C + m]));
        }
      if (asym > 1e-12 * mx)
        return set_error(c, DGX_ERR_ARG, "1D matrix %d of degree %d is not centro-symmetric (%g)", id, r, asym / mx);
      double *dst = &eo[eo_mat_off(N, id)];
      for (int o = 0; o < HO; ++o) {
        for (int m = 0; m < HI; ++m) {
          dst[o * HI + m] = 0.5 * (M[o * C + m] + M[o * C + C - 1 - m]);
          dst[HO * HI + o * HI + m] = 0.5 * (M[o * C + m] - M[o * C + C - 1 - m]);
        }
        if (C & 1) dst[2 * HO * HI + o] = M[o * C + HI];
      }
    }
  }
  std::vector<float> eo32(eo.begin(), eo.end());
  if (int e = check_cuda(c, cudaMemcpyToSymbol(c_eo64, eo.data(), eo.size() * sizeof(double)), "constant tables"))
    return e;
  if (int e = check_cuda(c, cudaMemcpyToSymbol(c_eo32, eo32.data(), eo32.size() * sizeof(float)), "constant tables"))
    return e;
  done[c->device] = true;
  return 0;
}


}  // namespace dgx
