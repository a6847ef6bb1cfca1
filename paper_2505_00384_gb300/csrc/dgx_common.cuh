// Internal declarations of the dgx library (not part of the C ABI).
//
// Discretisation (arXiv:2505.00384, Sec. 2 and 3): nodal DG of degree r on the
// (r+1)^3 Gauss-Lobatto points of each hexahedron; every volume and face
// integral uses the consistent Gauss rule with Q = 2r+1 points per direction
// (Sec. 3.3); the density-weighted velocity mass A is inverted with the
// r+1 point Gauss rule as S^-T J^-1 S^-1 (Sec. 3.3).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dgx.h"
#include "dgx_df64.cuh"

namespace dgx {

constexpr int kMaxDegree = 6;  // r = 1..6, N = r+1 <= 7, Q = 2r+1 <= 13

// ---------------------------------------------------------------- 1D tables
// Layout of the per-degree table block (element type T), N = r+1, Q = 2r+1:
//   I  [Q][N]  l_a(g_q)              D  [Q][N]  l_a'(g_q)
//   IT [N][Q]  transpose of I        DT [N][Q]  transpose of D
//   Ia [N][N]  l_a(ga_q)  (r+1 point Gauss rule of the fast inverse)
//   P  [N][N]  Ia^-1 stored [a][q]   PT [N][N]  its transpose [q][a]
//   IIT[N][Q]  l_a(g_q)^2            DDT[N][Q]  l_a'(g_q)^2     IDT[N][Q] l_a l_a'
//   wq [Q]     Gauss weights on [0,1]   wa [N]  weights of the fast rule
//   gq [Q]     Gauss points on [0,1]
__host__ __device__ constexpr int tab_off_I(int, int) { return 0; }
__host__ __device__ constexpr int tab_off_D(int N, int Q) { return Q * N; }
__host__ __device__ constexpr int tab_off_IT(int N, int Q) { return 2 * Q * N; }
__host__ __device__ constexpr int tab_off_DT(int N, int Q) { return 3 * Q * N; }
__host__ __device__ constexpr int tab_off_Ia(int N, int Q) { return 4 * Q * N; }
__host__ __device__ constexpr int tab_off_P(int N, int Q) { return 4 * Q * N + N * N; }
__host__ __device__ constexpr int tab_off_PT(int N, int Q) { return 4 * Q * N + 2 * N * N; }
__host__ __device__ constexpr int tab_off_IIT(int N, int Q) { return 4 * Q * N + 3 * N * N; }
__host__ __device__ constexpr int tab_off_DDT(int N, int Q) { return 5 * Q * N + 3 * N * N; }
__host__ __device__ constexpr int tab_off_IDT(int N, int Q) { return 6 * Q * N + 3 * N * N; }
__host__ __device__ constexpr int tab_off_wq(int N, int Q) { return 7 * Q * N + 3 * N * N; }
__host__ __device__ constexpr int tab_off_wa(int N, int Q) { return 7 * Q * N + 3 * N * N + Q; }
__host__ __device__ constexpr int tab_off_gq(int N, int Q) { return 7 * Q * N + 3 * N * N + Q + N; }
__host__ __device__ constexpr int tab_size(int N, int Q) { return 7 * Q * N + 3 * N * N + 2 * Q + N; }

// Identifiers of the 1D matrices used by the sum-factorisation sweeps and
// their even-odd (centro-symmetric) storage in constant memory, all degrees
// back to back.  A matrix of R rows and C columns stores E[(R+1)/2][C/2],
// Od[(R+1)/2][C/2] and, for odd C, the middle column Mc[(R+1)/2].
// M_PIT = PT IT and M_PDT = PT DT (N x Q): the test with the basis (or its
// derivative) followed by the fast inverse's first factor, in one product.
enum MatId : int { M_I = 0, M_D, M_IT, M_DT, M_IA, M_P, M_PT, M_IIT, M_DDT, M_IDT, M_IAT, M_PIT, M_PDT, M_COUNT };
__host__ __device__ constexpr int mat_rows(int id, int N) { return (id == M_I || id == M_D) ? 2 * N - 1 : N; }
__host__ __device__ constexpr int mat_cols(int id, int N) {
  return (id == M_I || id == M_D || id == M_IA || id == M_P || id == M_PT || id == M_IAT) ? N : 2 * N - 1;
}
__host__ __device__ constexpr int mat_parity(int id) {
  return (id == M_D || id == M_DT || id == M_IDT || id == M_PDT) ? -1 : 1;
}
__host__ __device__ constexpr int eo_size(int R, int C) { return 2 * ((R + 1) / 2) * (C / 2) + ((C & 1) ? (R + 1) / 2 : 0); }
__host__ __device__ constexpr int eo_deg_size(int N) {
  int s = 0;
  for (int id = 0; id < M_COUNT; ++id) s += eo_size(mat_rows(id, N), mat_cols(id, N));
  return s;
}
__host__ __device__ constexpr int eo_deg_base(int N) {
  int s = 0;
  for (int n = 2; n < N; ++n) s += eo_deg_size(n);
  return s;
}
__host__ __device__ constexpr int eo_mat_off(int N, int id) {
  int s = eo_deg_base(N);
  for (int j = 0; j < id; ++j) s += eo_size(mat_rows(j, N), mat_cols(j, N));
  return s;
}
constexpr int kEoTotal = eo_deg_base(kMaxDegree + 2);

// Per-column terrain table (curved meshes).  For column (cx, cy) the bottom
// height h is interpolated from its values at the column's (r+1)^2 GLL
// nodes; with z = zeta + h (1 - zeta/H) the Jacobian only needs h and its
// reference derivatives h1 = dh/dxi1, h2 = dh/dxi2:
//   hq, h1q, h2q [Q*Q]  at (g_i, g_j), index i + Q j
//   hx0, hx1     [Q]    h at xi1 = 0 / 1 along xi2 = g_j   (x faces)
//   hy0, hy1     [Q]    h at xi2 = 0 / 1 along xi1 = g_i   (y faces)
//   hqa          [N*N]  h at the fast-rule points (ga_i, ga_j)
__host__ __device__ constexpr int col_off_hq(int, int) { return 0; }
__host__ __device__ constexpr int col_off_h1q(int, int Q) { return Q * Q; }
__host__ __device__ constexpr int col_off_h2q(int, int Q) { return 2 * Q * Q; }
__host__ __device__ constexpr int col_off_hx(int, int Q, int s) { return 3 * Q * Q + s * Q; }
__host__ __device__ constexpr int col_off_hy(int, int Q, int s) { return 3 * Q * Q + 2 * Q + s * Q; }
__host__ __device__ constexpr int col_off_hqa(int, int Q) { return 3 * Q * Q + 4 * Q; }
// Weighted metric products of the column at (g_i, g_j), w_ij = wq_i wq_j, e = 1 - h/H:
//   wA = w_ij dy dz e,  wB = w_ij dx dz e,  wC = w_ij dx dy,
//   wE = -w_ij dy h1,   wF = -w_ij dx h2,   wG = w_ij dx dy dz e   [Q*Q each]
// so that at layer point k, with wk = wq_k and wf = wq_k (1 - zeta_k/H), the
// quadrature weight times the five nonzeros of adj(J) are wk wA, wk wB, wk wC,
// wf wE, wf wF and the weight times det J is wk wG.
__host__ __device__ constexpr int col_off_w(int N, int Q, int t) { return 3 * Q * Q + 4 * Q + N * N + t * Q * Q; }
__host__ __device__ constexpr int col_size(int N, int Q) { return 9 * Q * Q + 4 * Q + N * N; }

// Kernel parameters of the pressure operator.
template <typename T>
struct OpP {
  int nx, ny, nz, bc_lat;  // lateral faces: 0 slip wall, 1 far field, 2 periodic
  // non-conforming meshes: the cells of `hole` (x0, x1, y0, y1, z0, z1) are
  // dead and every face that touches them is skipped; a face of this patch's
  // box whose bit (1 << f) is set in `iface` borders the other patch and is
  // skipped too (its terms come from the hanging-face kernels)
  int hole[6];
  int iface, pad_;
  T dx, dy, dz, H;         // cell sizes (dz of the uniform zeta grid) and Lz
  T invH;                  // 1 / Lz (the map's factor 1 - zeta/H without a division per point)
  T alpha;                 // a~_ll * dt
  T gfac;                  // gamma / (gamma - 1)
  T igm1;                  // 1 / (gamma - 1)
  const T *tab;            // 1D tables of this degree
  const T *col;            // per-column terrain tables (nullptr when flat)
};

// One member of a multi-mesh (ensemble) launch: its operator parameters, its
// coefficient copies and V scratch, and its place in the concatenated vectors.
// (T = df64: double-word parameters, FP64 arrays)
template <typename T>
struct EnsMember {
  OpP<T> P;
  const store_t<T> *rho, *pk;
  store_t<T> *V;
  long long cell_off, dof_off, N;
};

// ---------------------------------------------------------------- context
struct Buf {
  void *p = nullptr;
  size_t bytes = 0;
};

struct Learned;    // learned preconditioner state (dgx_learned.cu)
struct Multigrid;  // geometric multigrid hierarchy (dgx_mg.cu)

}  // namespace dgx

struct dgx_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;

  // mesh
  bool has_mesh = false;
  dgx_mesh_desc mesh{};
  int n = 0, q = 0;
  long long ncell = 0, N = 0;
  bool curved = false;
  double *tab64 = nullptr;
  float *tab32 = nullptr;
  double *col64 = nullptr;
  float *col32 = nullptr;
  float *coldf = nullptr;  // the same values as double-words (hi, lo pairs)

  // background
  bool has_bg = false;
  dgx_background bg{};
  double *rho_bar = nullptr, *p_bar = nullptr;

  // coefficients of the current fixed-point iterate
  bool has_coef = false;
  double alpha = 0.0, gamma = 1.4;
  double *rho64 = nullptr, *pk64 = nullptr;
  float *rho32 = nullptr, *pk32 = nullptr;
  double *diag64[3] = {nullptr, nullptr, nullptr};  // index DGX_PC_*: diagonal
  double *dinv64[3] = {nullptr, nullptr, nullptr};  // inverse diagonal
  float *diag32[3] = {nullptr, nullptr, nullptr};
  float *dinv32[3] = {nullptr, nullptr, nullptr};
  bool diag64_ok = false, diag32_ok = false;         // valid for the current coefficients
  // alpha gamma/(gamma-1) p_k at the Q^3 Gauss points (FP64 k_div), with the coefficient version it holds
  double *kq64 = nullptr;
  long long kq64_version = -1;
  bool use_kappa = true;  // ensembles' member contexts (multi-mesh kernels) do without

  // operator scratch: V = A^-1 B p (3N)
  double *V64 = nullptr;
  float *V32 = nullptr;

  // quadrature of the density-weighted mass A(rho) wherever it is applied or
  // inverted: DGX_MASS_FAST (r+1 points, closed-form inverse) or
  // DGX_MASS_CONSISTENT (2r+1 points, inverse by per-cell PCG to mass_tol
  // relative residual, at most mass_maxit iterations; FP32 uses max(mass_tol, 1e-5))
  int mass_rule = DGX_MASS_FAST;
  double mass_tol = 1e-13;
  int mass_maxit = 50;
  int *mass_stats = nullptr;  // device [2]: largest PCG iteration count, unconverged cells

  // non-conforming mesh (mesh.refine box not empty): patch 0 = the nx*ny*nz
  // base cells (those in the box dead), patch 1 = the children block fine[3]
  // from cell ncell0 on; the terrain tables of patch 1 follow patch 0's in
  // col64 / col32 / coldf at column col1_off; hang64 / hang32: the 1D tables
  // of the hanging-face kernels; hcells: their work list (nhcell cells)
  bool nc = false;
  long long ncell0 = 0;
  int fine[3] = {0, 0, 0};
  long long col1_off = 0;
  double zoff = 0.0;      // zeta of the children block's bottom
  double *hn1 = nullptr;  // nodal terrain heights of the children's columns (node coordinates)
  double *hang64 = nullptr;
  float *hang32 = nullptr;
  void *hcells = nullptr;
  int nhcell = 0;

  // launch variant of the operator kernels per precision ([0] FP64, [1] FP32):
  // 0..2 one cell per CTA (k_grad / k_div) with 128 / 192 / 256 threads, 3..4
  // the fused multi-cell kernels in configuration v - 3 (fused_cpb), 5..6 (FP64
  // only) the fused kernels in double-word arithmetic, configuration v - 5; -1 = the
  // default of the degree.  Chosen by the timing autotuner (op_tuned) unless
  // pinned by dgx_set_operator_variant (op_pinned).
  int op_variant[2] = {-1, -1};
  // arithmetic of the explicit fluxes: 1 double-words on the FP32 pipes (degrees
  // up to 4), 0 the FP64 pipe
  int explicit_variant = 1;
  bool op_tuned[2] = {false, false};
  bool op_pinned[2] = {false, false};

  // Krylov workspace (grown on demand)
  double *kry64 = nullptr;
  size_t kry64_elems = 0;
  float *kry32 = nullptr;
  size_t kry32_elems = 0;
  double *red = nullptr;       // reduction partials
  double *red_out = nullptr;   // reduced scalars (device)
  double *host_red = nullptr;  // pinned host mirror
  cudaEvent_t arn_ev = nullptr;  // marks the Arnoldi scalars' copy to host_red
  size_t red_elems = 0;

  // IMEX step: tableaux (s <= 4, row-major), time step, fixed-point iterations
  bool has_imex = false;
  int imex_s = 0, imex_K = 0;
  double imex_A[16] = {}, imex_At[16] = {}, imex_dt = 0.0;
  double *imex_ws = nullptr;
  size_t imex_ws_elems = 0;

  // recorder of the pressure systems solved inside dgx_imex_step
  double *rec_store = nullptr;
  int rec_cap = 0, rec_stride = 1, rec_count = 0, rec_seen = 0;

  // incremented by every dgx_set_coefficients (invalidates derived caches)
  long long coef_version = 0;
  dgx::Learned *learned = nullptr;
  dgx::Multigrid *mg = nullptr;

  std::vector<void *> owned;  // everything cudaMalloc'd for the mesh
};

namespace dgx {

int set_error(dgx_ctx *c, int code, const char *fmt, ...);
// process-wide count of kernel launches made by the library
void count_launch(int n = 1);
long long launch_count();
int check_cuda(dgx_ctx *c, cudaError_t e, const char *what);

// 1D Gauss and Gauss-Lobatto rules on [0, 1] (dgx_api.cu)
void rule_gauss(int q, std::vector<double> &x, std::vector<double> &w);
void rule_gll(int n, std::vector<double> &x, std::vector<double> &w);
// host 1D table block of degree r (layout above), dgx_api.cu
bool build_table_block(int r, std::vector<double> &tab);
// multigrid transfer tables of degree r (dgx_api.cu), GLL nodes x_a on [0, 1]:
//   E[s][a_f][a_c] = l_{a_c}((x_{a_f} + s) / 2)  (coarse basis at child s's nodes)
//   side[a] = 1 if x_a > 1/2 else 0, F[a][i] = l_i(2 x_a - side[a])  (fine basis at coarse node a)
bool child_tables(int r, std::vector<double> &E, std::vector<int> &side, std::vector<double> &F);
// upload the even-odd matrices of all degrees to constant memory of the
// context's device (once per device), dgx_operator.cu
int ensure_const_tables(dgx_ctx *c);

// operator kernels (dgx_operator.cu)
// alpha < 0: use the context's a~_ll dt; inv = false: k_grad writes the dual B p
template <typename T>
int launch_grad(dgx_ctx *c, const T *p, const T *rho, T *V, cudaStream_t s, bool inv = true, double alpha = -1.0);
template <typename T>
int launch_div(dgx_ctx *c, const T *V, const T *p, const T *pk, T *y, cudaStream_t s, double alpha = -1.0);
template <typename T>
int launch_mass_inverse(dgx_ctx *c, const T *in, const T *rho, T *out, cudaStream_t s, int nf = 3);
// consistent (2r+1 point) density-weighted mass of nf fields (dgx_mass.cu):
// inverse = 0: out = A_c(rho) in; inverse = 1: out = A_c(rho)^-1 in by per-cell PCG
template <typename T>
int launch_mass_cons(dgx_ctx *c, const T *in, const T *rho, T *out, cudaStream_t s, int nf, int inverse);
// the context's mass rule: A(rho)^-1 of nf fields, A(rho) v of 3 fields (FP64),
// and V = A(rho)^-1 B p (B scaled by the context's a~_ll dt)
template <typename T>
inline int mass_inverse_rule(dgx_ctx *c, const T *in, const T *rho, T *out, cudaStream_t s, int nf = 3) {
  if (c->mass_rule == DGX_MASS_CONSISTENT) return launch_mass_cons<T>(c, in, rho, out, s, nf, 1);
  return launch_mass_inverse<T>(c, in, rho, out, s, nf);
}
int launch_mass_fwd(dgx_ctx *c, const double *rho, const double *v, double *out, cudaStream_t s);
inline int mass_forward_rule(dgx_ctx *c, const double *rho, const double *v, double *out, cudaStream_t s) {
  if (c->mass_rule == DGX_MASS_CONSISTENT) return launch_mass_cons<double>(c, v, rho, out, s, 3, 0);
  return launch_mass_fwd(c, rho, v, out, s);
}
template <typename T>
inline int grad_inverse_rule(dgx_ctx *c, const T *p, const T *rho, T *V, cudaStream_t s) {
  if (c->mass_rule != DGX_MASS_CONSISTENT) return launch_grad<T>(c, p, rho, V, s);  // fused B and fast A^-1
  if (int e = launch_grad<T>(c, p, rho, V, s, false)) return e;
  return launch_mass_cons<T>(c, V, rho, V, s, 3, 1);  // in place: each cell reads its block first
}
// fused multi-cell operator kernels (dgx_fused.cuh): configuration cfg (0, 1)
// of degree N = r+1 has fused_cpb cells and fused_nt threads per CTA, the
// threads covering the cells' Q x Q Gauss-point columns of the z pass in one
// round (whole warps); fused_grad with inv = false writes the dual vector
// B p; fused_div uses kq (FP64 only) when not null
__host__ __device__ constexpr int fused_cpb(int N, int cfg) { return N <= 3 ? (cfg ? 8 : 4) : (cfg ? 2 : 1); }
__host__ __device__ constexpr int fused_nt(int N, int cfg) {
  return ((fused_cpb(N, cfg) * (2 * N - 1) * (2 * N - 1) + 31) / 32) * 32;
}
constexpr size_t kFusedMaxSmem = 227 * 1024;
// (T = df64: double-word arithmetic on FP64 arrays, store_t<df64> = double)
template <typename T, int N, bool CURVED>
int fused_grad(dgx_ctx *c, const store_t<T> *p, const store_t<T> *rho, store_t<T> *V, cudaStream_t s, bool inv,
               double alpha, int cfg);
template <typename T, int N, bool CURVED>
int fused_div(dgx_ctx *c, const store_t<T> *V, const store_t<T> *p, const store_t<T> *pk, store_t<T> *y,
              cudaStream_t s, double alpha, const store_t<T> *kq, int cfg);
template <typename T, int N, bool CURVED>
size_t fused_smem(int cfg);
// multi-mesh fused operator (FP32, or FP64 arrays in double-words): members' CTA ranges in cta_off (nmem + 1 entries, device)
template <typename T, int N, bool CURVED>
int fused_operator_multi(dgx_ctx *c0, const EnsMember<T> *mem, int nmem, const int *cta_off, int nblocks,
                         const store_t<T> *x, store_t<T> *y, cudaStream_t s, int cfg);
// multi-mesh operator y = S x for members of one degree (N = r+1) and terrain kind;
// `mem` is a device array of nmem members with consecutive cell ranges totalling ncell_total
template <typename T>
int launch_operator_multi(dgx_ctx *c0, int n, bool curved, const EnsMember<T> *mem, int nmem, long long ncell_total,
                          const T *x_all, T *y_all, cudaStream_t s, int threads);
// explicit part of the IMEX step (dgx_explicit.cu), FP64
int launch_explicit(dgx_ctx *c, const double *rho, const double *u, const double *rho_bar, double *Er, double *Em,
                    double *Ee, cudaStream_t s);
// consistent mass of scale*f0 (mode 0) or scale*f0*|fv|^2/2 (mode 1)
int launch_cmass(dgx_ctx *c, int mode, double scale, const double *f0, const double *fv, double *out,
                 cudaStream_t s);
// forward fast density-weighted mass A(rho) v, 3 components
int launch_mass_fwd(dgx_ctx *c, const double *rho, const double *v, double *out, cudaStream_t s);
// kq = alpha gamma/(gamma-1) p_k at the Gauss points of every cell (Q^3 per cell)
template <typename T>
int launch_kappa(dgx_ctx *c, const T *pk, T *kq, cudaStream_t s);
// Helmholtz (dh) and internal-energy (die) diagonals of Sec. 3.1 in precision T
template <typename T>
int launch_diag(dgx_ctx *c, const T *rho, const T *pk, T *dh, T *die, cudaStream_t s);
// Jacobi diagonals of the current coefficients, computed on first use:
// FP64 (diag64, dinv64, and dinv32 rounded from them) or, when only FP32 is
// needed (the mixed solver's inner GMRES), the FP32 diagonal kernel (dinv32).
int ensure_diag(dgx_ctx *c, bool f64);
// kernel parameters of patch `patch` (0, or 1 = the children block of a
// non-conforming mesh)
template <typename T>
OpP<T> make_params(const dgx_ctx *c, int patch = 0);
template <>
OpP<df64> make_params<df64>(const dgx_ctx *c, int patch);
// patches of the mesh: one, or two on non-conforming meshes (the base cells,
// then the children block); first cell and number of cells of each
inline int num_patches(const dgx_ctx *c) { return c->nc ? 2 : 1; }
inline long long patch_cell0(const dgx_ctx *c, int i) { return i ? c->ncell0 : 0; }
inline long long patch_ncell(const dgx_ctx *c, int i) {
  return c->nc ? (i ? c->ncell - c->ncell0 : c->ncell0) : c->ncell;
}
// hanging-face terms of non-conforming meshes (dgx_nonconf.cu), added to what
// the per-patch kernels wrote: V += A^-1 B_h p (inv) or V += B_h p; y -= C_h V;
// explicit tendencies += the hanging faces' flux terms
template <typename T>
int launch_hang_grad(dgx_ctx *c, const T *p, const T *rho, T *V, cudaStream_t s, bool inv, double alpha);
template <typename T>
int launch_hang_div(dgx_ctx *c, const T *V, const T *pk, T *y, cudaStream_t s, double alpha);
int launch_hang_explicit(dgx_ctx *c, const double *rho, const double *u, double *Er, double *Em, double *Ee,
                         cudaStream_t s);
// x[cell * n3 + node] = v (or src at the same index) on the dead cells of a
// non-conforming mesh (nf fields of stride N)
template <typename T>
int fill_dead(dgx_ctx *c, T *x, int nf, double v, cudaStream_t s, const T *src = nullptr);
// mesh set-up of a non-conforming mesh (dgx_nonconf.cu): the hanging-face work
// list and tables (after the patches' cells and tables are known)
int nonconf_setup(dgx_ctx *c);
// operator launch variants (see dgx_ctx::op_variant): count, whether variant v
// fits this context's mesh and precision, and its threads per CTA
constexpr int kOpVariants = 7;
template <typename T>
bool op_variant_ok(const dgx_ctx *c, int v);
int op_variant_threads(const dgx_ctx *c, int v);

// vector kernels (dgx_vector.cu)
template <typename T>
void vec_axpby(long long n, double a, const T *x, double b, T *y, cudaStream_t s);
template <typename T>
void vec_mul(long long n, const T *a, const T *x, T *y, cudaStream_t s);  // y = a .* x
template <typename TO, typename TI>
void vec_convert(long long n, const TI *x, TO *y, cudaStream_t s);
void vec_inv(long long n, const double *d, double *dinv64, float *dinv32, cudaStream_t s);
void vec_inv32(long long n, const float *d, float *dinv, cudaStream_t s);
// h[i] = <V_i, w> for i < nv (V_i = V + i*ld), written to out (device doubles)
template <typename T>
void vec_mdot(long long n, int nv, const T *V, long long ld, const T *w, double *partial, double *out,
              cudaStream_t s);
// w -= sum_i h[i] V_i (h on device); optional: out_norm2 = <w,w> after update
template <typename T>
void vec_mupdate(long long n, int nv, const T *V, long long ld, const double *h, T *w, double *partial,
                 double *out_norm2, cudaStream_t s);
// y = x * (1 / sqrt(*nrm2)) with the scalar read on the device
template <typename T>
void vec_scale_by_inv_sqrt(long long n, const double *nrm2, const T *x, T *y, cudaStream_t s);
// x += sum_i c[i] Z_i (c on host, passed by value array)
template <typename T, typename TX>
void vec_lincomb(long long n, int nv, const T *Z, long long ld, const double *c_dev, TX *x, cudaStream_t s);
template <typename T>
void vec_dot(long long n, const T *a, const T *b, double *partial, double *out, cudaStream_t s);
int vec_partials();  // number of reduction blocks per vector pass

// dgx_solve_pressure that also returns Vx = A^-1 B x (3N) of the solution (dgx_api.cu)
int solve_pressure_vx(dgx_ctx *c, const double *b, double *x, const dgx_solve_opts *opts, dgx_solve_info *info,
                      double *Vx);

// geometric multigrid (dgx_mg.cu): z = one V-cycle applied to b (FP64); release
int mg_vcycle(dgx_ctx *c, const double *b, double *z);
bool mg_ready(const dgx_ctx *c);
void mg_free(dgx_ctx *c);

// learned preconditioner (dgx_learned.cu)
void learned_free(dgx_ctx *c);          // release everything (dgx_destroy)
void learned_mesh_changed(dgx_ctx *c);  // drop mesh-dependent buffers and samples (keeps the weights)
bool learned_ready(const dgx_ctx *c);
// z = M(v): Helmholtz Jacobi guess plus the network's correction, current coefficients
template <typename T>
int learned_apply(dgx_ctx *c, const T *v, T *z);
// host: terrain height h(x, y) at every DoF of the mesh (dgx_api.cu)
void node_terrain_heights(const dgx_ctx *c, std::vector<double> &h);

}  // namespace dgx
