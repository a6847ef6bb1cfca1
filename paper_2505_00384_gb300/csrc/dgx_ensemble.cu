// Batched ensemble of pressure solves: several independent meshes (different
// sizes, degrees and terrain), one Schur system S_m p_m = b_m each
// (arXiv:2505.00384, Sec. 2 fixed-point form; Sec. 3.1 Krylov + Helmholtz
// Jacobi), solved together.
//
// Design: one dgx_ctx per member holds its mesh tables, coefficients and
// diagonals; the ensemble owns concatenated vectors (member m at dof_off[m]).
// The operator of all members of one degree runs as one kernel pair
// (k_grad_multi / k_div_multi over the members' cells).  The solver is FP64
// iterative refinement around an FP32 GMRES(m) cycle for all members at once,
// with per-member Hessenberg matrices and Givens rotations kept on the
// device.  The whole solve is one CUDA graph, launched once: a prologue forms
// ||b_m||, the FP64 residual b - S x of every member and its norm, and a check
// kernel that freezes converged members and sets the condition of a WHILE
// conditional node; its body runs one inner cycle, adds the correction, forms
// the new residuals and runs the check again.  The loop ends when every member
// has converged, a residual is not finite, or maxit cycles have run (a bound
// counted on the device); the host reads the per-member results once at the
// end.  Threads per CTA of the multi-mesh operator are chosen per degree group
// by a small timing autotuner before the graph is captured.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "dgx_common.cuh"

using namespace dgx;

namespace {

constexpr int kMaxMembers = 64;
constexpr int kMaxRestart = 64;
constexpr int kSegBlocks = 48;  // CTAs per member in segmented vector kernels
constexpr int kT = 256;

struct Group {
  int n = 0;
  bool curved = false;
  std::vector<int> idx;  // members of this group
  long long ncell = 0;
  EnsMember<double> *d64 = nullptr;
  EnsMember<float> *d32 = nullptr;
  int threads64 = 256, threads32 = 256;
  // FP32 tile shape: -1 = one cell per CTA (k_grad_multi / k_div_multi, threads32),
  // 0 / 1 = the fused kernels in configuration tile32 (fused_cpb cells, fused_nt threads)
  int tile32 = -1;
  // FP64 tile shape: -1 = one cell per CTA (threads64), 0 / 1 = the fused kernels in
  // double-word arithmetic in configuration tile64
  int tile64 = -1;
  EnsMember<df64> *ddf = nullptr;        // member tables for the double-word kernels
  int *cta_off[2] = {nullptr, nullptr};  // per fused configuration: members' first CTA (device)
  int nblocks[2] = {0, 0};
  bool fits32[2] = {false, false}, fits64[2] = {false, false};
};

}  // namespace

struct dgx_ensemble {
  int device = 0;
  cudaStream_t stream = nullptr;       // the ensemble's own non-blocking stream (capturable)
  cudaStream_t user_stream = nullptr;  // the caller's stream, ordered with `stream` by events
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::string err;
  int nm = 0;
  std::vector<dgx_ctx *> mem;
  std::vector<long long> N, off;
  long long Ntot = 0;
  std::vector<Group> groups;
  bool has_coef = false;
  bool tuned = false;
  // concatenated vectors
  double *r64 = nullptr, *t64 = nullptr;
  float *r32 = nullptr, *d32 = nullptr, *w32 = nullptr, *u32 = nullptr, *dinv32 = nullptr, *V32 = nullptr;
  int vm = 0;  // restart length the basis was sized for
  // per-member device scalars
  double *bn = nullptr;       // ||b_m||
  double *part = nullptr;     // [member][block][k] partial sums
  double *h1 = nullptr, *h2 = nullptr, *nrm = nullptr;  // [member][kMaxRestart+1]
  double *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr, *scl = nullptr, *beta0 = nullptr;
  int *jj = nullptr, *act = nullptr;
  double *host = nullptr;  // pinned mirror of per-member scalars
  long long *seg_off = nullptr, *seg_len = nullptr;
  // graph of one whole solve (refinement loop in a WHILE conditional node) and
  // the arguments it was captured with
  cudaGraphExec_t gexec = nullptr;
  const double *graph_b = nullptr;
  double *graph_x = nullptr;
  int graph_m = 0, graph_maxit = 0, graph_x0 = 0;
  double graph_tol = 0.0, graph_itol = 0.0;
  long long graph_pro_launches = 0, graph_body_launches = 0;
  // per-member results of a solve on the device: relative residual, cycles;
  // ctl[0] = cycles run, ctl[1] = 1 after a non-finite residual
  double *relres_d = nullptr;
  int *its_d = nullptr, *ctl_d = nullptr;
  std::vector<void *> owned;
};

namespace {

// Order the ensemble's stream after the caller's work, and the caller's stream after ours.
void enter(dgx_ensemble *e) {
  cudaEventRecord(e->ev_in, e->user_stream);
  cudaStreamWaitEvent(e->stream, e->ev_in, 0);
}
void leave(dgx_ensemble *e) {
  cudaEventRecord(e->ev_out, e->stream);
  cudaStreamWaitEvent(e->user_stream, e->ev_out, 0);
}

int eset(dgx_ensemble *e, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  e->err = buf;
  return code;
}

int echeck(dgx_ensemble *e, cudaError_t r, const char *what) {
  if (r == cudaSuccess) return 0;
  return eset(e, r == cudaErrorMemoryAllocation ? DGX_ERR_OOM : DGX_ERR_CUDA, "%s: %s", what, cudaGetErrorString(r));
}

template <typename T>
int ealloc(dgx_ensemble *e, T **p, size_t elems) {
  void *q = nullptr;
  if (int r = echeck(e, cudaMalloc(&q, std::max<size_t>(elems, 1) * sizeof(T)), "cudaMalloc")) return r;
  e->owned.push_back(q);
  *p = reinterpret_cast<T *>(q);
  return 0;
}

// ---------------------------------------------------------------- segmented vector kernels
// grid (kSegBlocks, nm): blockIdx.y = member, grid-stride over that member's segment.
__device__ __forceinline__ double bsum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  return t;
}

// part[m][b][i0 + c] = sum over block b's share of member m of V_{i0+c} . w
template <typename T>
__global__ void __launch_bounds__(kT) k_seg_mdot(const long long *off, const long long *len, int i0, int cnt,
                                                 const T *__restrict__ V, long long ld, const T *__restrict__ w,
                                                 double *__restrict__ part) {
  __shared__ double sh[32];
  const int m = blockIdx.y;
  const long long o = off[m], n = len[m];
  float acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = 0.f;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
  long long done = 0;
  if constexpr (sizeof(T) == 4) {
    // 16-byte loads when the member's segment starts on a 16-byte boundary
    if (((o | ld) & 3) == 0) {
      const long long n4 = n / 4;
      const float4 *w4 = reinterpret_cast<const float4 *>(w + o);
      for (long long i = tid; i < n4; i += stride) {
        const float4 wi = w4[i];
#pragma unroll
        for (int c = 0; c < 8; ++c)
          if (c < cnt) {
            const float4 a = reinterpret_cast<const float4 *>(V + (long long)(i0 + c) * ld + o)[i];
            acc[c] += a.x * wi.x + a.y * wi.y + a.z * wi.z + a.w * wi.w;
          }
      }
      done = n4 * 4;
    }
  }
  for (long long i = done + tid; i < n; i += stride) {
    const float wi = (float)w[o + i];
#pragma unroll
    for (int c = 0; c < 8; ++c)
      if (c < cnt) acc[c] += (float)V[(long long)(i0 + c) * ld + o + i] * wi;
  }
  for (int c = 0; c < cnt; ++c) {
    const double t = bsum((double)acc[c], sh);
    if (threadIdx.x == 0) part[((long long)m * kSegBlocks + blockIdx.x) * (kMaxRestart + 1) + i0 + c] = t;
  }
}

// out[m][i] = sum_b part[m][b][i], grid (nv, nm)
__global__ void k_seg_reduce(const double *__restrict__ part, double *__restrict__ out) {
  __shared__ double sh[32];
  const int m = blockIdx.y, i = blockIdx.x;
  double a = 0.0;
  for (int b = threadIdx.x; b < kSegBlocks; b += blockDim.x)
    a += part[((long long)m * kSegBlocks + b) * (kMaxRestart + 1) + i];
  const double t = bsum(a, sh);
  if (threadIdx.x == 0) out[m * (kMaxRestart + 1) + i] = t;
}

// w_m -= sum_k h[m][k] V_k (member m's segment); part[m][b][0] = partial |w_m|^2 when norm != 0
__global__ void __launch_bounds__(kT) k_seg_mupdate(const long long *off, const long long *len, int nv,
                                                    const float *__restrict__ V, long long ld,
                                                    const double *__restrict__ h, float *__restrict__ w,
                                                    double *__restrict__ part, int norm) {
  __shared__ double sh[32];
  __shared__ float hs[kMaxRestart + 1];
  const int m = blockIdx.y;
  for (int k = threadIdx.x; k < nv; k += blockDim.x) hs[k] = (float)h[m * (kMaxRestart + 1) + k];
  __syncthreads();
  const long long o = off[m], n = len[m];
  float acc = 0.f;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
  long long done = 0;
  if (((o | ld) & 3) == 0) {  // 16-byte loads and stores
    const long long n4 = n / 4;
    float4 *w4 = reinterpret_cast<float4 *>(w + o);
    for (long long i = tid; i < n4; i += stride) {
      float4 v = w4[i];
      for (int k = 0; k < nv; ++k) {
        const float4 a = reinterpret_cast<const float4 *>(V + (long long)k * ld + o)[i];
        v.x -= hs[k] * a.x;
        v.y -= hs[k] * a.y;
        v.z -= hs[k] * a.z;
        v.w -= hs[k] * a.w;
      }
      w4[i] = v;
      acc += v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w;
    }
    done = n4 * 4;
  }
  for (long long i = done + tid; i < n; i += stride) {
    float v = w[o + i];
    for (int k = 0; k < nv; ++k) v -= hs[k] * V[(long long)k * ld + o + i];
    w[o + i] = v;
    acc += v * v;
  }
  if (norm) {
    const double t = bsum((double)acc, sh);
    if (threadIdx.x == 0) part[((long long)m * kSegBlocks + blockIdx.x) * (kMaxRestart + 1)] = t;
  }
}

// y_m = x_m * s[m]
template <typename TX, typename TY>
__global__ void __launch_bounds__(kT) k_seg_scale(const long long *off, const long long *len, const double *s,
                                                  const TX *__restrict__ x, TY *__restrict__ y) {
  // arithmetic in the wider of the two types (FP32 for FP32 vectors: FP64 is 1/64 rate)
  using A = typename std::conditional<(sizeof(TX) > sizeof(TY)), TX, TY>::type;
  const int m = blockIdx.y;
  const long long o = off[m], n = len[m];
  const A f = (A)s[m];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[o + i] = (TY)((A)x[o + i] * f);
}

// u_m = sum_k y[m][k] V_k
__global__ void __launch_bounds__(kT) k_seg_lincomb(const long long *off, const long long *len, int nv,
                                                    const float *__restrict__ V, long long ld,
                                                    const double *__restrict__ yv, float *__restrict__ u) {
  __shared__ float ys[kMaxRestart];
  const int m = blockIdx.y;
  for (int k = threadIdx.x; k < nv; k += blockDim.x) ys[k] = (float)yv[m * kMaxRestart + k];
  __syncthreads();
  const long long o = off[m], n = len[m];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float v = 0.f;
    for (int k = 0; k < nv; ++k) v += ys[k] * V[(long long)k * ld + o + i];
    u[o + i] = v;
  }
}

__global__ void __launch_bounds__(kT) k_mul32(long long n, const float *__restrict__ a, const float *__restrict__ x,
                                              float *__restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = a[i] * x[i];
}

__global__ void __launch_bounds__(kT) k_resid(long long n, const double *__restrict__ b, const double *__restrict__ Sx,
                                              double *__restrict__ r) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    r[i] = b[i] - Sx[i];
}

// part[m][b][0] = block b's share of |v_m|^2 in FP64 (grid (kSegBlocks, nm))
__global__ void __launch_bounds__(kT) k_seg_norm2_64(const long long *off, const long long *len,
                                                     const double *__restrict__ v, double *__restrict__ part) {
  __shared__ double sh[32];
  const int m = blockIdx.y;
  const long long o = off[m], n = len[m];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    acc += v[o + i] * v[o + i];
  const double t = bsum(acc, sh);
  if (threadIdx.x == 0) part[((long long)m * kSegBlocks + blockIdx.x) * (kMaxRestart + 1)] = t;
}

__global__ void k_sqrt_members(int nm, const double *nrm, double *out) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < nm) out[m] = sqrt(nrm[m * (kMaxRestart + 1)]);
}

// Convergence check of the refinement loop (one CTA, one thread per member):
// relres_m = |r_m| / |b_m|; a member at or below tol is frozen (its later inner
// cycles leave it alone); the loop goes on while some member is above tol, all
// residuals are finite and fewer than maxit cycles have run.  The decision sets
// the WHILE node's condition; the cycle counters advance with it.
__global__ void k_refine_check(int nm, double tol, int maxit, const double *nrm, const double *bn, int *frozen,
                               double *relres, int *its, int *ctl, cudaGraphConditionalHandle cond) {
  const int m = threadIdx.x;
  bool d = true, bad = false;
  if (m < nm) {
    const double rel = bn[m] > 0.0 ? sqrt(nrm[m * (kMaxRestart + 1)]) / bn[m] : 0.0;
    relres[m] = rel;
    bad = !isfinite(rel);
    d = rel <= tol;
    frozen[m] = d ? 1 : 0;
  }
  const int cycles = ctl[0];
  const bool all = __syncthreads_and(d), anybad = __syncthreads_or(bad);
  const bool go = !all && !anybad && cycles < maxit;
  if (m < nm && go && !d) its[m] += 1;
  if (threadIdx.x == 0) {
    if (anybad) ctl[1] = 1;
    if (go) ctl[0] = cycles + 1;
    cudaGraphSetConditional(cond, go ? 1u : 0u);
  }
}

__global__ void __launch_bounds__(kT) k_addf(long long n, const float *__restrict__ d, double *__restrict__ x) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] += (double)d[i];
}

// Start of a cycle, per member: beta = |r|, scale = 1/beta, g = (beta, 0, ...),
// active iff beta > 0 and the refinement loop has not frozen the member.
__global__ void k_cycle_start(int nm, const double *nrm, const int *frozen, double *scl, double *g, int *act, int *jj,
                              double *beta0) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nm) return;
  const double beta = sqrt(nrm[m * (kMaxRestart + 1)]);
  beta0[m] = beta;
  const bool a = beta > 0.0 && !frozen[m];
  for (int k = 0; k <= kMaxRestart; ++k) g[m * (kMaxRestart + 1) + k] = 0.0;
  g[m * (kMaxRestart + 1)] = a ? beta : 0.0;
  scl[m] = a ? 1.0 / beta : 0.0;
  act[m] = a ? 1 : 0;
  jj[m] = 0;
}

// Arnoldi column j of every active member: H(:,j) = h1 + h2, subdiagonal |w|,
// previous Givens rotations, a new rotation, the residual estimate; the scale
// 1/h_{j+1,j} of the next basis vector (0 when the member stops).
__global__ void k_givens(int nm, int j, int m_rs, double tol, const double *h1, const double *h2, const double *nrm,
                         const double *beta0, double *H, double *cs, double *sn, double *g, double *scl, int *act,
                         int *jj) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nm) return;
  if (!act[m]) {
    scl[m] = 0.0;
    return;
  }
  double *Hm = H + (long long)m * (kMaxRestart + 1) * kMaxRestart;
  double *csm = cs + m * kMaxRestart, *snm = sn + m * kMaxRestart, *gm = g + m * (kMaxRestart + 1);
  for (int i = 0; i <= j; ++i) Hm[i * kMaxRestart + j] = h1[m * (kMaxRestart + 1) + i] + h2[m * (kMaxRestart + 1) + i];
  const double hn = sqrt(nrm[m * (kMaxRestart + 1)]);
  for (int i = 0; i < j; ++i) {
    const double a = Hm[i * kMaxRestart + j], b = Hm[(i + 1) * kMaxRestart + j];
    Hm[i * kMaxRestart + j] = csm[i] * a + snm[i] * b;
    Hm[(i + 1) * kMaxRestart + j] = -snm[i] * a + csm[i] * b;
  }
  const double a = Hm[j * kMaxRestart + j], b = hn;
  const double r = hypot(a, b);
  csm[j] = r > 0.0 ? a / r : 1.0;
  snm[j] = r > 0.0 ? b / r : 0.0;
  Hm[j * kMaxRestart + j] = r;
  gm[j + 1] = -snm[j] * gm[j];
  gm[j] = csm[j] * gm[j];
  jj[m] = j + 1;
  // stop this member on (near) breakdown, on a NaN, once the inner tolerance is
  // met (|g_{j+1}| is the residual estimate), or at the end of the cycle
  const bool stop = !(hn > 1e-30) || isnan(hn) || fabs(gm[j + 1]) <= tol * beta0[m] || j + 1 >= m_rs;
  if (stop) {
    act[m] = 0;
    scl[m] = 0.0;
  } else {
    scl[m] = 1.0 / hn;
  }
}

// y = R^-1 g per member (upper triangular, size jj[m])
__global__ void k_backsolve(int nm, const double *H, const double *g, const int *jj, double *yv) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nm) return;
  const double *Hm = H + (long long)m * (kMaxRestart + 1) * kMaxRestart;
  const double *gm = g + m * (kMaxRestart + 1);
  double *ym = yv + m * kMaxRestart;
  const int k = jj[m];
  for (int i = kMaxRestart - 1; i >= k; --i) ym[i] = 0.0;
  for (int i = k - 1; i >= 0; --i) {
    double s = gm[i];
    for (int l = i + 1; l < k; ++l) s -= Hm[i * kMaxRestart + l] * ym[l];
    const double d = Hm[i * kMaxRestart + i];
    ym[i] = d != 0.0 ? s / d : 0.0;
  }
}

int vblocks(long long n) {
  long long b = (n + kT * 4 - 1) / (kT * 4);
  return (int)std::min<long long>(std::max<long long>(b, 1), 608);
}

// ---------------------------------------------------------------- operations
// the fused multi-mesh operator of one group (degree and terrain dispatch):
// FP32, or FP64 arrays in double-word arithmetic
template <typename T>
int fused_group(dgx_ensemble *e, const Group &G, int cfg, const T *x, T *y) {
  dgx_ctx *c0 = e->mem[G.idx[0]];
  const int nm = (int)G.idx.size(), nb = G.nblocks[cfg];
  const int *co = G.cta_off[cfg];
  using C = typename std::conditional<sizeof(T) == 8, df64, float>::type;
  const EnsMember<C> *tab;
  if constexpr (sizeof(T) == 8) tab = G.ddf;
  else tab = G.d32;
#define FG(NN) (G.curved ? fused_operator_multi<C, NN, true>(c0, tab, nm, co, nb, x, y, e->stream, cfg) \
                         : fused_operator_multi<C, NN, false>(c0, tab, nm, co, nb, x, y, e->stream, cfg))
  int r;
  switch (G.n) {
    case 2: r = FG(2); break;
    case 3: r = FG(3); break;
    case 4: r = FG(4); break;
    case 5: r = FG(5); break;
    case 6: r = FG(6); break;
    case 7: r = FG(7); break;
    default: return eset(e, DGX_ERR_ARG, "unsupported degree %d", G.n - 1);
  }
#undef FG
  if (r) e->err = c0->err;
  return r;
}

template <typename T>
int apply_all(dgx_ensemble *e, const T *x, T *y) {
  for (auto &G : e->groups) {
    const EnsMember<T> *d;
    int th;
    if constexpr (sizeof(T) == 8) {
      if (G.tile64 >= 0) {
        if (int r = fused_group<double>(e, G, G.tile64, x, y)) return r;
        continue;
      }
      d = G.d64;
      th = G.threads64;
    } else {
      if (G.tile32 >= 0) {
        if (int r = fused_group<float>(e, G, G.tile32, x, y)) return r;
        continue;
      }
      d = G.d32;
      th = G.threads32;
    }
    if (int r = launch_operator_multi<T>(e->mem[G.idx[0]], G.n, G.curved, d, (int)G.idx.size(), G.ncell, x, y,
                                         e->stream, th)) {
      e->err = e->mem[G.idx[0]]->err;
      return r;
    }
  }
  return 0;
}

// per-member inner products of `cnt` basis vectors from index i0 with w -> out (device)
void seg_mdot(dgx_ensemble *e, int nv, const float *V, const float *w, double *out) {
  const dim3 grid(kSegBlocks, e->nm);
  for (int i0 = 0; i0 < nv; i0 += 8) {
    const int cnt = std::min(8, nv - i0);
    count_launch();
    k_seg_mdot<float><<<grid, kT, 0, e->stream>>>(e->seg_off, e->seg_len, i0, cnt, V, e->Ntot, w, e->part);
  }
  count_launch();
  k_seg_reduce<<<dim3(nv, e->nm), 64, 0, e->stream>>>(e->part, out);
}

void seg_norm2(dgx_ensemble *e, const float *w, double *out) { seg_mdot(e, 1, w, w, out); }

int ensure_basis(dgx_ensemble *e, int m) {
  if (e->vm >= m && e->V32) return 0;
  if (e->V32) {
    cudaFree(e->V32);
    e->owned.erase(std::remove(e->owned.begin(), e->owned.end(), (void *)e->V32), e->owned.end());
    e->V32 = nullptr;
  }
  if (e->gexec) {
    cudaGraphExecDestroy(e->gexec);
    e->gexec = nullptr;
  }
  if (int r = ealloc(e, &e->V32, (size_t)(m + 1) * e->Ntot)) return r;
  e->vm = m;
  return 0;
}

// Enqueue one inner FP32 GMRES(m) cycle for all members: r32 -> d32 = M^-1-preconditioned correction.
int enqueue_cycle(dgx_ensemble *e, int m, double inner_tol, int *frozen_dev) {
  const long long Nt = e->Ntot;
  const dim3 sgrid(kSegBlocks, e->nm);
  cudaStream_t s = e->stream;
  const int mb = (e->nm + 31) / 32;
  seg_norm2(e, e->r32, e->nrm);
  count_launch(2);
  k_cycle_start<<<mb, 32, 0, s>>>(e->nm, e->nrm, frozen_dev, e->scl, e->g, e->act, e->jj, e->beta0);
  k_seg_scale<float, float><<<sgrid, kT, 0, s>>>(e->seg_off, e->seg_len, e->scl, e->r32, e->V32);
  for (int j = 0; j < m; ++j) {
    float *vj = e->V32 + (size_t)j * Nt;
    count_launch();
    k_mul32<<<vblocks(Nt), kT, 0, s>>>(Nt, e->dinv32, vj, e->u32);
    if (int r = apply_all<float>(e, e->u32, e->w32)) return r;
    seg_mdot(e, j + 1, e->V32, e->w32, e->h1);
    count_launch();
    k_seg_mupdate<<<sgrid, kT, 0, s>>>(e->seg_off, e->seg_len, j + 1, e->V32, Nt, e->h1, e->w32, e->part, 0);
    seg_mdot(e, j + 1, e->V32, e->w32, e->h2);
    count_launch(2);
    k_seg_mupdate<<<sgrid, kT, 0, s>>>(e->seg_off, e->seg_len, j + 1, e->V32, Nt, e->h2, e->w32, e->part, 1);
    k_seg_reduce<<<dim3(1, e->nm), 64, 0, s>>>(e->part, e->nrm);
    count_launch(2);
    k_givens<<<mb, 32, 0, s>>>(e->nm, j, m, inner_tol, e->h1, e->h2, e->nrm, e->beta0, e->H, e->cs, e->sn, e->g,
                               e->scl, e->act, e->jj);
    k_seg_scale<float, float><<<sgrid, kT, 0, s>>>(e->seg_off, e->seg_len, e->scl, e->w32,
                                                  e->V32 + (size_t)(j + 1) * Nt);
  }
  count_launch(3);
  k_backsolve<<<mb, 32, 0, s>>>(e->nm, e->H, e->g, e->jj, e->y);
  k_seg_lincomb<<<sgrid, kT, 0, s>>>(e->seg_off, e->seg_len, m, e->V32, Nt, e->y, e->u32);
  k_mul32<<<vblocks(Nt), kT, 0, s>>>(Nt, e->dinv32, e->u32, e->d32);
  return echeck(e, cudaGetLastError(), "inner cycle launch");
}

// Threads per CTA for each group and precision: time a few candidates.
int autotune(dgx_ensemble *e) {
  if (e->tuned) return 0;
  const int cand[3] = {128, 192, 256};
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  for (auto &G : e->groups) {
    for (int prec = 0; prec < 2; ++prec) {
      float best = 1e30f;
      int bt = 256;
      for (int th : cand) {
        if (prec == 0) G.threads64 = th;
        else G.threads32 = th;
        for (int rep = 0; rep < 3; ++rep) {
          if (rep == 1) cudaEventRecord(a, e->stream);
          int r = 0;
          // time only this group: temporarily apply with the others untouched
          if (prec == 0)
            r = launch_operator_multi<double>(e->mem[G.idx[0]], G.n, G.curved, G.d64, (int)G.idx.size(), G.ncell,
                                              e->r64, e->t64, e->stream, th);
          else
            r = launch_operator_multi<float>(e->mem[G.idx[0]], G.n, G.curved, G.d32, (int)G.idx.size(), G.ncell,
                                             e->r32, e->w32, e->stream, th);
          if (r) {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            e->err = e->mem[G.idx[0]]->err;
            return r;
          }
        }
        cudaEventRecord(b, e->stream);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best) {
          best = ms;
          bt = th;
        }
      }
      if (prec == 0) {
        G.threads64 = bt;
        G.tile64 = -1;
      } else {
        G.threads32 = bt;
        G.tile32 = -1;
      }
      // the fused kernels (FP32; FP64 in double-words) in each configuration that
      // fits (cells per CTA x threads)
      for (int cfg = 0; cfg < 2; ++cfg) {
        if (!(prec == 0 ? G.fits64[cfg] : G.fits32[cfg])) continue;
        for (int rep = 0; rep < 3; ++rep) {
          if (rep == 1) cudaEventRecord(a, e->stream);
          const int r = prec == 0 ? fused_group<double>(e, G, cfg, e->r64, e->t64)
                                  : fused_group<float>(e, G, cfg, e->r32, e->w32);
          if (r) {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            return r;
          }
        }
        cudaEventRecord(b, e->stream);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best) {
          best = ms;
          if (prec == 0) {
            G.tile64 = cfg;
            G.threads64 = fused_nt(G.n, cfg);
          } else {
            G.tile32 = cfg;
            G.threads32 = fused_nt(G.n, cfg);
          }
        }
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  e->tuned = true;
  return echeck(e, cudaGetLastError(), "autotune");
}

}  // namespace

extern "C" {

int dgx_ensemble_create(dgx_ensemble **out, int device, void *stream, int n, const dgx_mesh_desc *descs) {
  if (!out) return DGX_ERR_ARG;
  *out = nullptr;
  if (n < 1 || n > kMaxMembers || !descs) return DGX_ERR_ARG;
  dgx_ensemble *e = new dgx_ensemble();
  e->device = device;
  e->user_stream = reinterpret_cast<cudaStream_t>(stream);
  e->nm = n;
  auto fail = [&](int code) {
    *out = e;  // keep the error message readable; caller destroys
    return code;
  };
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&e->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&e->ev_out, cudaEventDisableTiming) != cudaSuccess)
    return fail(eset(e, DGX_ERR_CUDA, "stream or event creation failed"));
  for (int m = 0; m < n; ++m) {
    dgx_ctx *c = nullptr;
    int r = dgx_create(&c, device, e->stream);
    if (r) return fail(eset(e, r, "member %d: context creation failed", m));
    c->use_kappa = false;  // the multi-mesh kernels interpolate p_k themselves
    e->mem.push_back(c);
    r = dgx_mesh_build(c, &descs[m]);
    if (r) return fail(eset(e, r, "member %d: %s", m, c->err.c_str()));
    if (c->nc) return fail(eset(e, DGX_ERR_STATE, "member %d: ensembles take conforming meshes only", m));
    e->N.push_back(c->N);
    e->off.push_back(e->Ntot);
    e->Ntot += c->N;
  }
  // degree groups (members of equal degree and terrain kind share one launch)
  for (int m = 0; m < n; ++m) {
    const dgx_ctx *c = e->mem[m];
    auto it = std::find_if(e->groups.begin(), e->groups.end(),
                           [&](const Group &G) { return G.n == c->n && G.curved == c->curved; });
    if (it == e->groups.end()) {
      Group G;
      G.n = c->n;
      G.curved = c->curved;
      e->groups.push_back(G);
      it = e->groups.end() - 1;
    }
    it->idx.push_back(m);
  }
  int r;
  const size_t Nt = (size_t)e->Ntot;
  if ((r = ealloc(e, &e->r64, Nt)) || (r = ealloc(e, &e->t64, Nt)) || (r = ealloc(e, &e->r32, Nt)) ||
      (r = ealloc(e, &e->d32, Nt)) || (r = ealloc(e, &e->w32, Nt)) || (r = ealloc(e, &e->u32, Nt)) ||
      (r = ealloc(e, &e->dinv32, Nt)))
    return fail(r);
  const size_t S = (size_t)n * (kMaxRestart + 1);
  if ((r = ealloc(e, &e->bn, S)) || (r = ealloc(e, &e->part, (size_t)n * kSegBlocks * (kMaxRestart + 1))) ||
      (r = ealloc(e, &e->h1, S)) || (r = ealloc(e, &e->h2, S)) || (r = ealloc(e, &e->nrm, S)) ||
      (r = ealloc(e, &e->H, S * kMaxRestart)) || (r = ealloc(e, &e->cs, (size_t)n * kMaxRestart)) ||
      (r = ealloc(e, &e->sn, (size_t)n * kMaxRestart)) || (r = ealloc(e, &e->g, S)) ||
      (r = ealloc(e, &e->y, (size_t)n * kMaxRestart)) || (r = ealloc(e, &e->scl, (size_t)n)) ||
      (r = ealloc(e, &e->beta0, (size_t)n)) ||
      (r = ealloc(e, &e->jj, (size_t)n)) || (r = ealloc(e, &e->act, (size_t)2 * n)) ||
      (r = ealloc(e, &e->seg_off, (size_t)n)) || (r = ealloc(e, &e->seg_len, (size_t)n)) ||
      (r = ealloc(e, &e->relres_d, (size_t)n)) || (r = ealloc(e, &e->its_d, (size_t)n)) ||
      (r = ealloc(e, &e->ctl_d, (size_t)2)))
    return fail(r);
  if ((r = echeck(e, cudaMallocHost(&e->host, S * sizeof(double)), "cudaMallocHost"))) return fail(r);
  cudaMemset(e->r64, 0, Nt * sizeof(double));
  cudaMemset(e->t64, 0, Nt * sizeof(double));
  cudaMemset(e->r32, 0, Nt * sizeof(float));
  cudaMemset(e->w32, 0, Nt * sizeof(float));
  cudaMemcpy(e->seg_off, e->off.data(), n * sizeof(long long), cudaMemcpyHostToDevice);
  cudaMemcpy(e->seg_len, e->N.data(), n * sizeof(long long), cudaMemcpyHostToDevice);
  *out = e;
  return echeck(e, cudaDeviceSynchronize(), "ensemble create");
}

void dgx_ensemble_destroy(dgx_ensemble *e) {
  if (!e) return;
  cudaSetDevice(e->device);
  cudaStreamSynchronize(e->stream);
  if (e->gexec) cudaGraphExecDestroy(e->gexec);
  for (void *p : e->owned) cudaFree(p);
  if (e->host) cudaFreeHost(e->host);
  for (auto *c : e->mem) dgx_destroy(c);
  if (e->ev_in) cudaEventDestroy(e->ev_in);
  if (e->ev_out) cudaEventDestroy(e->ev_out);
  if (e->stream) cudaStreamDestroy(e->stream);
  delete e;
}

const char *dgx_ensemble_last_error(const dgx_ensemble *e) { return e ? e->err.c_str() : "null ensemble"; }

long long dgx_ensemble_num_dofs(const dgx_ensemble *e, int m) {
  if (!e) return -1;
  if (m < 0) return e->Ntot;
  return m < e->nm ? e->N[m] : -1;
}

long long dgx_ensemble_offset(const dgx_ensemble *e, int m) {
  if (!e || m < 0 || m >= e->nm) return -1;
  return e->off[m];
}

int dgx_ensemble_member(dgx_ensemble *e, int m, dgx_ctx **ctx) {
  if (!e || !ctx || m < 0 || m >= e->nm) return DGX_ERR_ARG;
  *ctx = e->mem[m];
  return DGX_OK;
}

int dgx_ensemble_set_coefficients(dgx_ensemble *e, const double *rho_all, const double *pk_all, double a_dt,
                                  double gamma) {
  if (!e || !rho_all || !pk_all) return DGX_ERR_ARG;
  enter(e);
  for (int m = 0; m < e->nm; ++m) {
    dgx_ctx *c = e->mem[m];
    if (int r = dgx_set_coefficients(c, rho_all + e->off[m], pk_all + e->off[m], a_dt, gamma))
      return eset(e, r, "member %d: %s", m, c->err.c_str());
    if (int r = ensure_diag(c, false))  // the FP32 cycles use the FP32 Helmholtz diagonal
      return eset(e, r, "member %d: %s", m, c->err.c_str());
    cudaMemcpyAsync(e->dinv32 + e->off[m], c->dinv32[DGX_PC_HELMHOLTZ], c->N * sizeof(float),
                    cudaMemcpyDeviceToDevice, e->stream);
  }
  // member tables per group (pointers into the member contexts)
  for (auto &G : e->groups) {
    std::vector<EnsMember<double>> h64;
    std::vector<EnsMember<float>> h32;
    std::vector<EnsMember<df64>> hdf;
    long long co = 0;
    for (int m : G.idx) {
      dgx_ctx *c = e->mem[m];
      EnsMember<double> a;
      a.P = make_params<double>(c);
      a.rho = c->rho64;
      a.pk = c->pk64;
      a.V = c->V64;
      a.cell_off = co;
      a.dof_off = e->off[m];
      a.N = c->N;
      EnsMember<float> f;
      f.P = make_params<float>(c);
      f.rho = c->rho32;
      f.pk = c->pk32;
      f.V = c->V32;
      f.cell_off = co;
      f.dof_off = e->off[m];
      f.N = c->N;
      EnsMember<df64> w;
      w.P = make_params<df64>(c);
      w.rho = c->rho64;
      w.pk = c->pk64;
      w.V = c->V64;
      w.cell_off = co;
      w.dof_off = e->off[m];
      w.N = c->N;
      h64.push_back(a);
      h32.push_back(f);
      hdf.push_back(w);
      co += c->ncell;
    }
    G.ncell = co;
    if (!G.d64) {
      int r;
      if ((r = ealloc(e, &G.d64, G.idx.size())) || (r = ealloc(e, &G.d32, G.idx.size())) ||
          (r = ealloc(e, &G.ddf, G.idx.size())))
        return r;
    }
    cudaMemcpyAsync(G.ddf, hdf.data(), hdf.size() * sizeof(EnsMember<df64>), cudaMemcpyHostToDevice, e->stream);
    cudaMemcpyAsync(G.d64, h64.data(), h64.size() * sizeof(EnsMember<double>), cudaMemcpyHostToDevice, e->stream);
    cudaMemcpyAsync(G.d32, h32.data(), h32.size() * sizeof(EnsMember<float>), cudaMemcpyHostToDevice, e->stream);
    // CTA ranges of the fused configurations that fit in shared memory
    for (int cfg = 0; cfg < 2; ++cfg) {
      dgx_ctx *c0 = e->mem[G.idx[0]];
      G.fits32[cfg] = op_variant_ok<float>(c0, 3 + cfg);
      G.fits64[cfg] = op_variant_ok<double>(c0, 5 + cfg);
      if (!G.fits32[cfg] && !G.fits64[cfg]) continue;
      const int cpb = fused_cpb(G.n, cfg);
      std::vector<int> co(G.idx.size() + 1, 0);
      for (size_t k = 0; k < G.idx.size(); ++k)
        co[k + 1] = co[k] + (int)((e->mem[G.idx[k]]->ncell + cpb - 1) / cpb);
      if (!G.cta_off[cfg])
        if (int r = ealloc(e, &G.cta_off[cfg], co.size())) return r;
      G.nblocks[cfg] = co.back();
      cudaMemcpyAsync(G.cta_off[cfg], co.data(), co.size() * sizeof(int), cudaMemcpyHostToDevice, e->stream);
    }
  }
  if (int r = echeck(e, cudaStreamSynchronize(e->stream), "ensemble coefficients")) return r;
  e->has_coef = true;
  return DGX_OK;  // synchronised: nothing left to order
}

int dgx_ensemble_apply_operator(dgx_ensemble *e, int prec, const void *x, void *y) {
  if (!e || !x || !y || x == y) return DGX_ERR_ARG;
  if (!e->has_coef) return eset(e, DGX_ERR_STATE, "no coefficients (call dgx_ensemble_set_coefficients)");
  if (prec != DGX_F64 && prec != DGX_F32) return eset(e, DGX_ERR_ARG, "precision %d", prec);
  enter(e);
  const int r = prec == DGX_F64 ? apply_all<double>(e, (const double *)x, (double *)y)
                                : apply_all<float>(e, (const float *)x, (float *)y);
  leave(e);
  return r;
}

int dgx_ensemble_autotune(dgx_ensemble *e) {
  if (!e) return DGX_ERR_ARG;
  if (!e->has_coef) return eset(e, DGX_ERR_STATE, "no coefficients (call dgx_ensemble_set_coefficients)");
  enter(e);
  const int r = autotune(e);
  leave(e);
  return r;
}

int dgx_ensemble_tile(const dgx_ensemble *e, int group, int prec, int *fused, int *cells_per_cta) {
  if (!e || group < 0 || group >= (int)e->groups.size() || (prec != DGX_F64 && prec != DGX_F32)) return DGX_ERR_ARG;
  const Group &G = e->groups[group];
  const int t = prec == DGX_F64 ? G.tile64 : G.tile32;
  if (fused) *fused = t >= 0 ? 1 : 0;
  if (cells_per_cta) *cells_per_cta = t < 0 ? 1 : fused_cpb(G.n, t);
  return DGX_OK;
}

int dgx_ensemble_tuning(const dgx_ensemble *e, int group, int *degree, int *members, int *threads64, int *threads32) {
  if (!e || group < 0 || group >= (int)e->groups.size()) return DGX_ERR_ARG;
  const Group &G = e->groups[group];
  if (degree) *degree = G.n - 1;
  if (members) *members = (int)G.idx.size();
  if (threads64) *threads64 = G.threads64;
  if (threads32) *threads32 = G.threads32;
  return DGX_OK;
}

int dgx_ensemble_solve(dgx_ensemble *e, const double *b, double *x, const dgx_solve_opts *opts,
                       dgx_solve_info *info) {
  if (!e || !b || !x || b == x) return DGX_ERR_ARG;
  if (!e->has_coef) return eset(e, DGX_ERR_STATE, "no coefficients (call dgx_ensemble_set_coefficients)");
  const auto t0 = std::chrono::steady_clock::now();
  enter(e);
  dgx_solve_opts o;
  if (opts) o = *opts;
  else dgx_default_solve_opts(&o);
  const int m = o.inner_maxit;
  if (m < 1 || m > kMaxRestart || !(o.tol > 0) || !(o.inner_tol > 0) || o.maxit < 1)
    return eset(e, DGX_ERR_ARG, "need 1 <= inner_maxit <= %d, tol > 0, inner_tol > 0, maxit >= 1", kMaxRestart);
  int r;
  if ((r = autotune(e))) return r;
  if ((r = ensure_basis(e, m))) return r;
  const long long Nt = e->Ntot;
  const int nm = e->nm;
  cudaStream_t s = e->stream;
  int *frozen = e->act + nm;  // device flags: member converged, stop correcting
  const int x0 = o.use_x0 ? 1 : 0;
  if (!e->gexec || e->graph_b != b || e->graph_x != x || e->graph_m != m || e->graph_tol != o.tol ||
      e->graph_itol != o.inner_tol || e->graph_maxit != o.maxit || e->graph_x0 != x0) {
    if (e->gexec) {
      cudaGraphExecDestroy(e->gexec);
      e->gexec = nullptr;
    }
    // warm every kernel once outside capture (attributes, lazy loading)
    cudaMemsetAsync(frozen, 0, nm * sizeof(int), s);
    if ((r = enqueue_cycle(e, 1, o.inner_tol, frozen))) return r;
    if ((r = apply_all<double>(e, x, e->t64))) return r;
    if ((r = echeck(e, cudaStreamSynchronize(s), "warm-up cycle"))) return r;
    const dim3 sgrid(kSegBlocks, nm);
    // FP64 residual r = b - S x of every member and |r_m|^2 into nrm
    auto residual = [&]() -> int {
      if (int q = apply_all<double>(e, x, e->t64)) return q;
      count_launch(3);
      k_resid<<<vblocks(Nt), kT, 0, s>>>(Nt, b, e->t64, e->r64);
      k_seg_norm2_64<<<sgrid, kT, 0, s>>>(e->seg_off, e->seg_len, e->r64, e->part);
      k_seg_reduce<<<dim3(1, nm), 64, 0, s>>>(e->part, e->nrm);
      return 0;
    };
    cudaGraph_t g = nullptr;
    cudaGraphConditionalHandle cond;
    if ((r = echeck(e, cudaGraphCreate(&g, 0), "graph create"))) return r;
    auto fail = [&](int code) {
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
        cudaGraph_t junk = nullptr;
        cudaStreamEndCapture(s, &junk);
      }
      cudaGraphDestroy(g);
      return code;
    };
    if ((r = echeck(e, cudaGraphConditionalHandleCreate(&cond, g, 0, 0), "conditional handle"))) return fail(r);
    if ((r = echeck(e, cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
                    "begin capture")))
      return fail(r);
    const long long c0 = launch_count();
    // prologue: counters, |b_m|, first residual and check
    cudaMemsetAsync(e->its_d, 0, nm * sizeof(int), s);
    cudaMemsetAsync(e->ctl_d, 0, 2 * sizeof(int), s);
    cudaMemsetAsync(frozen, 0, nm * sizeof(int), s);
    if (!x0) cudaMemsetAsync(x, 0, Nt * sizeof(double), s);
    count_launch(3);
    k_seg_norm2_64<<<sgrid, kT, 0, s>>>(e->seg_off, e->seg_len, b, e->part);
    k_seg_reduce<<<dim3(1, nm), 64, 0, s>>>(e->part, e->nrm);
    k_sqrt_members<<<1, 64, 0, s>>>(nm, e->nrm, e->bn);
    if ((r = residual())) return fail(r);
    count_launch();
    k_refine_check<<<1, 64, 0, s>>>(nm, o.tol, o.maxit, e->nrm, e->bn, frozen, e->relres_d, e->its_d, e->ctl_d, cond);
    // the WHILE node after everything captured so far
    cudaStreamCaptureStatus cst;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    if ((r = echeck(e, cudaStreamGetCaptureInfo(s, &cst, nullptr, &cg, &deps, nullptr, &ndeps), "capture info")))
      return fail(r);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    if ((r = echeck(e, cudaGraphAddNode(&cnode, cg, deps, nullptr, ndeps, &cp), "conditional node"))) return fail(r);
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if ((r = echeck(e, cudaStreamUpdateCaptureDependencies(s, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies),
                    "capture dependencies")))
      return fail(r);
    if ((r = echeck(e, cudaStreamEndCapture(s, &g), "end capture"))) return fail(r);
    const long long c1 = launch_count();
    // body: one inner cycle of all members, the correction, the new residual and check
    if ((r = echeck(e, cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
                    "begin body capture")))
      return fail(r);
    vec_convert<float, double>(Nt, e->r64, e->r32, s);
    if ((r = enqueue_cycle(e, m, o.inner_tol, frozen))) return fail(r);
    count_launch();
    k_addf<<<vblocks(Nt), kT, 0, s>>>(Nt, e->d32, x);
    if ((r = residual())) return fail(r);
    count_launch();
    k_refine_check<<<1, 64, 0, s>>>(nm, o.tol, o.maxit, e->nrm, e->bn, frozen, e->relres_d, e->its_d, e->ctl_d, cond);
    if ((r = echeck(e, cudaStreamEndCapture(s, &body), "end body capture"))) return fail(r);
    const long long c2 = launch_count();
    count_launch((int)-(c2 - c0));  // captured, not yet run: counted per run below
    r = echeck(e, cudaGraphInstantiate(&e->gexec, g, 0), "graph instantiate");
    cudaGraphDestroy(g);
    if (r) return r;
    e->graph_b = b;
    e->graph_x = x;
    e->graph_m = m;
    e->graph_tol = o.tol;
    e->graph_itol = o.inner_tol;
    e->graph_maxit = o.maxit;
    e->graph_x0 = x0;
    e->graph_pro_launches = c1 - c0;
    e->graph_body_launches = c2 - c1;
  }
  // the whole refinement loop: one launch
  if ((r = echeck(e, cudaGraphLaunch(e->gexec, s), "graph launch"))) return r;
  // per-member results back in one read
  double *hr = e->host;
  int *hi = reinterpret_cast<int *>(e->host + nm);
  cudaMemcpyAsync(hr, e->relres_d, nm * sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(hi, e->its_d, nm * sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(hi + nm, e->ctl_d, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
  if ((r = echeck(e, cudaStreamSynchronize(s), "ensemble solve"))) return r;
  const int cycles = hi[nm];
  count_launch((int)(1 + e->graph_pro_launches + cycles * e->graph_body_launches));
  if (hi[nm + 1]) {
    for (int mm = 0; mm < nm; ++mm)
      if (!std::isfinite(hr[mm])) return eset(e, DGX_ERR_BREAKDOWN, "member %d: non-finite residual", mm);
    return eset(e, DGX_ERR_BREAKDOWN, "non-finite residual");
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  int status = DGX_OK;
  std::vector<dgx_solve_info> inf(nm);
  for (int mm = 0; mm < nm; ++mm) {
    std::memset(&inf[mm], 0, sizeof(dgx_solve_info));
    const bool ok = hr[mm] <= o.tol;
    inf[mm].relres = hr[mm];
    inf[mm].iterations = hi[mm];
    inf[mm].inner_iterations = hi[mm] * m;
    inf[mm].operator_f32 = hi[mm] * m;
    inf[mm].operator_f64 = cycles + 1;
    inf[mm].status = ok ? DGX_OK : DGX_NOT_CONVERGED;
    inf[mm].seconds = secs;
    if (!ok) status = DGX_NOT_CONVERGED;
  }
  if (info) std::memcpy(info, inf.data(), nm * sizeof(dgx_solve_info));
  leave(e);
  return status;
}

}  // extern "C"
