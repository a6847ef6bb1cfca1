// Vector kernels of the Krylov solvers (Sec. 3.1: GMRES / CG with a Jacobi
// preconditioner), sm_103a.  These are HBM-bound streams: one pass over the
// operands, grid-stride loops.  FP64 vectors use FP64 throughout.  FP32
// vectors (the inner solve of the mixed-precision preconditioner) use FP32
// per-thread arithmetic -- FP64 runs at 1/64 of the FP32 rate on GB300 and
// would make these streams ALU bound -- and FP64 for the block and grid
// combination.  Reductions are deterministic: a fixed grid for a given
// length, per-block partial sums, then a fixed-order tree over blocks.
#include <atomic>
#include <cstdint>
#include <type_traits>

#include "dgx_common.cuh"

namespace dgx {

static std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 4 * 152;  // 4 CTAs on each of the 152 SMs
constexpr int kChunk = 8;            // vectors per inner-product pass

int nblocks(long long n) {
  long long b = (n + kThreads * 4 - 1) / (kThreads * 4);
  if (b < 1) b = 1;
  return (int)(b < kMaxBlocks ? b : kMaxBlocks);
}

__device__ __forceinline__ double block_sum(double v, double *sh) {
  // warp shuffle, then one value per warp through shared memory
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
  return t;  // valid in thread 0
}

template <typename T>
__global__ void k_axpby(long long n, double a, const T *__restrict__ x, double b, T *__restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (T)(a * (double)x[i] + b * (double)y[i]);
}

template <typename T>
__global__ void k_mul(long long n, const T *__restrict__ a, const T *__restrict__ x, T *__restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = a[i] * x[i];
}

template <typename TO, typename TI>
__global__ void k_convert(long long n, const TI *__restrict__ x, TO *__restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (TO)x[i];
}

__global__ void k_inv32(long long n, const float *__restrict__ d, float *__restrict__ di) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    di[i] = 1.0f / d[i];
}

__global__ void k_inv(long long n, const double *__restrict__ d, double *__restrict__ di64, float *__restrict__ di32) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = 1.0 / d[i];
    di64[i] = v;
    di32[i] = (float)v;
  }
}

// 16-byte vector of T
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int W = 4;
  __device__ static float dot(const float4 &a, const float4 &b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int W = 2;
  __device__ static double dot(const double2 &a, const double2 &b) { return a.x * b.x + a.y * b.y; }
};

// partial[blk * nv + i] = sum over this block's share of V_i . w, i in [i0, i0 + cnt).
// VEC: 16-byte loads (V_i and w 16-byte aligned, ld a multiple of the vector
// width), the n % W tail by the first threads.
template <typename T, bool VEC>
__global__ void __launch_bounds__(kThreads) k_mdot(long long n, int nv, int i0, int cnt, const T *__restrict__ V,
                                                   long long ld, const T *__restrict__ w, double *__restrict__ partial) {
  __shared__ double sh[32];
  T acc[kChunk];
#pragma unroll
  for (int c = 0; c < kChunk; ++c) acc[c] = T(0);
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
  long long done = 0;
  if (VEC) {
    using V16 = Vec16<T>;
    using VT = typename V16::type;
    constexpr int W = V16::W;
    const long long nw = n / W;
    const VT *w4 = reinterpret_cast<const VT *>(w);
    for (long long i = tid; i < nw; i += stride) {
      const VT wi = w4[i];
#pragma unroll
      for (int c = 0; c < kChunk; ++c)
        if (c < cnt) acc[c] += V16::dot(reinterpret_cast<const VT *>(V + (long long)(i0 + c) * ld)[i], wi);
    }
    done = nw * W;
  }
  for (long long i = done + tid; i < n; i += stride) {
    const T wi = w[i];
#pragma unroll
    for (int c = 0; c < kChunk; ++c)
      if (c < cnt) acc[c] += V[(long long)(i0 + c) * ld + i] * wi;
  }
  for (int c = 0; c < cnt; ++c) {
    const double t = block_sum((double)acc[c], sh);
    if (threadIdx.x == 0) partial[(long long)blockIdx.x * nv + i0 + c] = t;
  }
}

// out[i] = sum_b partial[b * nv + i] (fixed order), one block per i
__global__ void __launch_bounds__(kThreads) k_reduce(int nb, int nv, const double *__restrict__ partial,
                                                     double *__restrict__ out) {
  __shared__ double sh[32];
  double a = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) a += partial[(long long)b * nv + blockIdx.x];
  const double t = block_sum(a, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = t;
}

// w -= sum_i h[i] V_i ; partial norm^2 of the updated w (if partial != null)
template <typename T, bool VEC>
__global__ void __launch_bounds__(kThreads) k_mupdate(long long n, int nv, const T *__restrict__ V, long long ld,
                                                      const double *__restrict__ h, T *__restrict__ w,
                                                      double *__restrict__ partial) {
  __shared__ double sh[32];
  __shared__ T hs[128];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) hs[i] = (T)h[i];
  __syncthreads();
  T nrm = T(0);
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
  long long done = 0;
  if (VEC) {
    using V16 = Vec16<T>;
    using VT = typename V16::type;
    constexpr int W = V16::W;
    const long long nw = n / W;
    VT *w4 = reinterpret_cast<VT *>(w);
    for (long long i = tid; i < nw; i += stride) {
      VT v = w4[i];
      T *vv = reinterpret_cast<T *>(&v);
      for (int k = 0; k < nv; ++k) {
        const VT a = reinterpret_cast<const VT *>(V + (long long)k * ld)[i];
        const T *aa = reinterpret_cast<const T *>(&a);
#pragma unroll
        for (int q = 0; q < W; ++q) vv[q] -= hs[k] * aa[q];
      }
      w4[i] = v;
#pragma unroll
      for (int q = 0; q < W; ++q) nrm += vv[q] * vv[q];
    }
    done = nw * W;
  }
  for (long long i = done + tid; i < n; i += stride) {
    T v = w[i];
    for (int k = 0; k < nv; ++k) v -= hs[k] * V[(long long)k * ld + i];
    w[i] = v;
    nrm += v * v;
  }
  if (partial) {
    const double t = block_sum((double)nrm, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
  }
}

template <typename T>
__global__ void k_scale_inv_sqrt(long long n, const double *__restrict__ nrm2, const T *__restrict__ x,
                                 T *__restrict__ y) {
  const T s = (T)(1.0 / sqrt(*nrm2));
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i] * s;
}

template <typename T, typename TX>
__global__ void __launch_bounds__(kThreads) k_lincomb(long long n, int nv, const T *__restrict__ Z, long long ld,
                                                      const double *__restrict__ c, TX *__restrict__ x) {
  // arithmetic in the wider of the two types
  using A = typename std::conditional<(sizeof(T) > sizeof(TX)), T, TX>::type;
  __shared__ A cs[128];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) cs[i] = (A)c[i];
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    A v = (A)x[i];
    for (int k = 0; k < nv; ++k) v += cs[k] * (A)Z[(long long)k * ld + i];
    x[i] = (TX)v;
  }
}

}  // namespace

int vec_partials() { return kMaxBlocks; }

template <typename T>
void vec_axpby(long long n, double a, const T *x, double b, T *y, cudaStream_t s) {
  count_launch();
  k_axpby<T><<<nblocks(n), kThreads, 0, s>>>(n, a, x, b, y);
}
template <typename T>
void vec_mul(long long n, const T *a, const T *x, T *y, cudaStream_t s) {
  count_launch();
  k_mul<T><<<nblocks(n), kThreads, 0, s>>>(n, a, x, y);
}
template <typename TO, typename TI>
void vec_convert(long long n, const TI *x, TO *y, cudaStream_t s) {
  count_launch();
  k_convert<TO, TI><<<nblocks(n), kThreads, 0, s>>>(n, x, y);
}
void vec_inv32(long long n, const float *d, float *dinv, cudaStream_t s) {
  count_launch();
  k_inv32<<<nblocks(n), kThreads, 0, s>>>(n, d, dinv);
}
void vec_inv(long long n, const double *d, double *dinv64, float *dinv32, cudaStream_t s) {
  count_launch();
  k_inv<<<nblocks(n), kThreads, 0, s>>>(n, d, dinv64, dinv32);
}

// 16-byte loads when every vector starts on a 16-byte boundary
template <typename T>
bool vec16_ok(const void *a, const void *b, long long ld) {
  constexpr int W = 16 / sizeof(T);
  return ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15) == 0 && (ld % W) == 0;
}

template <typename T>
void vec_mdot(long long n, int nv, const T *V, long long ld, const T *w, double *partial, double *out,
              cudaStream_t s) {
  const int nb = nblocks(n);
  const bool vec = vec16_ok<T>(V, w, nv > 1 ? ld : 0);
  for (int i0 = 0; i0 < nv; i0 += kChunk) {
    const int cnt = nv - i0 < kChunk ? nv - i0 : kChunk;
    count_launch();
    if (vec) k_mdot<T, true><<<nb, kThreads, 0, s>>>(n, nv, i0, cnt, V, ld, w, partial);
    else k_mdot<T, false><<<nb, kThreads, 0, s>>>(n, nv, i0, cnt, V, ld, w, partial);
  }
  count_launch();
  k_reduce<<<nv, kThreads, 0, s>>>(nb, nv, partial, out);
}

template <typename T>
void vec_mupdate(long long n, int nv, const T *V, long long ld, const double *h, T *w, double *partial,
                 double *out_norm2, cudaStream_t s) {
  const int nb = nblocks(n);
  count_launch(out_norm2 ? 2 : 1);
  if (vec16_ok<T>(V, w, nv > 1 ? ld : 0))
    k_mupdate<T, true><<<nb, kThreads, 0, s>>>(n, nv, V, ld, h, w, out_norm2 ? partial : nullptr);
  else
    k_mupdate<T, false><<<nb, kThreads, 0, s>>>(n, nv, V, ld, h, w, out_norm2 ? partial : nullptr);
  if (out_norm2) k_reduce<<<1, kThreads, 0, s>>>(nb, 1, partial, out_norm2);
}

template <typename T>
void vec_scale_by_inv_sqrt(long long n, const double *nrm2, const T *x, T *y, cudaStream_t s) {
  count_launch();
  k_scale_inv_sqrt<T><<<nblocks(n), kThreads, 0, s>>>(n, nrm2, x, y);
}

template <typename T, typename TX>
void vec_lincomb(long long n, int nv, const T *Z, long long ld, const double *c_dev, TX *x, cudaStream_t s) {
  count_launch();
  k_lincomb<T, TX><<<nblocks(n), kThreads, 0, s>>>(n, nv, Z, ld, c_dev, x);
}

template <typename T>
void vec_dot(long long n, const T *a, const T *b, double *partial, double *out, cudaStream_t s) {
  vec_mdot<T>(n, 1, a, 0, b, partial, out, s);
}

template void vec_axpby<double>(long long, double, const double *, double, double *, cudaStream_t);
template void vec_axpby<float>(long long, double, const float *, double, float *, cudaStream_t);
template void vec_mul<double>(long long, const double *, const double *, double *, cudaStream_t);
template void vec_mul<float>(long long, const float *, const float *, float *, cudaStream_t);
template void vec_convert<float, double>(long long, const double *, float *, cudaStream_t);
template void vec_convert<double, float>(long long, const float *, double *, cudaStream_t);
template void vec_mdot<double>(long long, int, const double *, long long, const double *, double *, double *,
                               cudaStream_t);
template void vec_mdot<float>(long long, int, const float *, long long, const float *, double *, double *,
                              cudaStream_t);
template void vec_mupdate<double>(long long, int, const double *, long long, const double *, double *, double *,
                                  double *, cudaStream_t);
template void vec_mupdate<float>(long long, int, const float *, long long, const double *, float *, double *,
                                 double *, cudaStream_t);
template void vec_scale_by_inv_sqrt<double>(long long, const double *, const double *, double *, cudaStream_t);
template void vec_scale_by_inv_sqrt<float>(long long, const double *, const float *, float *, cudaStream_t);
template void vec_lincomb<double, double>(long long, int, const double *, long long, const double *, double *,
                                          cudaStream_t);
template void vec_lincomb<float, double>(long long, int, const float *, long long, const double *, double *,
                                         cudaStream_t);
template void vec_lincomb<float, float>(long long, int, const float *, long long, const double *, float *,
                                        cudaStream_t);
template void vec_dot<double>(long long, const double *, const double *, double *, double *, cudaStream_t);
template void vec_dot<float>(long long, const float *, const float *, double *, double *, cudaStream_t);

}  // namespace dgx
