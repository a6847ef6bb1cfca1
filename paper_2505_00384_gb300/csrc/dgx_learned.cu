// Learned preconditioner of the pressure Schur system (an extension of the
// Jacobi preconditioning of Sec. 3.1): z = D_H^-1 v + s c, c the output of a
// stack of 3x3x3 convolutions on the cell-DoF tensor.  Forward, backward-data,
// backward-weights, loss and Adam kernels for sm_103a; bfloat16 weights,
// FP32 activations and accumulation.
//
// Tensor layout: [sample][channel][Z][Y][X] FP32, X fastest, grid point
// (gx, gy, gz) holding DoF  cell (gx/n, gy/n, gz/n), node (gx%n, gy%n, gz%n).
// Each CTA of the convolution kernels owns a 4x4x4 tile of output points and
// stages the 6x6x6 halo of every input channel in shared memory.
#include <cuda_bf16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <map>
#include <set>
#include <tuple>
#include <utility>
#include <vector>

#include "dgx_common.cuh"

namespace dgx {

namespace {

constexpr int kCin = 5;                        // input channels
constexpr int kTile = 4;                       // output tile edge
constexpr int kHalo = kTile + 2;               // staged input tile edge
constexpr int kHalo3 = kHalo * kHalo * kHalo;  // 216
constexpr int kMaxBatch = 256;
constexpr int kRedBlocks = 128;  // partial sums of the feature reductions

struct Grid3 {
  int X, Y, Z, n, nx, ny;
  int tx, ty, tz;
  long long G;
  __host__ __device__ long long dof(int gx, int gy, int gz) const {
    const int cx = gx / n, a = gx - cx * n, cy = gy / n, b = gy - cy * n, cz = gz / n, cc = gz - cz * n;
    const long long cell = cx + (long long)nx * (cy + (long long)ny * cz);
    return cell * n * n * n + a + n * (b + n * cc);
  }
  __host__ __device__ int tiles() const { return tx * ty * tz; }
};

// ---------------------------------------------------------------- kernels
// Asynchronous global -> shared copies (no register round trip): every load of
// a CTA's staging phase is in flight at once.
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Same halo, one thread per halo point for all channels (the point's address
// and bounds test are computed once).
__device__ __forceinline__ void stage_halo_points(float *xs, const float *in, const Grid3 &g, int Ci, int x0,
                                                  int y0, int z0) {
  for (int l = threadIdx.x; l < kHalo3; l += blockDim.x) {
    const int gx = x0 + l % kHalo, gy = y0 + (l / kHalo) % kHalo, gz = z0 + l / (kHalo * kHalo);
    if (gx >= 0 && gx < g.X && gy >= 0 && gy < g.Y && gz >= 0 && gz < g.Z) {
      const float *src = in + gx + (long long)g.X * (gy + (long long)g.Y * gz);
      for (int ci = 0; ci < Ci; ++ci) cp_async4(xs + ci * kHalo3 + l, src + ci * g.G);
    } else {
      for (int ci = 0; ci < Ci; ++ci) xs[ci * kHalo3 + l] = 0.f;
    }
  }
}

__device__ __forceinline__ void relu_halo_points(float *xs, int Ci) {
  for (int l = threadIdx.x; l < kHalo3; l += blockDim.x)
    for (int ci = 0; ci < Ci; ++ci) xs[ci * kHalo3 + l] = fmaxf(xs[ci * kHalo3 + l], 0.f);
}

struct ConvArgs {
  Grid3 g;
  int Ci, Co;
  const float *in;
  long long in_bs;    // sample stride of the input
  const int *bidx;    // batch slot -> sample of the input (nullptr: slot itself)
  int relu_in;        // input is a pre-activation: apply max(., 0) on load
  const __nv_bfloat16 *W;  // [Ci][27][Co] bfloat16 weights, Co fastest (8-byte aligned rows of 4)
  const float *bias;  // [Co] or nullptr
  float *out;
  long long out_bs;
  const float *mask;  // nullptr, or zero the output where mask <= 0 (ReLU derivative)
  long long mask_bs;
};

// y[co][p] = b[co] + sum_ci sum_k W[co][ci][k] x[ci][p + k - 1].  16 KS
// threads: 16 rows of 4 points along x (a 4x4x4 tile) x KS input-channel
// groups; each thread keeps 4 points x COB output channels in registers and
// reuses the 6 staged inputs of its row for the three x taps.
template <int COB, int KS>
__global__ void __launch_bounds__(16 * KS) k_conv(ConvArgs a) {
  extern __shared__ __align__(16) float sm[];
  float *xs = sm;                     // [Ci][216]
  float *ws = xs + a.Ci * kHalo3;     // [Ci][27][COB]
  float *red = ws + a.Ci * 27 * COB;  // [KS][COB][64]
  const Grid3 &g = a.g;
  const int tile = blockIdx.x, co0 = blockIdx.y * COB, b = blockIdx.z;
  const int tx = tile % g.tx, ty = (tile / g.tx) % g.ty, tz = tile / (g.tx * g.ty);
  const int x0 = tx * kTile - 1, y0 = ty * kTile - 1, z0 = tz * kTile - 1;
  const long long sb = a.bidx ? a.bidx[b] : b;
  stage_halo_points(xs, a.in + sb * a.in_bs, g, a.Ci, x0, y0, z0);
  // weights: bfloat16 from global, widened to FP32 into [Ci][27][COB] while the halo copies fly
  if constexpr (COB % 4 == 0) {
#pragma unroll 4
    for (int i = threadIdx.x; i < a.Ci * 27 * (COB / 4); i += blockDim.x) {
      const int row = i / (COB / 4), part = i - row * (COB / 4);  // row = ci * 27 + k
      const uint2 u = *reinterpret_cast<const uint2 *>(a.W + (long long)row * a.Co + co0 + part * 4);
      const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.x));
      const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.y));
      *reinterpret_cast<float4 *>(ws + row * COB + part * 4) = make_float4(lo.x, lo.y, hi.x, hi.y);
    }
  } else {
    for (int i = threadIdx.x; i < a.Ci * 27 * COB; i += blockDim.x) {
      const int row = i / COB, co = i - row * COB;
      ws[i] = __bfloat162float(a.W[(long long)row * a.Co + co0 + co]);
    }
  }
  cp_async_wait_all();
  if (a.relu_in) relu_halo_points(xs, a.Ci);
  __syncthreads();
  const int r = threadIdx.x & 15, ks = threadIdx.x >> 4;
  const int py = r & 3, pz = r >> 2;
  float acc[4][COB];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int co = 0; co < COB; ++co) acc[p][co] = 0.f;
  for (int ci = ks; ci < a.Ci; ci += KS) {
#pragma unroll
    for (int dz = 0; dz < 3; ++dz)
#pragma unroll
      for (int dy = 0; dy < 3; ++dy) {
        const float2 *xr = reinterpret_cast<const float2 *>(xs + ci * kHalo3 + ((pz + dz) * kHalo + (py + dy)) * kHalo);
        const float2 u0 = xr[0], u1 = xr[1], u2 = xr[2];
        const float xv[6] = {u0.x, u0.y, u1.x, u1.y, u2.x, u2.y};
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          const float *w = ws + (ci * 27 + (dz * 3 + dy) * 3 + dx) * COB;
          float wv[COB];
          if constexpr (COB % 4 == 0) {
#pragma unroll
            for (int q = 0; q < COB / 4; ++q) {
              const float4 t = reinterpret_cast<const float4 *>(w)[q];
              wv[4 * q] = t.x;
              wv[4 * q + 1] = t.y;
              wv[4 * q + 2] = t.z;
              wv[4 * q + 3] = t.w;
            }
          } else {
#pragma unroll
            for (int co = 0; co < COB; ++co) wv[co] = w[co];
          }
#pragma unroll
          for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int co = 0; co < COB; ++co) acc[p][co] = fmaf(wv[co], xv[p + dx], acc[p][co]);
        }
      }
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int co = 0; co < COB; ++co) red[(ks * COB + co) * 64 + r * 4 + p] = acc[p][co];
  __syncthreads();
  for (int o = threadIdx.x; o < 64 * COB; o += blockDim.x) {
    const int co = o / 64, pt = o - co * 64;  // pt = row * 4 + px
    const int gx = tx * kTile + (pt & 3), gy = ty * kTile + ((pt >> 2) & 3), gz = tz * kTile + (pt >> 4);
    if (gx >= g.X || gy >= g.Y || gz >= g.Z) continue;
    float v = 0.f;
#pragma unroll
    for (int k = 0; k < KS; ++k) v += red[(k * COB + co) * 64 + pt];
    const long long gi = gx + (long long)g.X * (gy + (long long)g.Y * gz);
    if (a.bias) v += a.bias[co0 + co];
    if (a.mask && !(a.mask[b * a.mask_bs + (co0 + co) * g.G + gi] > 0.f)) v = 0.f;
    a.out[b * a.out_bs + (co0 + co) * g.G + gi] = v;
  }
}

// ---------------------------------------------------------------- tensor-core convolution
// Layers with 32 input and 32 output channels at training batch sizes run as
// implicit GEMMs on the 5th-generation tensor cores: tcgen05.mma (kind::f16,
// bf16 operands, FP32 accumulator in tensor memory), issued by one thread.
// One CTA computes M = 128 output points (a tile of 8 x 16 x 1 points in x, y,
// z) x N = 32 output channels; K runs over 27 taps x 32 input channels.
//
// The input halo (10 x 18 x 3 points) is staged once in shared memory in the
// canonical no-swizzle K-major layout: channels in chunks of 8 (16 bytes),
// chunk planes one after the other, x fastest within a plane.  Eight points
// consecutive in x then form one 8 x 16-byte core matrix, so the A operand of
// tap (dx, dy, dz) is just a descriptor at the halo point (dx, dy, dz): the
// 16 rows of 8 points are one halo row (160 bytes) apart, the two channel
// chunks of a K = 16 step one chunk plane apart.  No per-tap copy.  The
// weights are staged as [tap][chunk][co][8 channels] (B operand, K-major).
// FP32 activations are split into three bf16 terms, x = hi + mid + lo to
// 2^-24 relative (each term the bf16 rounding of what the previous ones leave);
// all three are multiplied with the (exactly bf16) weights: 162 MMAs of 128 x
// 32 x 16 per tile.  The tensor cores' FP32 accumulation does not round to
// nearest (measured: about 1e-5 relative error after 162 accumulations into one
// accumulator, consistent with truncation), so the MMAs are dealt round robin to
// 16 accumulators (all 512 TMEM columns, about 10 MMAs each) that the epilogue
// sums in FP32 on the CUDA cores.  Two bf16 terms, or one accumulator, are not
// enough for training: the backward pass's ReLU masks flip where
// pre-activations lie within ~1e-5 of zero, which moves the gradients by ~1e-3.
constexpr int kTcX = 8, kTcY = 16, kTcHX = kTcX + 2, kTcHY = kTcY + 2, kTcHZ = 3;
constexpr int kTcHP = kTcHX * kTcHY * kTcHZ;      // 540 halo points
constexpr int kTcPlane = kTcHP * 16;              // bytes of one 8-channel chunk plane
constexpr int kTcHalo = 4 * kTcPlane;             // one bf16 term of the 32 channels
constexpr int kTcTerms = 3;                       // hi, mid, lo
constexpr int kTcW = 27 * 4 * 32 * 16;            // weights
constexpr int kTcMbar = kTcTerms * kTcHalo + kTcW;  // mbarrier (8 bytes) and the TMEM address
constexpr int kTcSmem = kTcMbar + 128;
constexpr int kTcAcc = 16;                        // accumulators of 32 FP32 columns: the whole TMEM
constexpr int kTcThreads = 512;                   // 16 warps: staging loads in flight, 4 accumulators per warp
constexpr int kTcMinBatch = 8;

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle: start address, byte offset
// between core matrices along K (lbo) and along M / N (sbo), version 1.
__device__ __forceinline__ unsigned long long tc_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  return (unsigned long long)((addr >> 4) & 0x3FFFu) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, both
// K-major, N = 32, M = 128.
constexpr unsigned kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void tc_mma(unsigned dtmem, unsigned long long a, unsigned long long b, unsigned acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(kTcIdesc), "r"(acc));
}

// Bounded wait for phase `ph` of the mbarrier: false after `limit` polls.
__device__ __forceinline__ bool tc_wait(unsigned bar, unsigned ph, int limit) {
  for (int i = 0; i < limit; ++i) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok) : "r"(bar), "r"(ph) : "memory");
    if (ok) return true;
  }
  return false;
}

__global__ void __launch_bounds__(kTcThreads, 1) k_conv_tc(ConvArgs a, int *err) {
  extern __shared__ __align__(128) unsigned char tsm[];
  unsigned char *ws = tsm + kTcTerms * kTcHalo;
  unsigned long long *bar = reinterpret_cast<unsigned long long *>(tsm + kTcMbar);
  unsigned *taddr_s = reinterpret_cast<unsigned *>(tsm + kTcMbar + 8);
  const Grid3 &g = a.g;
  const int nxt = (g.X + kTcX - 1) / kTcX, nyt = (g.Y + kTcY - 1) / kTcY;
  const int tile = blockIdx.x, b = blockIdx.z;
  const int tx = tile % nxt, ty = (tile / nxt) % nyt, tz = tile / (nxt * nyt);
  const int x0 = tx * kTcX - 1, y0 = ty * kTcY - 1, z0 = tz - 1;
  const long long sb = a.bidx ? a.bidx[b] : b;
  const float *in = a.in + sb * a.in_bs;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {  // 16 x 32 TMEM columns (FP32 accumulators of N = 32), address into shared memory
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(taddr_s)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // halo: (chunk, point) items, point fastest (coalesced along x); the three
  // bf16 terms of 8 channels, each into its own copy of the halo
  for (int it = threadIdx.x; it < 4 * kTcHP; it += blockDim.x) {
    const int c = it / kTcHP, pnt = it - c * kTcHP;
    const int hx = pnt % kTcHX, hy = (pnt / kTcHX) % kTcHY, hz = pnt / (kTcHX * kTcHY);
    const int gx = x0 + hx, gy = y0 + hy, gz = z0 + hz;
    unsigned short t[kTcTerms][8];
    if (gx >= 0 && gx < g.X && gy >= 0 && gy < g.Y && gz >= 0 && gz < g.Z) {
      const float *src = in + (long long)(8 * c) * g.G + gx + (long long)g.X * (gy + (long long)g.Y * gz);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float v = src[(long long)j * g.G];
        if (a.relu_in) v = fmaxf(v, 0.f);
#pragma unroll
        for (int q = 0; q < kTcTerms; ++q) {  // v - (terms so far) is exact in FP32
          const __nv_bfloat16 tq = __float2bfloat16_rn(v);
          t[q][j] = __bfloat16_as_ushort(tq);
          v -= __bfloat162float(tq);
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < kTcTerms; ++q)
#pragma unroll
        for (int j = 0; j < 8; ++j) t[q][j] = 0;
    }
#pragma unroll
    for (int q = 0; q < kTcTerms; ++q) {
      uint4 u;
      u.x = t[q][0] | ((unsigned)t[q][1] << 16); u.y = t[q][2] | ((unsigned)t[q][3] << 16);
      u.z = t[q][4] | ((unsigned)t[q][5] << 16); u.w = t[q][6] | ((unsigned)t[q][7] << 16);
      *reinterpret_cast<uint4 *>(tsm + q * kTcHalo + c * kTcPlane + pnt * 16) = u;
    }
  }
  // weights W[(ci 27 + tap) Co + co] -> [tap][ci / 8][co][ci % 8]; co fastest across threads
  for (int it = threadIdx.x; it < 27 * 4 * 32; it += blockDim.x) {
    const int co = it % 32, c = (it / 32) % 4, tap = it / 128;
    unsigned short w[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) w[j] = __bfloat16_as_ushort(a.W[((long long)(8 * c + j) * 27 + tap) * 32 + co]);
    uint4 u;
    u.x = w[0] | ((unsigned)w[1] << 16); u.y = w[2] | ((unsigned)w[3] << 16);
    u.z = w[4] | ((unsigned)w[5] << 16); u.w = w[6] | ((unsigned)w[7] << 16);
    *reinterpret_cast<uint4 *>(ws + ((tap * 4 + c) * 32 + co) * 16) = u;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = *taddr_s;
  if (threadIdx.x == 0) {
    int i = 0;  // MMA count: accumulator i % kTcAcc, overwritten by its first MMA
    for (int part = 0; part < kTcTerms; ++part) {
      const unsigned base = smem_u32(tsm + part * kTcHalo);
      for (int tap = 0; tap < 27; ++tap) {
        const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
        const unsigned aoff = ((dz * kTcHY + dy) * kTcHX + dx) * 16;
        for (int ks = 0; ks < 2; ++ks, ++i) {
          const unsigned long long ad = tc_desc(base + 2 * ks * kTcPlane + aoff, kTcPlane, kTcHX * 16);
          const unsigned long long bd = tc_desc(smem_u32(ws) + (tap * 4 + 2 * ks) * 512, 512, 128);
          tc_mma(tmem + (unsigned)(i % kTcAcc) * 32, ad, bd, i >= kTcAcc ? 1u : 0u);
        }
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
  }
  // every thread polls (bounded); the CTA goes on only if all saw completion
  const bool ok = __syncthreads_and(tc_wait(smem_u32(bar), 0, 1 << 22));
  if (!ok && threadIdx.x == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    // warp w reads TMEM lanes 32 (w % 4) .. +31 (its lane quarter) of accumulators
    // 4 (w / 4) .. +3 and sums them in FP32; the four partial sums of every output
    // meet in shared memory (the halo's space: the MMAs that read it are complete)
    const int q = warp & 3, grp = warp >> 2;
    float sum[32];
#pragma unroll
    for (int co = 0; co < 32; ++co) sum[co] = 0.f;
    for (int acc = grp * 4; acc < grp * 4 + 4; ++acc) {
      unsigned r[32];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
          "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
            "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(tmem + ((unsigned)(q * 32) << 16) + (unsigned)acc * 32));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int co = 0; co < 32; ++co) sum[co] += __uint_as_float(r[co]);
    }
    float *red = reinterpret_cast<float *>(tsm);  // [group][co][m], 64 KB
    const int m = q * 32 + lane;
#pragma unroll
    for (int co = 0; co < 32; ++co) red[(grp * 32 + co) * 128 + m] = sum[co];
  }
  __syncthreads();
  if (ok) {
    // output (co, m) per thread, m fastest: row m of D is the point (x0 + 1 + m % 8, y0 + 1 + m / 8, z0 + 1)
    const float *red = reinterpret_cast<const float *>(tsm);
    for (int o = threadIdx.x; o < 32 * 128; o += blockDim.x) {
      const int co = o >> 7, m = o & 127;
      const int gx = x0 + 1 + (m & 7), gy = y0 + 1 + (m >> 3), gz = z0 + 1;
      if (gx >= g.X || gy >= g.Y) continue;
      const long long gi = gx + (long long)g.X * (gy + (long long)g.Y * gz);
      float v = ((red[co * 128 + m] + red[(32 + co) * 128 + m]) + red[(64 + co) * 128 + m]) + red[(96 + co) * 128 + m];
      if (a.bias) v += a.bias[co];
      if (a.mask && !(a.mask[b * a.mask_bs + co * g.G + gi] > 0.f)) v = 0.f;
      a.out[b * a.out_bs + co * g.G + gi] = v;
    }
  }
  // after a timeout the MMAs may still be writing TMEM: give them a second
  // bounded wait before the columns are freed
  if (!ok && warp == 0) tc_wait(smem_u32(bar), 0, 1 << 22);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

struct WgArgs {
  Grid3 g;
  int Ci, Co;
  const float *x;  // layer input
  long long x_bs;
  const int *bidx;
  int relu_in;
  const float *gy;  // gradient w.r.t. the layer's pre-activation, [slot][Co][G]
  long long gy_bs;
  int items, per;  // (slot, tile) items, items per chunk
  float *part;     // [chunk][Co Ci 27 + Co]
};

// Partial weight and bias gradients of one chunk of (slot, tile) items for
// COB output channels: dW[co][ci][k] = sum_p gy[co][p] x[ci][p + k - 1].
// Thread w < 9 Ci owns (ci, kz, ky) and the three kx taps.
template <int COB>
__global__ void __launch_bounds__(576) k_wgrad(WgArgs a) {
  extern __shared__ __align__(16) float sm[];
  float *xs = sm;                  // [Ci][216]
  float *gs = xs + a.Ci * kHalo3;  // [64][COB]
  const Grid3 &g = a.g;
  const int co0 = blockIdx.x * COB, chunk = blockIdx.y;
  const int w = threadIdx.x;
  const bool active = w < a.Ci * 9;
  const int ci = w / 9, kz = (w % 9) / 3, ky = w % 3;
  float acc[3][COB], bacc[COB];
#pragma unroll
  for (int co = 0; co < COB; ++co) {
    acc[0][co] = acc[1][co] = acc[2][co] = 0.f;
    bacc[co] = 0.f;
  }
  const int nt = g.tiles();
  const int it0 = chunk * a.per, it1 = min(a.items, it0 + a.per);
  for (int it = it0; it < it1; ++it) {
    const int b = it / nt, tile = it - b * nt;
    const int tx = tile % g.tx, ty = (tile / g.tx) % g.ty, tz = tile / (g.tx * g.ty);
    const int x0 = tx * kTile - 1, y0 = ty * kTile - 1, z0 = tz * kTile - 1;
    const long long sb = a.bidx ? a.bidx[b] : b;
    __syncthreads();  // the previous item is done with the staging buffers
    stage_halo_points(xs, a.x + sb * a.x_bs, g, a.Ci, x0, y0, z0);
    for (int i = threadIdx.x; i < 64 * COB; i += blockDim.x) {
      const int p = i / COB, co = i % COB;
      const int gx = tx * kTile + (p & 3), gy = ty * kTile + ((p >> 2) & 3), gz = tz * kTile + (p >> 4);
      if (gx < g.X && gy < g.Y && gz < g.Z)
        cp_async4(gs + i, a.gy + b * a.gy_bs + (co0 + co) * g.G + gx + (long long)g.X * (gy + (long long)g.Y * gz));
      else
        gs[i] = 0.f;
    }
    cp_async_wait_all();
    if (a.relu_in) relu_halo_points(xs, a.Ci);
    __syncthreads();
    if (active) {
      for (int p = 0; p < 64; ++p) {
        const int px = p & 3, py = (p >> 2) & 3, pz = p >> 4;
        const float *xr = xs + ci * kHalo3 + ((pz + kz) * kHalo + (py + ky)) * kHalo + px;
        const float x0v = xr[0], x1v = xr[1], x2v = xr[2];
#pragma unroll
        for (int co = 0; co < COB; ++co) {
          const float gv = gs[p * COB + co];
          acc[0][co] = fmaf(gv, x0v, acc[0][co]);
          acc[1][co] = fmaf(gv, x1v, acc[1][co]);
          acc[2][co] = fmaf(gv, x2v, acc[2][co]);
        }
      }
      if (w == 0)
        for (int p = 0; p < 64; ++p)
#pragma unroll
          for (int co = 0; co < COB; ++co) bacc[co] += gs[p * COB + co];
    }
  }
  float *P = a.part + (long long)chunk * ((long long)a.Co * a.Ci * 27 + a.Co);
  if (active) {
#pragma unroll
    for (int co = 0; co < COB; ++co)
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) P[((long long)(co0 + co) * a.Ci + ci) * 27 + (kz * 3 + ky) * 3 + kx] = acc[kx][co];
  }
  if (w == 0) {
#pragma unroll
    for (int co = 0; co < COB; ++co) P[(long long)a.Co * a.Ci * 27 + co0 + co] = bacc[co];
  }
}

struct AdamArgs {
  int Ci, Co, chunks, update;
  long long stride;  // per-chunk stride of the partials
  const float *part;
  float *grad, *master, *m, *v;  // layer slices (W then b)
  __nv_bfloat16 *wbf, *wtbf;     // layer weights [Ci][27][Co], and [Co][27][Ci] with flipped taps
  float lr, b1, b2, eps, c1, c2;  // c1 = 1/(1-b1^t), c2 = 1/(1-b2^t)
};

// Sum the chunk partials (fixed order) into the gradient and, with update,
// take one Adam step (Kingma & Ba 2015) on the FP32 master copy.
__global__ void k_adam(AdamArgs a) {
  const long long nW = (long long)a.Co * a.Ci * 27, n = nW + a.Co;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    float gsum = 0.f;
    for (int k = 0; k < a.chunks; ++k) gsum += a.part[k * a.stride + e];
    a.grad[e] = gsum;
    if (!a.update) continue;
    const float m = a.b1 * a.m[e] + (1.f - a.b1) * gsum;
    const float v = a.b2 * a.v[e] + (1.f - a.b2) * gsum * gsum;
    a.m[e] = m;
    a.v[e] = v;
    const float th = a.master[e] - a.lr * (m * a.c1) / (sqrtf(v * a.c2) + a.eps);
    a.master[e] = th;
    if (e < nW) {
      const int co = (int)(e / (a.Ci * 27)), ci = (int)((e / 27) % a.Ci), k = (int)(e % 27);
      const __nv_bfloat16 hb = __float2bfloat16_rn(th);
      a.wbf[((long long)ci * 27 + k) * a.Co + co] = hb;
      a.wtbf[((long long)co * 27 + 26 - k) * a.Ci + ci] = hb;
    }
  }
}

// bfloat16 weights of a layer from its FP32 master copy ([co][ci][k] ->
// [ci][k][co]), and the transposed copy with flipped taps ([co][26-k][ci]) used
// by the backward-data convolution: the layouts the convolution kernel stages.
__global__ void k_round_weights(int Ci, int Co, const float *master, __nv_bfloat16 *wbf, __nv_bfloat16 *wtbf) {
  const long long nW = (long long)Co * Ci * 27;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nW; e += (long long)gridDim.x * blockDim.x) {
    const int co = (int)(e / (Ci * 27)), ci = (int)((e / 27) % Ci), k = (int)(e % 27);
    const __nv_bfloat16 hb = __float2bfloat16_rn(master[e]);
    wbf[((long long)ci * 27 + k) * Co + co] = hb;
    wtbf[((long long)co * 27 + 26 - k) * Ci + ci] = hb;
  }
}

__device__ __forceinline__ double block_sum(double v, double *sh) {
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

// Channel 0 before scaling: j = dinv .* v gathered to the grid; partial sums of j^2.
template <typename T>
__global__ void k_feat_j(Grid3 g, const T *__restrict__ v, const double *__restrict__ dinv, float *__restrict__ ch0,
                         double *__restrict__ part) {
  __shared__ double sh[32];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.G; i += (long long)gridDim.x * blockDim.x) {
    const int gx = (int)(i % g.X), gy = (int)((i / g.X) % g.Y), gz = (int)(i / ((long long)g.X * g.Y));
    const long long d = g.dof(gx, gy, gz);
    const double j = dinv[d] * (double)v[d];
    ch0[i] = (float)j;
    s += j * j;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// s = rms(j) (every block reduces the partials in the same order); ch0 /= s;
// with e: t = e / s gathered to the grid and partial sums of t^2.
__global__ void k_feat_scale(Grid3 g, const double *__restrict__ part, int nblk, float *__restrict__ ch0,
                             const double *__restrict__ e, float *__restrict__ t, double *__restrict__ tpart,
                             double *__restrict__ s_out) {
  __shared__ double sh[32];
  __shared__ double s_sh;
  if (threadIdx.x == 0) {
    double s2 = 0.0;
    for (int k = 0; k < nblk; ++k) s2 += part[k];
    const double s = sqrt(s2 / (double)g.G);
    s_sh = s > 0.0 ? s : 1.0;
    if (blockIdx.x == 0 && s_out) *s_out = s_sh;
  }
  __syncthreads();
  const double s = s_sh;
  const float inv = (float)(1.0 / s);
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.G; i += (long long)gridDim.x * blockDim.x) {
    ch0[i] *= inv;
    if (e) {
      const int gx = (int)(i % g.X), gy = (int)((i / g.X) % g.Y), gz = (int)(i / ((long long)g.X * g.Y));
      const float tv = (float)(e[g.dof(gx, gy, gz)] / s);
      t[i] = tv;
      acc += (double)tv * tv;
    }
  }
  if (e) {
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) tpart[blockIdx.x] = acc;
  }
}

__global__ void k_sum_to(const double *__restrict__ part, int n, float *__restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += part[k];
    *out = (float)s;
  }
}

// Coefficient channels 1..4 (sums: sum d, sum p_k, sum rho on the device).
__global__ void k_feat_coef(Grid3 g, const double *__restrict__ d, const double *__restrict__ pk,
                            const double *__restrict__ rho, const float *__restrict__ hn,
                            const double *__restrict__ sums, float *__restrict__ ch) {
  const double md = sums[0] / (double)g.G, mp = sums[1] / (double)g.G, mr = sums[2] / (double)g.G;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.G; i += (long long)gridDim.x * blockDim.x) {
    const int gx = (int)(i % g.X), gy = (int)((i / g.X) % g.Y), gz = (int)(i / ((long long)g.X * g.Y));
    const long long q = g.dof(gx, gy, gz);
    ch[i] = (float)log(d[q] / md);
    ch[g.G + i] = (float)(pk[q] / mp - 1.0);
    ch[2 * g.G + i] = (float)(rho[q] / mr - 1.0);
    ch[3 * g.G + i] = hn[q];
  }
}

// z = dinv .* v + s c, scattered back to DoF order.
template <typename T>
__global__ void k_learn_out(Grid3 g, const T *__restrict__ v, const double *__restrict__ dinv,
                            const float *__restrict__ c, const double *__restrict__ s, T *__restrict__ z) {
  const double sv = *s;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.G; i += (long long)gridDim.x * blockDim.x) {
    const int gx = (int)(i % g.X), gy = (int)((i / g.X) % g.Y), gz = (int)(i / ((long long)g.X * g.Y));
    const long long d = g.dof(gx, gy, gz);
    z[d] = (T)(dinv[d] * (double)v[d] + sv * (double)c[i]);
  }
}

// Loss of a batch: e = ch0 + c - t; gout = 2 e / (B ||t||^2); per-block sums
// of e^2 / ||t||^2.
__global__ void k_loss(long long G, int B, const float *__restrict__ c, const float *__restrict__ ds, long long ss,
                       const int *__restrict__ bidx, const float *__restrict__ tn2, float *__restrict__ gout,
                       double *__restrict__ lpart) {
  __shared__ double sh[32];
  const int b = blockIdx.y;
  const long long s = bidx[b];
  const float *ch0 = ds + s * ss, *t = ds + s * ss + (long long)kCin * G;
  const float w = 2.f / ((float)B * tn2[s]);
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < G; i += (long long)gridDim.x * blockDim.x) {
    const float e = ch0[i] + c[b * G + i] - t[i];
    gout[b * G + i] = w * e;
    acc += (double)e * e;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) lpart[b * gridDim.x + blockIdx.x] = acc / (double)tn2[s];
}

__global__ void k_fill_d(long long n, double v, double *x) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = v;
}

int blocks_for(long long n, int cap = 4 * 152) {
  return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, cap));
}

// Opt in to large dynamic shared memory once per (device, kernel).
int prep(dgx_ctx *c, const void *fn) {
  static std::mutex mu;
  static std::set<std::pair<int, const void *>> done;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({c->device, fn})) return 0;
  if (int e = check_cuda(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024),
                         "cudaFuncSetAttribute"))
    return e;
  done.insert({c->device, fn});
  return 0;
}

// host PRNG: splitmix64 (Steele, Lea & Flood 2014) and Box-Muller
struct SplitMix {
  unsigned long long s;
  unsigned long long next() {
    unsigned long long z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
  double normal() {
    const double u1 = uniform(), u2 = uniform();
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  }
};

}  // namespace

struct Learned {
  // network
  int L = 0, C = 0;
  std::vector<int> ci, co;
  std::vector<long long> poff, woff;  // layer offsets: parameter vector, bf16 weights
  long long P = 0, nW = 0;
  float *master = nullptr, *am = nullptr, *av = nullptr, *grad = nullptr;
  __nv_bfloat16 *wbf = nullptr;
  __nv_bfloat16 *wtbf = nullptr;
  // CUDA graphs of the apply, per (v, z, type); replayed on a private stream
  struct GraphRec {
    cudaGraphExec_t exec;
    long long launches;
  };
  std::map<std::tuple<const void *, void *, int>, GraphRec> graphs;
  cudaStream_t gstream = nullptr;
  cudaEvent_t gev0 = nullptr, gev1 = nullptr;
  int adam_t = 0;
  // mesh-dependent
  bool has_grid = false;
  Grid3 g{};
  float *hnode = nullptr;     // h / Lz per DoF
  float *live = nullptr;      // (kCin + 1) G: features of the current apply
  long long live_version = -1;
  double *ones = nullptr;     // N ones (means of the coefficient fields)
  double *scal = nullptr;     // [0..2] sums, [3] s, partials after
  float *iact = nullptr;      // inference activations, 2 x C G (ping-pong)
  // dataset: samples of (kCin + 1) G floats
  float *ds = nullptr;
  float *tn2 = nullptr;
  long long ds_cap = 0, ds_n = 0;
  std::vector<char> is_test;
  // training buffers
  int tB = 0;
  float *tact = nullptr, *tg0 = nullptr, *tg1 = nullptr, *wpart = nullptr;
  long long wpart_elems = 0;
  int *bidx = nullptr;
  long long bidx_cap = 0;
  double *lpart = nullptr;
  double *host_lpart = nullptr;
  int *tc_err = nullptr;  // set by a tensor-core convolution whose MMAs did not complete in time
};

namespace {

// Buffers of the current mesh (terrain channel, live features, inference activations).
void free_graphs(Learned *m);

void free_grid(Learned *m) {
  free_graphs(m);
  for (void *p : {(void *)m->hnode, (void *)m->live, (void *)m->ones, (void *)m->scal, (void *)m->iact})
    if (p) cudaFree(p);
  m->hnode = m->live = m->iact = nullptr;
  m->ones = m->scal = nullptr;
  m->has_grid = false;
  m->live_version = -1;
}

// Samples and training buffers: they depend on the grid extents only, so they
// survive a new mesh of the same extents (e.g. another terrain).
void free_dataset(Learned *m) {
  for (void *p : {(void *)m->ds, (void *)m->tn2, (void *)m->tact, (void *)m->tg0, (void *)m->tg1,
                  (void *)m->wpart, (void *)m->bidx, (void *)m->lpart})
    if (p) cudaFree(p);
  if (m->host_lpart) cudaFreeHost(m->host_lpart);
  m->ds = m->tn2 = m->tact = m->tg0 = m->tg1 = m->wpart = nullptr;
  m->lpart = m->host_lpart = nullptr;
  m->bidx = nullptr;
  m->ds_cap = m->ds_n = 0;
  m->is_test.clear();
  m->tB = 0;
  m->wpart_elems = 0;
  m->bidx_cap = 0;
}

void free_graphs(Learned *m) {
  for (auto &kv : m->graphs) cudaGraphExecDestroy(kv.second.exec);
  m->graphs.clear();
}

void free_net(Learned *m) {
  free_graphs(m);
  for (void *p : {(void *)m->master, (void *)m->am, (void *)m->av, (void *)m->grad, (void *)m->wbf, (void *)m->wtbf,
                  (void *)m->tc_err})
    if (p) cudaFree(p);
  m->tc_err = nullptr;
  m->master = m->am = m->av = m->grad = nullptr;
  m->wtbf = nullptr;
  m->wbf = nullptr;
  if (m->gev0) cudaEventDestroy(m->gev0);
  if (m->gev1) cudaEventDestroy(m->gev1);
  if (m->gstream) cudaStreamDestroy(m->gstream);
  m->gev0 = m->gev1 = nullptr;
  m->gstream = nullptr;
}

template <typename T>
int dmalloc(dgx_ctx *c, T **p, size_t elems) {
  *p = nullptr;
  void *q = nullptr;
  if (int e = check_cuda(c, cudaMalloc(&q, std::max<size_t>(1, elems) * sizeof(T)), "cudaMalloc (learned)")) return e;
  *p = reinterpret_cast<T *>(q);
  return 0;
}

// Error flag of the tensor-core convolutions (read after a synchronisation):
// DGX_ERR_DEVICE_TIMEOUT (and the flag cleared) when an MMA batch did not complete.
int tc_status(dgx_ctx *c) {
  Learned *m = c->learned;
  if (!m || !m->tc_err) return 0;
  int flag = 0;
  if (int e = check_cuda(c, cudaMemcpy(&flag, m->tc_err, sizeof(int), cudaMemcpyDeviceToHost), "tensor-core status"))
    return e;
  if (!flag) return 0;
  cudaMemset(m->tc_err, 0, sizeof(int));
  return set_error(c, DGX_ERR_DEVICE_TIMEOUT, "tensor-core convolution: MMAs did not complete within the wait limit");
}

// Host-to-device copy ordered on the context's stream; returns when done.
int h2d(dgx_ctx *c, void *dst, const void *src, size_t bytes, const char *what) {
  if (int e = check_cuda(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream), what)) return e;
  return check_cuda(c, cudaStreamSynchronize(c->stream), what);
}

int need_net(dgx_ctx *c) {
  if (!c->learned || !c->learned->master) return set_error(c, DGX_ERR_STATE, "no network (call dgx_learned_create)");
  return 0;
}

// Mesh-dependent buffers: grid description, terrain channel, live features.
int ensure_grid(dgx_ctx *c) {
  Learned *m = c->learned;
  if (m->has_grid) return 0;
  Grid3 g{};
  g.n = c->n;
  g.nx = c->mesh.nx;
  g.ny = c->mesh.ny;
  g.X = c->mesh.nx * c->n;
  g.Y = c->mesh.ny * c->n;
  g.Z = c->mesh.nz * c->n;
  g.tx = (g.X + kTile - 1) / kTile;
  g.ty = (g.Y + kTile - 1) / kTile;
  g.tz = (g.Z + kTile - 1) / kTile;
  g.G = (long long)g.X * g.Y * g.Z;
  if (m->g.X != g.X || m->g.Y != g.Y || m->g.Z != g.Z) free_dataset(m);
  std::vector<double> h;
  node_terrain_heights(c, h);
  std::vector<float> hf(h.size());
  for (size_t i = 0; i < h.size(); ++i) hf[i] = (float)(h[i] / c->mesh.Lz);
  int e;
  if ((e = dmalloc(c, &m->hnode, g.G)) || (e = dmalloc(c, &m->live, (size_t)(kCin + 1) * g.G)) ||
      (e = dmalloc(c, &m->ones, g.G)) || (e = dmalloc(c, &m->scal, 8 + 2 * kRedBlocks)) ||
      (e = dmalloc(c, &m->iact, (size_t)2 * std::max(m->C, 1) * g.G)))
    return e;
  if ((e = h2d(c, m->hnode, hf.data(), hf.size() * sizeof(float), "upload terrain channel"))) return e;
  count_launch();
  k_fill_d<<<blocks_for(g.G), 256, 0, c->stream>>>(g.G, 1.0, m->ones);
  m->g = g;
  m->has_grid = true;
  m->live_version = -1;
  return check_cuda(c, cudaGetLastError(), "learned grid");
}

// Coefficient channels of the live feature buffer for the current coefficients.
int ensure_coef_features(dgx_ctx *c) {
  Learned *m = c->learned;
  if (int e = ensure_diag(c, true)) return e;  // the Helmholtz diagonal in FP64
  if (m->live_version == c->coef_version) return 0;
  const long long G = m->g.G;
  vec_dot<double>(G, c->diag64[DGX_PC_HELMHOLTZ], m->ones, c->red, m->scal + 0, c->stream);
  vec_dot<double>(G, c->pk64, m->ones, c->red, m->scal + 1, c->stream);
  vec_dot<double>(G, c->rho64, m->ones, c->red, m->scal + 2, c->stream);
  count_launch();
  k_feat_coef<<<blocks_for(G), 256, 0, c->stream>>>(m->g, c->diag64[DGX_PC_HELMHOLTZ], c->pk64, c->rho64, m->hnode,
                                                     m->scal, m->live + G);
  if (int e = check_cuda(c, cudaGetLastError(), "k_feat_coef")) return e;
  m->live_version = c->coef_version;
  return 0;
}

// Channel 0 (and, with e, the target) of `dst` (kCin + 1) G from v; s on the device at m->scal[3].
template <typename T>
int features(dgx_ctx *c, const T *v, const double *e, float *dst, float *tn2_out) {
  Learned *m = c->learned;
  const long long G = m->g.G;
  const int nb = blocks_for(G, kRedBlocks);
  double *part = m->scal + 8, *tpart = m->scal + 8 + kRedBlocks;
  count_launch(2);
  k_feat_j<T><<<nb, 256, 0, c->stream>>>(m->g, v, c->dinv64[DGX_PC_HELMHOLTZ], dst, part);
  k_feat_scale<<<nb, 256, 0, c->stream>>>(m->g, part, nb, dst, e, e ? dst + (long long)kCin * G : nullptr, tpart,
                                          m->scal + 3);
  if (e) {
    count_launch();
    k_sum_to<<<1, 32, 0, c->stream>>>(tpart, nb, tn2_out);
  }
  return check_cuda(c, cudaGetLastError(), "learned features");
}

size_t conv_smem(int Ci, int cob, int ks) { return (size_t)(Ci * kHalo3 + Ci * 27 * cob + ks * cob * 64) * sizeof(float); }

template <int COB, int KS>
int launch_conv_t(dgx_ctx *c, const ConvArgs &a, int B) {
  if (int e = prep(c, (const void *)k_conv<COB, KS>)) return e;
  count_launch();
  k_conv<COB, KS><<<dim3(a.g.tiles(), a.Co / COB, B), 16 * KS, conv_smem(a.Ci, COB, KS), c->stream>>>(a);
  return check_cuda(c, cudaGetLastError(), "k_conv");
}

// Hidden layers: 8 output channels x 8 channel groups per CTA when the grid
// of CTAs fills the GPU several times over (training batches), else 4 x 16
// (more, shorter threads for single-sample inference); output layer 1 x 16.
int launch_conv(dgx_ctx *c, const ConvArgs &a, int B) {
  if (a.Ci == 32 && a.Co == 32 && B >= kTcMinBatch) {  // training batches: tensor cores
    Learned *m = c->learned;
    if (int e = prep(c, (const void *)k_conv_tc)) return e;
    const int tiles = ((a.g.X + kTcX - 1) / kTcX) * ((a.g.Y + kTcY - 1) / kTcY) * a.g.Z;
    count_launch();
    k_conv_tc<<<dim3(tiles, 1, B), kTcThreads, kTcSmem, c->stream>>>(a, m->tc_err);
    return check_cuda(c, cudaGetLastError(), "k_conv_tc");
  }
  if (a.Co % 8 == 0 && (long long)a.g.tiles() * (a.Co / 8) * B >= 4 * 152) return launch_conv_t<8, 8>(c, a, B);
  if (a.Co % 4 == 0) return launch_conv_t<4, 16>(c, a, B);
  return launch_conv_t<1, 16>(c, a, B);
}

int wgrad_chunks(int items, int cogroups) {
  const int target = std::max(1, (2 * 152) / std::max(1, cogroups));
  return std::max(1, std::min(items, target));
}

int launch_wgrad(dgx_ctx *c, WgArgs a, int B, int *chunks_out) {
  Learned *m = c->learned;
  const int cob = a.Co % 8 == 0 ? 8 : 1;
  const int groups = a.Co / cob;
  a.items = B * a.g.tiles();
  const int chunks = wgrad_chunks(a.items, groups);
  a.per = (a.items + chunks - 1) / chunks;
  const long long need = (long long)chunks * ((long long)a.Co * a.Ci * 27 + a.Co);
  if (need > m->wpart_elems) {
    if (m->wpart) cudaFree(m->wpart);
    m->wpart = nullptr;
    m->wpart_elems = 0;
    if (int e = dmalloc(c, &m->wpart, (size_t)need)) return e;
    m->wpart_elems = need;
  }
  a.part = m->wpart;
  const int threads = 32 * ((a.Ci * 9 + 31) / 32);
  const size_t sm = (size_t)(a.Ci * kHalo3 + 64 * cob) * sizeof(float);
  count_launch();
  if (cob == 8) {
    if (int e = prep(c, (const void *)k_wgrad<8>)) return e;
    k_wgrad<8><<<dim3(groups, chunks), threads, sm, c->stream>>>(a);
  } else {
    if (int e = prep(c, (const void *)k_wgrad<1>)) return e;
    k_wgrad<1><<<dim3(groups, chunks), threads, sm, c->stream>>>(a);
  }
  *chunks_out = chunks;
  return check_cuda(c, cudaGetLastError(), "k_wgrad");
}

// Network forward on one sample held in `src` ((kCin + 1) G layout); output channel in out (G).
int net_forward1(dgx_ctx *c, const float *src, float **out) {
  Learned *m = c->learned;
  const long long G = m->g.G;
  const float *in = src;
  long long in_bs = (long long)(kCin + 1) * G;
  for (int l = 0; l < m->L; ++l) {
    float *dst = m->iact + (size_t)(l & 1) * m->C * G;
    ConvArgs a{};
    a.g = m->g;
    a.Ci = m->ci[l];
    a.Co = m->co[l];
    a.in = in;
    a.in_bs = in_bs;
    a.bidx = nullptr;
    a.relu_in = l > 0;
    a.W = m->wbf + m->woff[l];
    a.bias = m->master + m->poff[l] + (long long)a.Co * a.Ci * 27;
    a.out = dst;
    a.out_bs = (long long)a.Co * G;
    if (int e = launch_conv(c, a, 1)) return e;
    in = dst;
    in_bs = (long long)a.Co * G;
  }
  *out = const_cast<float *>(in);
  return 0;
}

int ensure_train_buffers(dgx_ctx *c, int B) {
  Learned *m = c->learned;
  if (m->tB >= B) return 0;
  for (void *p : {(void *)m->tact, (void *)m->tg0, (void *)m->tg1, (void *)m->lpart})
    if (p) cudaFree(p);
  if (m->host_lpart) cudaFreeHost(m->host_lpart);
  m->tact = m->tg0 = m->tg1 = nullptr;
  m->lpart = m->host_lpart = nullptr;
  m->tB = 0;
  const long long G = m->g.G;
  size_t acts = 0;
  for (int l = 0; l < m->L; ++l) acts += (size_t)B * m->co[l] * G;
  int e;
  if ((e = dmalloc(c, &m->tact, acts)) || (e = dmalloc(c, &m->tg0, (size_t)B * m->C * G)) ||
      (e = dmalloc(c, &m->tg1, (size_t)B * m->C * G)) || (e = dmalloc(c, &m->lpart, (size_t)B * kRedBlocks)))
    return e;
  if ((e = check_cuda(c, cudaMallocHost(&m->host_lpart, (size_t)B * kRedBlocks * sizeof(double)), "cudaMallocHost")))
    return e;
  m->tB = B;
  return 0;
}

float *act_of(Learned *m, int l, int B) {
  size_t off = 0;
  for (int k = 0; k < l; ++k) off += (size_t)B * m->co[k] * m->g.G;
  return m->tact + off;
}

// Forward and loss of a batch whose sample indices are at bidx (device).
int batch_forward_loss(dgx_ctx *c, const int *bidx, int B) {
  Learned *m = c->learned;
  const long long G = m->g.G, ss = (long long)(kCin + 1) * G;
  for (int l = 0; l < m->L; ++l) {
    ConvArgs a{};
    a.g = m->g;
    a.Ci = m->ci[l];
    a.Co = m->co[l];
    if (l == 0) {
      a.in = m->ds;
      a.in_bs = ss;
      a.bidx = bidx;
      a.relu_in = 0;
    } else {
      a.in = act_of(m, l - 1, B);
      a.in_bs = (long long)m->co[l - 1] * G;
      a.relu_in = 1;
    }
    a.W = m->wbf + m->woff[l];
    a.bias = m->master + m->poff[l] + (long long)a.Co * a.Ci * 27;
    a.out = act_of(m, l, B);
    a.out_bs = (long long)a.Co * G;
    if (int e = launch_conv(c, a, B)) return e;
  }
  const int nb = blocks_for(G, kRedBlocks);
  count_launch();
  k_loss<<<dim3(nb, B), 256, 0, c->stream>>>(G, B, act_of(m, m->L - 1, B), m->ds, ss, bidx, m->tn2, m->tg0,
                                             m->lpart);
  return check_cuda(c, cudaGetLastError(), "k_loss");
}

// Backward of the batch after batch_forward_loss; update = Adam step, else
// gradients only (into m->grad).
int batch_backward(dgx_ctx *c, const int *bidx, int B, bool update, float lr, float b1, float b2, float eps) {
  Learned *m = c->learned;
  const long long G = m->g.G, ss = (long long)(kCin + 1) * G;
  float *gcur = m->tg0, *gnext = m->tg1;
  if (update) ++m->adam_t;
  const float c1 = update ? (float)(1.0 / (1.0 - std::pow((double)b1, m->adam_t))) : 1.f;
  const float c2 = update ? (float)(1.0 / (1.0 - std::pow((double)b2, m->adam_t))) : 1.f;
  for (int l = m->L - 1; l >= 0; --l) {
    WgArgs w{};
    w.g = m->g;
    w.Ci = m->ci[l];
    w.Co = m->co[l];
    if (l == 0) {
      w.x = m->ds;
      w.x_bs = ss;
      w.bidx = bidx;
      w.relu_in = 0;
    } else {
      w.x = act_of(m, l - 1, B);
      w.x_bs = (long long)m->co[l - 1] * G;
      w.relu_in = 1;
    }
    w.gy = gcur;
    w.gy_bs = (long long)w.Co * G;
    int chunks = 0;
    if (int e = launch_wgrad(c, w, B, &chunks)) return e;
    if (l > 0) {
      ConvArgs a{};
      a.g = m->g;
      a.Ci = m->co[l];
      a.Co = m->ci[l];
      a.in = gcur;
      a.in_bs = (long long)m->co[l] * G;
      a.relu_in = 0;
      a.W = m->wtbf + m->woff[l];
      a.bias = nullptr;
      a.out = gnext;
      a.out_bs = (long long)m->ci[l] * G;
      a.mask = act_of(m, l - 1, B);
      a.mask_bs = (long long)m->ci[l] * G;
      if (int e = launch_conv(c, a, B)) return e;
    }
    AdamArgs ad{};
    ad.Ci = m->ci[l];
    ad.Co = m->co[l];
    ad.chunks = chunks;
    ad.update = update ? 1 : 0;
    ad.stride = (long long)ad.Co * ad.Ci * 27 + ad.Co;
    ad.part = m->wpart;
    ad.grad = m->grad + m->poff[l];
    ad.master = m->master + m->poff[l];
    ad.m = m->am + m->poff[l];
    ad.v = m->av + m->poff[l];
    ad.wbf = m->wbf + m->woff[l];
    ad.wtbf = m->wtbf + m->woff[l];
    ad.lr = lr;
    ad.b1 = b1;
    ad.b2 = b2;
    ad.eps = eps;
    ad.c1 = c1;
    ad.c2 = c2;
    count_launch();
    k_adam<<<blocks_for(ad.stride), 256, 0, c->stream>>>(ad);
    if (int e = check_cuda(c, cudaGetLastError(), "k_adam")) return e;
    std::swap(gcur, gnext);
  }
  return 0;
}

int ensure_bidx(dgx_ctx *c, long long n) {
  Learned *m = c->learned;
  if (m->bidx_cap >= n) return 0;
  if (m->bidx) cudaFree(m->bidx);
  m->bidx = nullptr;
  m->bidx_cap = 0;
  if (int e = dmalloc(c, &m->bidx, (size_t)n)) return e;
  m->bidx_cap = n;
  return 0;
}

// Mean loss over the listed samples (forward only, batches of up to tB).
int eval_loss(dgx_ctx *c, const std::vector<int> &idx, double *loss) {
  Learned *m = c->learned;
  *loss = 0.0;
  if (idx.empty()) return 0;
  const int B = std::max(1, std::min<int>(m->tB, (int)idx.size()));
  const long long G = m->g.G;
  const int nb = blocks_for(G, kRedBlocks);
  if (int e = ensure_bidx(c, (long long)idx.size())) return e;
  if (int e = h2d(c, m->bidx, idx.data(), idx.size() * sizeof(int), "upload batch")) return e;
  double sum = 0.0;
  for (size_t s = 0; s < idx.size(); s += B) {
    const int nbatch = (int)std::min<size_t>(B, idx.size() - s);
    if (int e = batch_forward_loss(c, m->bidx + s, nbatch)) return e;
    if (int e = check_cuda(c, cudaMemcpyAsync(m->host_lpart, m->lpart, (size_t)nbatch * nb * sizeof(double),
                                              cudaMemcpyDeviceToHost, c->stream), "loss copy")) return e;
    if (int e = check_cuda(c, cudaStreamSynchronize(c->stream), "loss sync")) return e;
    for (int k = 0; k < nbatch * nb; ++k) sum += m->host_lpart[k];
  }
  *loss = sum / (double)idx.size();
  return 0;
}

int grow_dataset(dgx_ctx *c, long long need) {
  Learned *m = c->learned;
  if (need <= m->ds_cap) return 0;
  const long long cap = std::max<long long>(need, std::max<long long>(64, 2 * m->ds_cap));
  const long long ss = (long long)(kCin + 1) * m->g.G;
  float *nds = nullptr, *ntn = nullptr;
  if (int e = dmalloc(c, &nds, (size_t)(cap * ss))) return e;
  if (int e = dmalloc(c, &ntn, (size_t)cap)) {
    cudaFree(nds);
    return e;
  }
  if (m->ds_n) {
    cudaMemcpyAsync(nds, m->ds, (size_t)(m->ds_n * ss) * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(ntn, m->tn2, (size_t)m->ds_n * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
  }
  if (int e = check_cuda(c, cudaStreamSynchronize(c->stream), "grow dataset")) return e;
  if (m->ds) cudaFree(m->ds);
  if (m->tn2) cudaFree(m->tn2);
  m->ds = nds;
  m->tn2 = ntn;
  m->ds_cap = cap;
  return 0;
}

// Append the pair (v, e) (device FP64, DoF order) with the live coefficient channels.
int add_pair(dgx_ctx *c, const double *v, const double *e, bool test) {
  Learned *m = c->learned;
  if (int err = grow_dataset(c, m->ds_n + 1)) return err;
  const long long G = m->g.G, ss = (long long)(kCin + 1) * G;
  float *dst = m->ds + m->ds_n * ss;
  cudaMemcpyAsync(dst + G, m->live + G, (size_t)(kCin - 1) * G * sizeof(float), cudaMemcpyDeviceToDevice, c->stream);
  if (int err = features<double>(c, v, e, dst, m->tn2 + m->ds_n)) return err;
  m->ds_n += 1;
  m->is_test.push_back(test ? 1 : 0);
  return 0;
}

int check_learned(dgx_ctx *c) {
  if (!c) return DGX_ERR_ARG;
  if (int e = need_net(c)) return e;
  if (!c->has_mesh) return set_error(c, DGX_ERR_STATE, "no mesh (call dgx_mesh_build)");
  if (c->nc) return set_error(c, DGX_ERR_STATE, "the learned preconditioner is not available on non-conforming meshes");
  return ensure_grid(c);
}

}  // namespace

// ---------------------------------------------------------------- internal API
void learned_free(dgx_ctx *c) {
  if (!c->learned) return;
  free_grid(c->learned);
  free_dataset(c->learned);
  free_net(c->learned);
  delete c->learned;
  c->learned = nullptr;
}

void learned_mesh_changed(dgx_ctx *c) {
  if (c->learned) free_grid(c->learned);
}

bool learned_ready(const dgx_ctx *c) { return c->learned && c->learned->master; }

namespace {

// The launches of one apply on c->stream: features, the network, the output.
template <typename T>
int apply_direct(dgx_ctx *c, const T *v, T *z) {
  Learned *m = c->learned;
  if (int e = features<T>(c, v, nullptr, m->live, nullptr)) return e;
  float *out = nullptr;
  if (int e = net_forward1(c, m->live, &out)) return e;
  count_launch();
  k_learn_out<T><<<blocks_for(m->g.G), 256, 0, c->stream>>>(m->g, v, c->dinv64[DGX_PC_HELMHOLTZ], out, m->scal + 3, z);
  return check_cuda(c, cudaGetLastError(), "k_learn_out");
}

// Capture the launches of apply_direct(v, z) as a CUDA graph on the private stream.
template <typename T>
int capture_apply(dgx_ctx *c, const T *v, T *z, Learned::GraphRec *rec) {
  Learned *m = c->learned;
  if (!m->gstream) {
    if (int e = check_cuda(c, cudaStreamCreateWithFlags(&m->gstream, cudaStreamNonBlocking), "stream")) return e;
    if (int e = check_cuda(c, cudaEventCreateWithFlags(&m->gev0, cudaEventDisableTiming), "event")) return e;
    if (int e = check_cuda(c, cudaEventCreateWithFlags(&m->gev1, cudaEventDisableTiming), "event")) return e;
  }
  const long long n0 = launch_count();
  cudaStream_t saved = c->stream;
  c->stream = m->gstream;
  cudaGraph_t graph = nullptr;
  int e = check_cuda(c, cudaStreamBeginCapture(m->gstream, cudaStreamCaptureModeThreadLocal), "begin capture");
  if (!e) {
    e = apply_direct<T>(c, v, z);
    const cudaError_t ce = cudaStreamEndCapture(m->gstream, &graph);
    if (!e) e = check_cuda(c, ce, "end capture");
  }
  c->stream = saved;
  const long long n = launch_count() - n0;
  count_launch((int)-n);  // nothing ran: the replays count their launches
  if (!e) e = check_cuda(c, cudaGraphInstantiate(&rec->exec, graph, 0), "graph instantiate");
  if (graph) cudaGraphDestroy(graph);
  rec->launches = n;
  return e;
}

}  // namespace

// z = M(v).  Outside a caller's stream capture, the launches of each (v, z)
// pair are captured once and replayed as a graph (ordered after and before
// the context's stream by events): the network's dozen small kernels then
// cost one launch.
template <typename T>
int learned_apply(dgx_ctx *c, const T *v, T *z) {
  if (int e = check_learned(c)) return e;
  Learned *m = c->learned;
  if (int e = ensure_coef_features(c)) return e;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (int e = check_cuda(c, cudaStreamIsCapturing(c->stream, &cs), "capture status")) return e;
  if (cs != cudaStreamCaptureStatusNone) return apply_direct<T>(c, v, z);
  const auto key = std::make_tuple((const void *)v, (void *)z, (int)sizeof(T));
  auto it = m->graphs.find(key);
  if (it == m->graphs.end()) {
    if (int e = apply_direct<T>(c, v, z)) return e;  // also sets the kernels' attributes
    if (m->graphs.size() >= 256) free_graphs(m);
    Learned::GraphRec rec{};
    if (int e = capture_apply<T>(c, v, z, &rec)) return e;
    m->graphs[key] = rec;
    return 0;
  }
  int e;
  if ((e = check_cuda(c, cudaEventRecord(m->gev0, c->stream), "event")) ||
      (e = check_cuda(c, cudaStreamWaitEvent(m->gstream, m->gev0, 0), "wait")) ||
      (e = check_cuda(c, cudaGraphLaunch(it->second.exec, m->gstream), "graph launch")) ||
      (e = check_cuda(c, cudaEventRecord(m->gev1, m->gstream), "event")) ||
      (e = check_cuda(c, cudaStreamWaitEvent(c->stream, m->gev1, 0), "wait")))
    return e;
  count_launch((int)it->second.launches);
  return 0;
}
template int learned_apply<double>(dgx_ctx *, const double *, double *);
template int learned_apply<float>(dgx_ctx *, const float *, float *);

}  // namespace dgx

using namespace dgx;

extern "C" {

int dgx_learned_create(dgx_ctx *c, int layers, int channels, unsigned long long seed) {
  if (!c) return DGX_ERR_ARG;
  if (layers < 2 || layers > 16 || channels < 8 || channels > 64 || channels % 8)
    return set_error(c, DGX_ERR_ARG, "need 2 <= layers <= 16 and channels in 8..64, a multiple of 8");
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  learned_free(c);
  Learned *m = new Learned();
  c->learned = m;
  m->L = layers;
  m->C = channels;
  for (int l = 0; l < layers; ++l) {
    m->ci.push_back(l == 0 ? kCin : channels);
    m->co.push_back(l == layers - 1 ? 1 : channels);
    m->poff.push_back(m->P);
    m->woff.push_back(m->nW);
    const long long nw = (long long)m->ci[l] * m->co[l] * 27;
    m->P += nw + m->co[l];
    m->nW += (nw + 3) / 4 * 4;  // layers start on 8-byte boundaries (rows of 4 bf16)
  }
  std::vector<float> p((size_t)m->P, 0.f);
  SplitMix rng{seed};
  for (int l = 0; l + 1 < layers; ++l) {
    const double sd = std::sqrt(2.0 / (27.0 * m->ci[l]));
    const long long nw = (long long)m->ci[l] * m->co[l] * 27;
    for (long long k = 0; k < nw; ++k) p[(size_t)(m->poff[l] + k)] = (float)(sd * rng.normal());
  }
  int e;
  if ((e = dmalloc(c, &m->master, m->P)) || (e = dmalloc(c, &m->am, m->P)) || (e = dmalloc(c, &m->av, m->P)) ||
      (e = dmalloc(c, &m->grad, m->P)) || (e = dmalloc(c, &m->wbf, m->nW)) ||
      (e = dmalloc(c, &m->wtbf, m->nW)) || (e = dmalloc(c, &m->tc_err, 1)) ||
      (e = check_cuda(c, cudaMemset(m->tc_err, 0, sizeof(int)), "memset"))) {
    learned_free(c);
    return e;
  }
  return dgx_learned_set_params(c, p.data());
}

long long dgx_learned_num_params(const dgx_ctx *c) { return (c && c->learned) ? c->learned->P : -1; }

int dgx_learned_set_params(dgx_ctx *c, const float *host) {
  if (!c) return DGX_ERR_ARG;
  if (int e = need_net(c)) return e;
  if (!host) return set_error(c, DGX_ERR_ARG, "null parameter array");
  Learned *m = c->learned;
  cudaStreamSynchronize(c->stream);
  if (int e = h2d(c, m->master, host, (size_t)m->P * sizeof(float), "upload parameters")) return e;
  cudaMemsetAsync(m->am, 0, (size_t)m->P * sizeof(float), c->stream);
  cudaMemsetAsync(m->av, 0, (size_t)m->P * sizeof(float), c->stream);
  m->adam_t = 0;
  for (int l = 0; l < m->L; ++l) {
    count_launch();
    k_round_weights<<<blocks_for((long long)m->ci[l] * m->co[l] * 27), 256, 0, c->stream>>>(
        m->ci[l], m->co[l], m->master + m->poff[l], m->wbf + m->woff[l], m->wtbf + m->woff[l]);
  }
  return check_cuda(c, cudaStreamSynchronize(c->stream), "set parameters");
}

int dgx_learned_get_params(dgx_ctx *c, float *host) {
  if (!c) return DGX_ERR_ARG;
  if (int e = need_net(c)) return e;
  if (!host) return set_error(c, DGX_ERR_ARG, "null parameter array");
  cudaStreamSynchronize(c->stream);
  return check_cuda(c, cudaMemcpy(host, c->learned->master, (size_t)c->learned->P * sizeof(float),
                                  cudaMemcpyDeviceToHost), "download parameters");
}

int dgx_learned_apply(dgx_ctx *c, int prec, const void *v, void *z) {
  if (!c) return DGX_ERR_ARG;
  if (!c->has_coef) return set_error(c, DGX_ERR_STATE, "no coefficients (call dgx_set_coefficients)");
  if (!v || !z || v == z) return set_error(c, DGX_ERR_ARG, "v, z must be distinct non-null arrays");
  if (prec == DGX_F64) return learned_apply<double>(c, (const double *)v, (double *)z);
  if (prec == DGX_F32) return learned_apply<float>(c, (const float *)v, (float *)z);
  return set_error(c, DGX_ERR_ARG, "precision %d", prec);
}

int dgx_learned_add_system(dgx_ctx *c, const double *rho, const double *pk, double a_dt, double gamma,
                           const double *b, const double *x, int pairs, int stride, int test) {
  if (int e = check_learned(c)) return e;
  if (!b || !x) return set_error(c, DGX_ERR_ARG, "null b or x");
  if (pairs < 1 || stride < 1 || stride > 64) return set_error(c, DGX_ERR_ARG, "need pairs >= 1, 1 <= stride <= 64");
  if (int e = dgx_set_coefficients(c, rho, pk, a_dt, gamma)) return e;
  if (int e = ensure_coef_features(c)) return e;
  if (int e = add_pair(c, b, x, test != 0)) return e;
  if (pairs == 1) return check_cuda(c, cudaStreamSynchronize(c->stream), "add system");
  const long long N = c->N;
  double *buf = nullptr;
  if (int e = dmalloc(c, &buf, (size_t)3 * N)) return e;
  double *xk = buf, *r = buf + N, *err = buf + 2 * N;
  cudaMemsetAsync(xk, 0, N * sizeof(double), c->stream);
  dgx_solve_opts o;
  dgx_default_solve_opts(&o);
  o.method = DGX_SOLVER_FGMRES;
  o.pc = DGX_PC_HELMHOLTZ;
  o.restart = stride;
  o.maxit = stride;
  o.tol = 1e-300;
  o.use_x0 = 1;
  int rc = 0;
  for (int k = 1; k < pairs && rc == 0; ++k) {
    dgx_solve_info si;
    const int s = dgx_solve_pressure(c, b, xk, &o, &si);
    if (s < 0) {
      rc = s;
      break;
    }
    if (!(si.relres >= 1e-6)) break;  // the pair would be dominated by the error of x
    rc = dgx_apply_operator(c, DGX_F64, xk, r);
    if (rc) break;
    vec_axpby<double>(N, 1.0, b, -1.0, r, c->stream);  // r = b - S x_k
    cudaMemcpyAsync(err, x, N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    vec_axpby<double>(N, -1.0, xk, 1.0, err, c->stream);  // e = x - x_k
    rc = add_pair(c, r, err, test != 0);
  }
  const int e2 = check_cuda(c, cudaStreamSynchronize(c->stream), "add system");
  cudaFree(buf);
  return rc ? rc : e2;
}

int dgx_learned_num_samples(const dgx_ctx *c, int *train, int *test) {
  if (!c) return DGX_ERR_ARG;
  int tr = 0, te = 0;
  if (c->learned)
    for (char t : c->learned->is_test) (t ? te : tr) += 1;
  if (train) *train = tr;
  if (test) *test = te;
  return DGX_OK;
}

int dgx_learned_sample(dgx_ctx *c, int i, float *host) {
  if (int e = check_learned(c)) return e;
  Learned *m = c->learned;
  if (i < 0 || i >= m->ds_n || !host) return set_error(c, DGX_ERR_ARG, "sample %d of %lld", i, m->ds_n);
  const long long ss = (long long)(kCin + 1) * m->g.G;
  cudaStreamSynchronize(c->stream);
  return check_cuda(c, cudaMemcpy(host, m->ds + (long long)i * ss, (size_t)ss * sizeof(float), cudaMemcpyDeviceToHost),
                    "download sample");
}

int dgx_learned_clear_samples(dgx_ctx *c) {
  if (!c) return DGX_ERR_ARG;
  if (c->learned) {
    c->learned->ds_n = 0;
    c->learned->is_test.clear();
  }
  return DGX_OK;
}

int dgx_learned_loss(dgx_ctx *c, int first, int count, double *loss, float *grad_host) {
  if (int e = check_learned(c)) return e;
  Learned *m = c->learned;
  if (first < 0 || count < 1 || count > kMaxBatch || first + count > m->ds_n)
    return set_error(c, DGX_ERR_ARG, "samples %d..%d of %lld (at most %d)", first, first + count - 1, m->ds_n, kMaxBatch);
  if (int e = ensure_train_buffers(c, count)) return e;
  if (int e = ensure_bidx(c, count)) return e;
  std::vector<int> idx(count);
  std::iota(idx.begin(), idx.end(), first);
  if (int e = h2d(c, m->bidx, idx.data(), count * sizeof(int), "upload batch")) return e;
  if (int e = batch_forward_loss(c, m->bidx, count)) return e;
  if (int e = batch_backward(c, m->bidx, count, false, 0.f, 0.f, 0.f, 0.f)) return e;
  const int nb = blocks_for(m->g.G, kRedBlocks);
  if (int e = check_cuda(c, cudaMemcpyAsync(m->host_lpart, m->lpart, (size_t)count * nb * sizeof(double),
                                            cudaMemcpyDeviceToHost, c->stream), "loss copy")) return e;
  if (int e = check_cuda(c, cudaStreamSynchronize(c->stream), "loss")) return e;
  if (int e = tc_status(c)) return e;
  double s = 0.0;
  for (int k = 0; k < count * nb; ++k) s += m->host_lpart[k];
  if (loss) *loss = s / count;
  if (grad_host)
    return check_cuda(c, cudaMemcpy(grad_host, m->grad, (size_t)m->P * sizeof(float), cudaMemcpyDeviceToHost),
                      "download gradient");
  return DGX_OK;
}

void dgx_default_train_opts(dgx_train_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->epochs = 40;
  o->batch = 16;
  o->lr = 2e-3;
  o->lr_final = 1e-4;
  o->beta1 = 0.9;
  o->beta2 = 0.999;
  o->eps = 1e-8;
  o->seed = 20250501ull;
  o->shuffle = 1;
}

int dgx_learned_train(dgx_ctx *c, const dgx_train_opts *opts, dgx_train_info *info) {
  if (int e = check_learned(c)) return e;
  Learned *m = c->learned;
  dgx_train_opts o;
  if (opts) o = *opts;
  else dgx_default_train_opts(&o);
  if (o.epochs < 0 || o.batch < 1 || o.batch > kMaxBatch || !(o.lr > 0) || !(o.lr_final > 0))
    return set_error(c, DGX_ERR_ARG, "need epochs >= 0, 1 <= batch <= %d, lr > 0", kMaxBatch);
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<int> tr, te;
  for (long long i = 0; i < m->ds_n; ++i) (m->is_test[(size_t)i] ? te : tr).push_back((int)i);
  if (tr.empty()) return set_error(c, DGX_ERR_STATE, "no training samples (dgx_learned_add_system)");
  dgx_train_info inf;
  std::memset(&inf, 0, sizeof(inf));
  inf.train_samples = (int)tr.size();
  inf.test_samples = (int)te.size();
  const int B = std::min<int>(o.batch, (int)tr.size());
  if (int e = ensure_train_buffers(c, B)) return e;
  if (int e = eval_loss(c, tr, &inf.loss_train0)) return e;
  if (int e = eval_loss(c, te, &inf.loss_test0)) return e;
  const int steps_per_epoch = (int)(tr.size() / B);
  const long long total = (long long)steps_per_epoch * o.epochs;
  SplitMix rng{o.seed};
  std::vector<int> order = tr;
  if (int e = ensure_bidx(c, (long long)order.size())) return e;
  long long step = 0;
  for (int ep = 0; ep < o.epochs; ++ep) {
    if (o.shuffle)
      for (size_t i = order.size(); i > 1; --i) std::swap(order[i - 1], order[(size_t)(rng.next() % i)]);
    if (int e = check_cuda(c, cudaStreamSynchronize(c->stream), "epoch")) return e;
    if (int e = h2d(c, m->bidx, order.data(), order.size() * sizeof(int), "upload order")) return e;
    for (int s = 0; s < steps_per_epoch; ++s, ++step) {
      const double f = total > 1 ? (double)step / (double)(total - 1) : 0.0;
      const double lr = o.lr_final + 0.5 * (o.lr - o.lr_final) * (1.0 + std::cos(3.141592653589793 * f));
      const int *bi = m->bidx + (size_t)s * B;
      if (int e = batch_forward_loss(c, bi, B)) return e;
      if (int e = batch_backward(c, bi, B, true, (float)lr, (float)o.beta1, (float)o.beta2, (float)o.eps)) return e;
    }
  }
  inf.steps = (int)step;
  if (int e = check_cuda(c, cudaStreamSynchronize(c->stream), "train")) return e;
  if (int e = tc_status(c)) return e;
  if (int e = eval_loss(c, tr, &inf.loss_train)) return e;
  if (int e = eval_loss(c, te, &inf.loss_test)) return e;
  inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  return DGX_OK;
}

}  // extern "C"
