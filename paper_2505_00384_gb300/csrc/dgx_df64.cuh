// Double-word ("double-float") arithmetic: a value is the unevaluated sum
// hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant
// bits.  On GB300 the FP32 pipes are 64 times the FP64 pipe, so FP64-accuracy
// kernels can run on FP32 arithmetic.  Building blocks (each FP32 operation
// rounded to nearest, no contraction: the __f*_rn intrinsics):
//   TwoSum (Knuth) and Fast2Sum (Dekker): the exact error of a sum;
//   TwoProd with FMA: the exact error of a product;
//   sum of two double-words: "SloppyDWPlusDW", product: "DWTimesDW2",
//   quotient: "DWDivDW2" of Joldes, Muller and Popescu, "Tight and rigorous
//   error bounds for basic building blocks of double-word arithmetic", ACM
//   TOMS 44 (2017).  The product and quotient have relative errors of a few
//   u^2 (u = 2^-24); the sloppy sum has an absolute error of a few
//   u^2 (|x| + |y|) (no relative bound under cancellation), which is what a
//   sum-factorised contraction needs: its error is measured against the size
//   of the terms.
// The exponent range is FP32's: values (and the low parts) must stay within
// about 1e-30 .. 1e38 in magnitude for the full precision.
#pragma once

#include <cuda_runtime.h>

namespace dgx {

struct df64;
#ifdef __CUDACC__
__device__ __forceinline__ df64 dw_split_device(double d);
#endif

struct df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  // hi = RN(d) to 24 bits, lo = RN(d - hi)
  __host__ __device__ df64(double d);
  __host__ __device__ df64(int i) : df64((double)i) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

#ifdef __CUDACC__
// The split of a double into a double-word without the FP64 pipe (its
// conversions run at 1/64 of the FP32 rate on this GPU): the 53-bit
// significand is rounded to 24 bits to nearest even with integer operations,
// and the remainder (at most 29 bits, signed) is converted to float and scaled
// by a power of two.  The result equals the FP64-pipe split bit for bit:
// d - hi is exact, and RN of the scaled remainder is the scaled RN.  Doubles
// whose hi or lo would leave the normal float range (|d| outside [2^-74,
// 2^127)), zeros, subnormals, infinities and NaNs take the FP64 path.
__device__ __forceinline__ df64 dw_split_device(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e < 949 || e > 1149) {
    const float h = __double2float_rn(d);
    return df64(h, __double2float_rn(d - (double)h));
  }
  const unsigned sgn = (unsigned)(b >> 63) << 31;
  const long long m = (long long)((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);  // 53-bit significand
  long long mh = m >> 29;
  const long long rem = m & 0x1FFFFFFFll, half = 1ll << 28;
  if (rem > half || (rem == half && (mh & 1))) ++mh;  // round to nearest even
  const int r = (int)(m - (mh << 29));                // d - hi in units of 2^(e - 1075), |r| <= 2^28
  int eh = e - 1023 + 127;
  if (mh == (1ll << 24)) {  // rounded up into the next binade
    mh >>= 1;
    ++eh;
  }
  const float hi = __uint_as_float(sgn | ((unsigned)eh << 23) | ((unsigned)mh & 0x7FFFFFu));
  const float scale = __uint_as_float((unsigned)(e - 1075 + 127) << 23);  // 2^(e - 1075), normal for e >= 949
  return df64(hi, __fmul_rn(__int2float_rn(sgn ? -r : r), scale));
}
#endif

__host__ __device__ inline df64::df64(double d) {
#ifdef __CUDA_ARCH__
  *this = dw_split_device(d);
#else
  hi = (float)d;
  lo = (float)(d - (double)(float)d);
#endif
}

// storage type of a compute type: double-word kernels read and write FP64 arrays
template <typename T>
struct Store {
  using type = T;
};
template <>
struct Store<df64> {
  using type = double;
};
template <typename T>
using store_t = typename Store<T>::type;

#ifdef __CUDACC__
__device__ __forceinline__ df64 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float a1 = __fsub_rn(s, b);
  const float b1 = __fsub_rn(s, a1);
  const float da = __fsub_rn(a, a1);
  const float db = __fsub_rn(b, b1);
  return df64(s, __fadd_rn(da, db));
}
__device__ __forceinline__ df64 fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  return df64(s, __fsub_rn(b, z));
}
__device__ __forceinline__ df64 operator+(df64 x, df64 y) {
  const df64 s = two_sum(x.hi, y.hi);
  const float v = __fadd_rn(x.lo, y.lo);
  const float w = __fadd_rn(s.lo, v);
  return fast_two_sum(s.hi, w);
}
__device__ __forceinline__ df64 operator-(df64 x) { return df64(-x.hi, -x.lo); }
__device__ __forceinline__ df64 operator-(df64 x, df64 y) { return x + (-y); }
__device__ __forceinline__ df64 operator*(df64 x, df64 y) {
  const float ch = __fmul_rn(x.hi, y.hi);
  const float cl1 = __fmaf_rn(x.hi, y.hi, -ch);
  const float tl = __fmul_rn(x.hi, y.lo);
  const float cl2 = __fmaf_rn(x.lo, y.hi, tl);
  const float cl3 = __fadd_rn(cl1, cl2);
  return fast_two_sum(ch, cl3);
}
__device__ __forceinline__ df64 operator/(df64 x, df64 y) {
  const float th = __fdiv_rn(x.hi, y.hi);
  // r = y * th (double-word times float), then the remainder x - r
  const float rh0 = __fmul_rn(y.hi, th);
  const float rl0 = __fmaf_rn(y.hi, th, -rh0);
  const float rl1 = __fmaf_rn(y.lo, th, rl0);
  const df64 r = fast_two_sum(rh0, rl1);
  const df64 pi = two_sum(x.hi, -r.hi);
  const float dh = __fsub_rn(pi.lo, r.lo);
  const float dl = __fadd_rn(dh, x.lo);
  const float d = __fadd_rn(pi.hi, dl);
  return fast_two_sum(th, __fdiv_rn(d, y.hi));
}
// |x| and max(a, b) for code written once for double and double-word values
// (double-words are normalised, |lo| <= ulp(hi)/2: compare hi, then lo)
__device__ __forceinline__ double tabs(double x) { return fabs(x); }
__device__ __forceinline__ double tmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ df64 tabs(df64 x) { return (x.hi < 0.f || (x.hi == 0.f && x.lo < 0.f)) ? -x : x; }
__device__ __forceinline__ df64 tmax(df64 a, df64 b) { return (a.hi > b.hi || (a.hi == b.hi && a.lo >= b.lo)) ? a : b; }
__device__ __forceinline__ df64 &operator+=(df64 &x, df64 y) { return x = x + y; }
__device__ __forceinline__ df64 &operator-=(df64 &x, df64 y) { return x = x - y; }
__device__ __forceinline__ df64 &operator*=(df64 &x, df64 y) { return x = x * y; }
#endif

}  // namespace dgx
