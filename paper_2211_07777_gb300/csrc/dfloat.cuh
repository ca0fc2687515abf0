// Double-float ("double-word") arithmetic on the FP32 units: a value is
// hi + lo with |lo| <= ulp(hi)/2, about 48 significant bits (unit roundoff
// u = 2^-48 for the operations below).  On GB300 the FP32 lanes outnumber the
// FP64 units 64:1, so FFT butterflies in double-float arithmetic run several
// times faster than in native FP64 while keeping the FP64 path's accuracy.
//
// Building blocks (published algorithms, written here from their definitions):
//   TwoSum (Knuth): s + e = a + b exactly.
//   FastTwoSum (Dekker): the same when |a| >= |b|.
//   TwoProd with FMA: p + e = a * b exactly.
//   Double-word sum "SloppyDWPlusDW" and product "DWTimesDW3" of Joldes,
//   Muller and Popescu (ACM TOMS 44, 2017): the sum's error is bounded
//   normwise by about 2u(|x| + |y|) -- what a butterfly's error analysis
//   needs -- and the product's relative error by about 4u^2 (relative to u).
// The code relies on IEEE round-to-nearest FP32 operations evaluated as
// written (no -use_fast_math; FMA contraction cannot change these sequences
// since their products are explicit fmaf calls).
#pragma once
#include <cuda_runtime.h>

namespace flups {

struct __align__(8) dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr explicit dfloat(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ constexpr explicit dfloat(int i) : hi((float)i), lo(0.0f) {}
};

__device__ __forceinline__ dfloat two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return dfloat(s, e);
}

__device__ __forceinline__ dfloat fast_two_sum(float a, float b) {
  const float s = a + b;
  const float e = b - (s - a);
  return dfloat(s, e);
}

__device__ __forceinline__ dfloat operator+(dfloat x, dfloat y) {
  const dfloat s = two_sum(x.hi, y.hi);
  const float v = x.lo + y.lo;
  const float w = s.lo + v;
  return fast_two_sum(s.hi, w);
}

__device__ __forceinline__ dfloat operator-(dfloat x) { return dfloat(-x.hi, -x.lo); }
__device__ __forceinline__ dfloat operator-(dfloat x, dfloat y) { return x + dfloat(-y.hi, -y.lo); }

__device__ __forceinline__ dfloat operator*(dfloat x, dfloat y) {
  const float ch = x.hi * y.hi;
  const float cl1 = fmaf(x.hi, y.hi, -ch);
  const float tl0 = x.lo * y.lo;
  const float tl1 = fmaf(x.hi, y.lo, tl0);
  const float cl2 = fmaf(x.lo, y.hi, tl1);
  const float cl3 = cl1 + cl2;
  return fast_two_sum(ch, cl3);
}

__device__ __forceinline__ dfloat& operator+=(dfloat& x, dfloat y) { return x = x + y; }

// Conversions between FP64 and double-float: hi = d rounded to the nearest float, lo = the
// remainder rounded to the nearest float (hi + lo represents d to 2^-48 relative, |lo| <=
// ulp(hi)/2); back, the FP64 value nearest to hi + lo.  (Integer-only versions that avoid GB300's
// FP64 units were measured slower in the double-float x passes: forward 13.9 -> 16.3 ms at
// 1024^3.)
__host__ __device__ __forceinline__ dfloat df_from_double(double d) {
  const float h = (float)d;
  return dfloat(h, (float)(d - (double)h));
}

__host__ __device__ __forceinline__ double df_to_double(dfloat x) { return (double)x.hi + (double)x.lo; }

// complex double-float: 16 bytes, laid out like double2 (hi/lo of re, then of im)
struct __align__(16) cdfloat {
  dfloat x, y;
};

}  // namespace flups
