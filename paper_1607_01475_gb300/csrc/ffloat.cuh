// Double-word ("float-float") arithmetic: a value is the unevaluated sum
// hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant
// bits.  On GB300 the FP32 pipes issue 64 times as many operations per
// clock as the FP64 pipe, so a transform done in float-float costs a small
// fraction of the same transform in FP64 while keeping a relative accuracy
// of a few 2^-48.
//
// Algorithms (all with fused multiply-add):
//   two_sum       Knuth's error-free sum (6 operations, any operands);
//   fast_two_sum  Dekker's error-free sum for |a| >= |b| (3 operations);
//   the error-free product a b = p + fma(a, b, -p) inside the products;
//   ff_add        "AccurateDWPlusDW" and ff_mul "DWTimesDW" (with FMA) of
//                 M. Joldes, J.-M. Muller, V. Popescu, "Tight and rigorous
//                 error bounds for basic building blocks of double-word
//                 arithmetic", ACM TOMS 44(2), 2017: relative errors of a
//                 few u^2 (u = 2^-24);
//   ff_mul_f      a double-word times an FP32 number exactly representable
//                 in it (as DWTimesFP with FMA from the same paper).
// The compiler must not reassociate these: the build uses no fast-math.
#pragma once

#include <cuda_runtime.h>

namespace psd {

struct __align__(8) ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  // nearest double-word to a double (exact up to the 48-bit rounding of lo)
  __host__ __device__ constexpr explicit ff(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ ff ff_add(ff x, ff y) {
  float sh, sl, th, tl, vh, vl;
  two_sum(x.hi, y.hi, sh, sl);
  two_sum(x.lo, y.lo, th, tl);
  const float c = __fadd_rn(sl, th);
  fast_two_sum(sh, c, vh, vl);
  const float w = __fadd_rn(tl, vl);
  ff z;
  fast_two_sum(vh, w, z.hi, z.lo);
  return z;
}

__device__ __forceinline__ ff ff_neg(ff x) { return ff(-x.hi, -x.lo); }
__device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }

__device__ __forceinline__ ff ff_mul(ff x, ff y) {
  const float ch = __fmul_rn(x.hi, y.hi);
  const float cl1 = __fmaf_rn(x.hi, y.hi, -ch);
  const float tl0 = __fmul_rn(x.lo, y.lo);
  const float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
  const float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
  const float cl3 = __fadd_rn(cl1, cl2);
  ff z;
  fast_two_sum(ch, cl3, z.hi, z.lo);
  return z;
}

__device__ __forceinline__ ff ff_mul_f(ff x, float y) {
  const float ch = __fmul_rn(x.hi, y);
  const float cl1 = __fmaf_rn(x.hi, y, -ch);
  const float cl3 = __fmaf_rn(x.lo, y, cl1);
  ff z;
  fast_two_sum(ch, cl3, z.hi, z.lo);
  return z;
}

// Exact scaling by a power of two.
__device__ __forceinline__ ff ff_scale2(ff x, float p2) { return ff(x.hi * p2, x.lo * p2); }

__host__ __device__ __forceinline__ double ff_to_double(ff v) { return (double)v.hi + (double)v.lo; }

// Arithmetic operators so that the line-FFT templates run on ff.
__device__ __forceinline__ ff operator+(ff a, ff b) { return ff_add(a, b); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return ff_sub(a, b); }
__device__ __forceinline__ ff operator-(ff a) { return ff_neg(a); }
__device__ __forceinline__ ff operator*(ff a, ff b) { return ff_mul(a, b); }

}  // namespace psd
