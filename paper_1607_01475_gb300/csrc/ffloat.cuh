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
//                 in it (as DWTimesFP with FMA from the same paper);
//   ff_add_fast   "SloppyDWPlusDW" of the same paper, for FFT butterflies.
// The compiler must not reassociate these: the build uses no fast-math.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

namespace psd {

struct __align__(8) ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  // nearest double-word to a double (exact up to the 48-bit rounding of lo)
  __host__ __device__ constexpr explicit ff(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
};

// Round-to-nearest FP32 primitives: the intrinsics on the device (never
// contracted into FMAs), plain IEEE operations on the host (built without
// contraction).
__host__ __device__ __forceinline__ float f_add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
__host__ __device__ __forceinline__ float f_sub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
__host__ __device__ __forceinline__ float f_mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
__host__ __device__ __forceinline__ float f_fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return fmaf(a, b, c);
#endif
}

__host__ __device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = f_add(a, b);
  const float bb = f_sub(s, a);
  e = f_add(f_sub(a, f_sub(s, bb)), f_sub(b, bb));
}

__host__ __device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = f_add(a, b);
  e = f_sub(b, f_sub(s, a));
}

__host__ __device__ __forceinline__ ff ff_add(ff x, ff y) {
  float sh, sl, th, tl, vh, vl;
  two_sum(x.hi, y.hi, sh, sl);
  two_sum(x.lo, y.lo, th, tl);
  const float c = f_add(sl, th);
  fast_two_sum(sh, c, vh, vl);
  const float w = f_add(tl, vl);
  ff z;
  fast_two_sum(vh, w, z.hi, z.lo);
  return z;
}

__host__ __device__ __forceinline__ ff ff_neg(ff x) { return ff(-x.hi, -x.lo); }
__host__ __device__ __forceinline__ ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }

// The cheaper double-word sum ("SloppyDWPlusDW" of the same paper: 11
// operations).  Its error is below a few u^2 (|x| + |y|) in absolute terms
// but not relative to a sum that cancels; that is the bound the error
// analysis of an FFT butterfly needs (its error is measured against the
// norm of the data), so the line FFT uses it.  Where the cancellation is
// the point (a residual as the difference of two nearly equal transforms)
// ff_add is used.
__host__ __device__ __forceinline__ ff ff_add_fast(ff x, ff y) {
  float sh, sl;
  two_sum(x.hi, y.hi, sh, sl);
  const float v = f_add(sl, f_add(x.lo, y.lo));
  ff z;
  fast_two_sum(sh, v, z.hi, z.lo);
  return z;
}

__host__ __device__ __forceinline__ ff ff_mul(ff x, ff y) {
  const float ch = f_mul(x.hi, y.hi);
  const float cl1 = f_fma(x.hi, y.hi, -ch);
  const float tl0 = f_mul(x.lo, y.lo);
  const float tl1 = f_fma(x.hi, y.lo, tl0);
  const float cl2 = f_fma(x.lo, y.hi, tl1);
  const float cl3 = f_add(cl1, cl2);
  ff z;
  fast_two_sum(ch, cl3, z.hi, z.lo);
  return z;
}

__host__ __device__ __forceinline__ ff ff_mul_f(ff x, float y) {
  const float ch = f_mul(x.hi, y);
  const float cl1 = f_fma(x.hi, y, -ch);
  const float cl3 = f_fma(x.lo, y, cl1);
  ff z;
  fast_two_sum(ch, cl3, z.hi, z.lo);
  return z;
}

// 1/a for a normal positive a: the FP32 reciprocal of a.hi refined by one
// Newton-Raphson step in double-word arithmetic, r = r0 + r0 (1 - a r0),
// which squares the ~2^-23 error of r0 (result within a few 2^-47).
__host__ __device__ __forceinline__ ff ff_recip(ff a) {
#ifdef __CUDA_ARCH__
  float r0;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(a.hi));
#else
  float r0 = 1.0f / a.hi;
#endif
  r0 = f_fma(r0, f_fma(-a.hi, r0, 1.0f), r0);
  const ff e = ff_sub(ff(1.0f, 0.0f), ff_mul_f(a, r0));
  return ff_add(ff(r0, 0.0f), ff_mul_f(e, r0));
}

// Exact scaling by a power of two.
__host__ __device__ __forceinline__ ff ff_scale2(ff x, float p2) { return ff(x.hi * p2, x.lo * p2); }

__host__ __device__ __forceinline__ double ff_to_double(ff v) { return (double)v.hi + (double)v.lo; }

// ---- conversions between FP64 and float-float by bit manipulation (no FP64
// arithmetic, whose pipe is 1/64 of the FP32 rate on GB300)
__host__ __device__ __forceinline__ unsigned long long ff_dbits(double v) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(v);
#else
  unsigned long long b;
  std::memcpy(&b, &v, 8);
  return b;
#endif
}
__host__ __device__ __forceinline__ double ff_bitsd(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double v;
  std::memcpy(&v, &b, 8);
  return v;
#endif
}
__host__ __device__ __forceinline__ unsigned ff_fbits(float v) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(v);
#else
  unsigned b;
  std::memcpy(&b, &v, 4);
  return b;
#endif
}
__host__ __device__ __forceinline__ float ff_bitsf(unsigned b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float v;
  std::memcpy(&v, &b, 4);
  return v;
#endif
}

// double -> float-float: hi = v truncated to 24 significant bits, lo = the
// remaining 29 bits rounded to a float, then renormalised (hi + lo = v to a
// relative 2^-47).  Magnitudes below the float normal range give 0 (with
// the sign), above it +-inf; NaN stays NaN.
__host__ __device__ __forceinline__ ff ff_from_double_bits(double v) {
  const unsigned long long b = ff_dbits(v);
  const unsigned sgn = (unsigned)(b >> 63) << 31;
  const int E = (int)((b >> 52) & 0x7FF);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFULL;
  if (E == 0x7FF) return ff(ff_bitsf(sgn | 0x7F800000u | (m ? 0x400000u : 0u)), 0.0f);
  const int e = E - 1023;
  if (e < -126) return ff(ff_bitsf(sgn), 0.0f);
  if (e > 127) return ff(ff_bitsf(sgn | 0x7F800000u), 0.0f);
  const float hi = ff_bitsf(sgn | ((unsigned)(e + 127) << 23) | (unsigned)(m >> 29));
  const unsigned r = (unsigned)(m & 0x1FFFFFFFu);  // the remainder is r 2^(e - 52)
  if (r == 0) return ff(hi, 0.0f);
#ifdef __CUDA_ARCH__
  const float rf = __uint2float_rn(r);
#else
  const float rf = (float)r;
#endif
  float lo = (rf * ff_bitsf(0x25800000u)) * ff_bitsf((unsigned)(e + 127) << 23);  // r 2^-52 2^e
  if (sgn) lo = -lo;
  ff z;
  fast_two_sum(hi, lo, z.hi, z.lo);
  return z;
}

// float-float -> double, hi + lo assembled as a 53-bit integer significand
// (exact for a normalised pair up to the truncation of bits of lo below
// 2^-53 of hi; lo may be subnormal).  A zero or subnormal hi gives a signed
// zero.
__host__ __device__ __forceinline__ double ff_to_double_bits(ff x) {
  const unsigned hb = ff_fbits(x.hi), lb = ff_fbits(x.lo);
  const unsigned long long sgn = (unsigned long long)(hb >> 31) << 63;
  const int eh = (int)((hb >> 23) & 0xFF);
  if (eh == 0) return ff_bitsd(sgn);
  if (eh == 0xFF) return ff_bitsd(sgn | (0x7FFULL << 52) | ((hb & 0x7FFFFFu) ? (1ULL << 51) : 0ULL));
  long long n = (long long)((hb & 0x7FFFFFu) | 0x800000u) << 29;  // in units of 2^(eh - 127 - 52)
  int el = (int)((lb >> 23) & 0xFF);
  if (el != 0xFF && (lb & 0x7FFFFFFFu) != 0) {
    // in units of 2^(el - 127 - 23); a subnormal lo has no implicit bit and el = 1
    const long long ml = (long long)((lb & 0x7FFFFFu) | (el ? 0x800000u : 0u));
    if (el == 0) el = 1;
    const int sh = el - eh + 29;
    long long t = 0;
    if (sh >= 0)
      t = sh < 32 ? ml << sh : 0;
    else if (sh > -25)
      t = ml >> (-sh);
    n += ((lb ^ hb) >> 31) ? -t : t;
  }
  int e = eh - 127;
  while (n >= (1LL << 53)) {
    n >>= 1;
    ++e;
  }
  while (n > 0 && n < (1LL << 52)) {
    n <<= 1;
    --e;
  }
  if (n <= 0) return ff_bitsd(sgn);
  return ff_bitsd(sgn | ((unsigned long long)(e + 1023) << 52) | ((unsigned long long)n & 0xFFFFFFFFFFFFFULL));
}

// ---- fixed point: v -> round(v 2^S) as a 64-bit integer (ties away from
// zero) by bit manipulation, for |v| 2^S < 2^62 (the caller picks S from a
// bound on |v|; larger values are not representable).  Sums and differences
// of such integers are exact, which the FP64 residual uses for its linear
// part.  Subnormal v is handled; NaN and infinity are not (the caller
// excludes them).
__host__ __device__ __forceinline__ long long fx_from_double(double v, int S) {
  const unsigned long long b = ff_dbits(v);
  const int E = (int)((b >> 52) & 0x7FF);
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFULL) | (E ? (1ULL << 52) : 0ULL);
  const int sh = (E ? E : 1) - 1075 + S;  // |v| = m 2^(E - 1075), subnormal: E = 1 without the implicit bit
  unsigned long long a = 0;
  if (sh >= 0)
    a = m << (sh < 10 ? sh : 9);  // sh <= 9 when |v| 2^S < 2^62
  else if (sh > -54)
    a = (m + (1ULL << (-sh - 1))) >> (-sh);
  return (b >> 63) ? -(long long)a : (long long)a;
}
// 2^-S as a double (|S| <= 1000), by bits
__host__ __device__ __forceinline__ double fx_unit(int S) { return ff_bitsd((unsigned long long)(1023 - S) << 52); }

// x 2^-S as a float-float, by integer operations only (|x| < 2^63,
// 15 <= S <= 120, so that every exponent below is that of a normal float):
// hi holds the leading 24 bits of |x|, lo the next 24 (both truncated), and a
// fast two-sum normalises the pair; the relative error is below 2^-47.
__host__ __device__ __forceinline__ int fx_clz64(unsigned long long a) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)a);
#else
  return __builtin_clzll(a);
#endif
}
// x as a double, rounded to nearest (ties to even), by integer operations
// only (|x| < 2^63): the same value as the hardware conversion.
__host__ __device__ __forceinline__ double fx_to_double(long long x) {
  if (x == 0) return 0.0;
  const unsigned long long sgn = (unsigned long long)x & (1ULL << 63);
  const unsigned long long a = sgn ? 0ULL - (unsigned long long)x : (unsigned long long)x;
  int e = 63 - fx_clz64(a);  // a in [2^e, 2^(e+1))
  unsigned long long m;
  if (e <= 52) {
    m = a << (52 - e);
  } else {
    const int sh = e - 52;  // 1 .. 10
    const unsigned long long rem = a & ((1ULL << sh) - 1ULL), half = 1ULL << (sh - 1);
    m = a >> sh;
    if (rem > half || (rem == half && (m & 1ULL))) ++m;
    if (m >> 53) {  // rounding carried into a new leading bit
      m >>= 1;
      ++e;
    }
  }
  return ff_bitsd(sgn | ((unsigned long long)(e + 1023) << 52) | (m & 0xFFFFFFFFFFFFFULL));
}
__host__ __device__ __forceinline__ ff fx_to_ff(long long x, int S) {
  if (x == 0) return ff(0.0f, 0.0f);
  const bool neg = x < 0;
  const unsigned long long a = neg ? 0ULL - (unsigned long long)x : (unsigned long long)x;
  const int e = 63 - fx_clz64(a);  // a in [2^e, 2^(e+1))
  const int sh = e - 23;
  const unsigned long long top = sh > 0 ? a >> sh : a << (-sh);
  const unsigned long long rem = sh > 0 ? a - (top << sh) : 0ULL;  // < 2^sh
  const float hi = ff_bitsf(((unsigned)(e - S + 127) << 23) | (unsigned)(top & 0x7FFFFFu));
  float lo = 0.0f;
  if (rem != 0) {
    const int e2 = 63 - fx_clz64(rem);
    const int sh2 = e2 - 23;
    const unsigned long long top2 = sh2 > 0 ? rem >> sh2 : rem << (-sh2);
    lo = ff_bitsf(((unsigned)(e2 - S + 127) << 23) | (unsigned)(top2 & 0x7FFFFFu));
  }
  ff z;
  fast_two_sum(hi, lo, z.hi, z.lo);
  if (neg) {
    z.hi = -z.hi;
    z.lo = -z.lo;
  }
  return z;
}

// Arithmetic operators so that the line-FFT templates run on ff (sums with
// the butterfly-grade ff_add_fast).
__host__ __device__ __forceinline__ ff operator+(ff a, ff b) { return ff_add_fast(a, b); }
__host__ __device__ __forceinline__ ff operator-(ff a, ff b) { return ff_add_fast(a, ff_neg(b)); }
__host__ __device__ __forceinline__ ff operator-(ff a) { return ff_neg(a); }
__host__ __device__ __forceinline__ ff operator*(ff a, ff b) { return ff_mul(a, b); }

}  // namespace psd
