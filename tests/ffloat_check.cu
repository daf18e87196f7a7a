// Host check of the float-float primitives used by the FP64-storage DHT
// passes: conversions to and from FP64 by bit manipulation, and the
// double-word sum and product, against long-double arithmetic; and the
// FP64 -> fixed-point conversion of the FP64 residual's linear part.  Built and
// run by tests/test_ffloat.py (no GPU needed).  Exit status 0 = pass.
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstdint>

#include "../paper_1607_01475_gb300/csrc/ffloat.cuh"

using psd::ff;

static uint64_t rng_state = 0x1607014750ULL;
static uint64_t next_u64() {  // SplitMix64
  uint64_t z = (rng_state += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static double uniform() { return (double)(next_u64() >> 11) * 0x1p-53; }
// random double: sign, decade in [lo_e, hi_e], full 53-bit mantissa
static double rand_double(int lo_e, int hi_e) {
  const double m = 1.0 + uniform();
  const int e = lo_e + (int)(uniform() * (hi_e - lo_e + 1));
  const double v = std::ldexp(m, e);
  return (next_u64() & 1) ? -v : v;
}
static long double exact(ff x) { return (long double)x.hi + (long double)x.lo; }
static bool normalised(ff x) {
  if (x.hi == 0.0f) return x.lo == 0.0f;
  const float ulp = std::nextafter(std::fabs(x.hi), INFINITY) - std::fabs(x.hi);
  return std::fabs(x.lo) <= 0.5f * ulp;
}

int main() {
  int fails = 0;
  double worst_rt = 0, worst_split = 0, worst_add = 0, worst_mul = 0, worst_back = 0, worst_rcp = 0, worst_fast = 0;
  for (int t = 0; t < 200000; ++t) {
    const double v = rand_double(-100, 100);
    const ff a = psd::ff_from_double_bits(v);
    if (!normalised(a)) ++fails;
    const double rel_split = (double)(std::fabs(exact(a) - (long double)v) / std::fabs((long double)v));
    if (rel_split > worst_split) worst_split = rel_split;
    const double back = psd::ff_to_double_bits(a);
    const double rel_rt = std::fabs(back - v) / std::fabs(v);
    if (rel_rt > worst_rt) worst_rt = rel_rt;
    // to double: within one ulp of the exact hi + lo
    const long double ex = exact(a);
    const double rel_b = (double)(std::fabs((long double)back - ex) / std::fabs(ex));
    if (rel_b > worst_back) worst_back = rel_b;
    // sum and product of two double-words
    const ff b = psd::ff_from_double_bits(rand_double(-30, 30));
    const ff c = psd::ff_from_double_bits(rand_double(-30, 30));
    const ff s = psd::ff_add(b, c), p = psd::ff_mul(b, c);
    const long double es = exact(b) + exact(c), ep = exact(b) * exact(c);
    if (es != 0) {
      const double r = (double)(std::fabs(exact(s) - es) / std::fabs(es));
      if (r > worst_add) worst_add = r;
    }
    const double rp = (double)(std::fabs(exact(p) - ep) / std::fabs(ep));
    if (rp > worst_mul) worst_mul = rp;
    if (!normalised(s) || !normalised(p)) ++fails;
    // the butterfly sum: absolute error within a few u^2 (|b| + |c|), also under cancellation
    {
      const ff cc = (t & 1) ? psd::ff_neg(psd::ff_add(b, psd::ff_from_double_bits(rand_double(-60, -40)))) : c;
      const ff q = psd::ff_add_fast(b, cc);
      const long double eq = exact(b) + exact(cc);
      const double r = (double)(std::fabs(exact(q) - eq) / (std::fabs(exact(b)) + std::fabs(exact(cc))));
      if (r > worst_fast) worst_fast = r;
      if (!normalised(q)) ++fails;
    }
    // reciprocal of a positive double-word (the symbols of -Delta_h)
    const ff m = psd::ff_from_double_bits(std::fabs(rand_double(-20, 20)));
    const ff rm = psd::ff_recip(m);
    const double rr = (double)std::fabs(exact(rm) * exact(m) - 1.0L);
    if (rr > worst_rcp) worst_rcp = rr;
  }
  // special values
  if (psd::ff_to_double_bits(psd::ff_from_double_bits(0.0)) != 0.0) ++fails;
  if (!std::isinf(psd::ff_to_double_bits(psd::ff_from_double_bits(1e300)))) ++fails;
  if (!std::isnan(psd::ff_to_double_bits(psd::ff_from_double_bits(NAN)))) ++fails;
  if (psd::ff_to_double_bits(psd::ff_from_double_bits(-1e-300)) != 0.0) ++fails;
  if (std::signbit(psd::ff_to_double_bits(psd::ff_from_double_bits(-1e-300))) == 0) ++fails;
  // exact values: powers of two and small integers survive the round trip
  for (int k = -120; k <= 120; ++k) {
    const double v = std::ldexp(1.0, k) * 3.0;
    if (psd::ff_to_double_bits(psd::ff_from_double_bits(v)) != v) ++fails;
  }
  // fixed point: round(v 2^S), ties away from zero, against long double
  // (64-bit significand: v 2^S is exact there) and llroundl
  {
    int fx_fails = 0;
    for (int t = 0; t < 200000; ++t) {
      const int S = -40 + (int)(uniform() * 200.0);          // scales in [-40, 159]
      const double v = rand_double(-70 - S, 60 - S);          // |v| 2^S in [2^-70, 2^61)
      const long long want = llroundl(ldexpl((long double)v, S));
      if (psd::fx_from_double(v, S) != want) ++fx_fails;
    }
    // ties (k + 1/2) 2^-S, both signs; zeros; subnormals; the largest values
    for (int k = -1000; k <= 1000; ++k) {
      const int S = 7 + (k & 31);
      const double v = std::ldexp((double)k + 0.5, -S);
      const long long want = k >= 0 ? (long long)k + 1 : (long long)k;  // away from zero
      if (psd::fx_from_double(v, S) != want) ++fx_fails;
    }
    if (psd::fx_from_double(0.0, 55) != 0 || psd::fx_from_double(-0.0, 55) != 0) ++fx_fails;
    if (psd::fx_from_double(std::ldexp(1.0, -1074), 1074) != 1) ++fx_fails;           // smallest subnormal
    if (psd::fx_from_double(-std::ldexp(3.0, -1074), 1073) != -2) ++fx_fails;         // 1.5 -> 2
    if (psd::fx_from_double(std::ldexp(1.0, -1074), 1000) != 0) ++fx_fails;
    if (psd::fx_from_double(std::nextafter(std::ldexp(1.0, 8), 0.0), 53) != (1LL << 61) - 256) ++fx_fails;  // exact
    if (psd::fx_from_double(-std::ldexp(1.0, 61), 0) != -(1LL << 61)) ++fx_fails;
    for (int S = -200; S <= 200; ++S)
      if (psd::fx_unit(S) != std::ldexp(1.0, -S)) ++fx_fails;
    // fixed point -> float-float: relative error below 2^-47, normalised,
    // exact for values with at most 24 significant bits
    double worst_fx = 0;
    for (int t = 0; t < 200000; ++t) {
      const int S = 15 + (int)(uniform() * 106.0);  // [15, 120]
      const int bits = 1 + (int)(uniform() * 62.0);
      long long x = (long long)(next_u64() >> (64 - bits));
      if (next_u64() & 1) x = -x;
      const ff z = psd::fx_to_ff(x, S);
      if (!normalised(z)) ++fx_fails;
      const long double ex = ldexpl((long double)x, -S);
      if (x == 0) {
        if (z.hi != 0.0f || z.lo != 0.0f) ++fx_fails;
        continue;
      }
      const double r = (double)(std::fabs(exact(z) - ex) / std::fabs(ex));
      if (r > worst_fx) worst_fx = r;
      if (bits <= 24 && exact(z) != ex) ++fx_fails;
    }
    if (worst_fx > 0x1p-47) ++fx_fails;
    // fixed point -> double: the same value as the C++ conversion (nearest, ties to even)
    for (int t = 0; t < 200000; ++t) {
      const int bits = 1 + (int)(uniform() * 62.0);
      long long x = (long long)(next_u64() >> (64 - bits));
      if (next_u64() & 1) x = -x;
      if (psd::fx_to_double(x) != (double)x) ++fx_fails;
    }
    for (int k = 53; k <= 62; ++k) {  // ties at every shift: both even and odd neighbours
      const long long base = 1LL << k, half = 1LL << (k - 53);
      for (long long x : {base + half, base + 3 * half, base - 1, 0x7FFFFFFFFFFFFFFFLL})
        if (psd::fx_to_double(x) != (double)x || psd::fx_to_double(-x) != (double)(-x)) ++fx_fails;
    }
    if (psd::fx_to_ff((1LL << 62) + 1, 62).hi != 1.0f) ++fx_fails;
    if (psd::fx_to_ff(-(3LL << 40), 41).hi != -1.5f) ++fx_fails;
    std::printf("fixed point: %d mismatches (to float-float: worst %.3g = %.2f units of 2^-48)\n", fx_fails,
                worst_fx, worst_fx / 0x1p-48);
    fails += fx_fails;
  }
  const double u2 = 0x1p-48;
  std::printf("split %.3g  roundtrip %.3g  to_double %.3g  add %.3g  mul %.3g  (units of 2^-48: %.2f %.2f %.2f %.2f %.2f)\n",
              worst_split, worst_rt, worst_back, worst_add, worst_mul, worst_split / u2, worst_rt / u2,
              worst_back / u2, worst_add / u2, worst_mul / u2);
  if (worst_split > 0x1p-47 || worst_rt > 0x1p-47 || worst_back > 0x1p-52 || worst_add > 4 * u2 ||
      worst_mul > 6 * u2)
    ++fails;
  std::printf("recip %.3g (%.2f units of 2^-48)  fast sum %.3g (%.2f units of 2^-48, normwise)\n", worst_rcp,
              worst_rcp / u2, worst_fast, worst_fast / u2);
  if (worst_rcp > 8 * u2 || worst_fast > 4 * u2) ++fails;
  std::printf("%s (%d failures)\n", fails ? "FAIL" : "OK", fails);
  return fails ? 1 : 0;
}
