// mpw_fixed.cuh -- exact fixed-point helpers for binary64 stencil arithmetic.
//
// GB300 executes FP64 FMAs at ~1/70 of its FP32/INT32 issue rate, so the
// stencil sums of the RHS are done in 64-bit integers instead.  A field
// buffer whose largest biased exponent is E is mapped onto integers at the
// scale 2^(E-1075): every value with exponent <= E becomes
//   q = round(x * 2^(1075-E)),   |q| < 2^53,
// exactly when its exponent is E and with an error below half a unit of
// 2^(E-1075) (half an ulp of the buffer's largest values) otherwise.  Integer
// sums of such q with small integer weights are then exact.  Real
// coefficients are applied as 64 x 64 -> high-64 products, and the result is
// rounded once back to binary64 by integer normalisation.
#pragma once
#include <cstdint>

namespace mpw {

// Exponent slots per patch: [buffer][field] of the live values (written by
// the RHS, the exponent scan and revival), then the same for the ghost
// values written by the ghost fill (EXP_GHOST on).  A buffer's scale is the
// larger of its two slots.
constexpr int EXP_SLOTS_PER_PATCH = 16;
constexpr int EXP_GHOST = 8;
constexpr int EXP_NONFINITE = 2047;

// Biased exponent field of a binary64 value (0 for zero/subnormal, 2047 for
// Inf/NaN).
__device__ __forceinline__ int biased_exponent(double x) {
  return (int)((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF;
}

// q = round-half-up(|x| * 2^(1075-E)) with the sign of x; 0 for values whose
// exponent exceeds E (such entries are never read by a live stencil: they are
// deactivated or stale cells of the buffer, see the exponent bookkeeping).
__device__ __forceinline__ long long to_fixed(double x, int E) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)(b >> 52) & 0x7FF;
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (e ? 0x10000000000000ull : 0ull);
  int sh = E - (e ? e : 1);
  if (sh < 0) return 0;
  sh = sh > 63 ? 63 : sh;
  const unsigned long long r = (m + ((1ull << sh) >> 1)) >> sh;
  return (b >> 63) ? -(long long)r : (long long)r;
}

// v * 2^S rounded to nearest-even binary64 (v != 0 has at most 63 bits).
__device__ __forceinline__ double fixed_to_double(long long v, int S) {
  if (v == 0) return 0.0;
  const unsigned long long sign = (unsigned long long)v & 0x8000000000000000ull;
  const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  int sh = 11 - __clzll((long long)a);  // a >> sh has 53 significant bits
  unsigned long long m;
  if (sh > 0) {
    const unsigned long long rem = a & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    m = a >> sh;
    if (rem > half || (rem == half && (m & 1ull))) ++m;
    if (m >> 53) {
      m >>= 1;
      ++sh;
    }
  } else {
    m = a << (-sh);
  }
  const int e = sh + S + 1075;
  if (e <= 0) return __longlong_as_double((long long)sign);
  return __longlong_as_double((long long)(sign | ((unsigned long long)e << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

// Signed high 64 bits of the 128-bit product a * b.
__device__ __forceinline__ long long mulhi(long long a, long long b) { return __mul64hi(a, b); }

// Fixed-point multiplier for a term coef * I * 2^(E-1075) accumulated at the
// output scale 2^S: M = round(coef * 2^(E - 1075 - S + 64)), so that the term
// equals mulhi(I, M) units of 2^S.  Computed once per CTA.
__device__ __forceinline__ long long term_multiplier(double coef, int E, int S) {
  if (coef == 0.0) return 0;
  return __double2ll_rn(scalbn(coef, E - 1075 - S + 64));
}

// Smallest output scale S with |coef| * 2^(E - 1075 - S) < 1/8 (so a sum of up
// to nine terms of at most 2^61 * 2^-3 stays inside int64).
__device__ __forceinline__ int term_scale(double coef, int E) {
  if (coef == 0.0) return -100000;
  return ilogb(coef) + E - 1075 + 4;
}

}  // namespace mpw
