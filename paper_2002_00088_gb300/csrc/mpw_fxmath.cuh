// mpw_fxmath.cuh -- exp(x) for x <= 0, and sqrt(y) with 1/(2 sqrt(y)), with
// the work in 64-bit integers.
//
// GB300 issues FP64 operations at a small fraction of its integer rate, and
// the Gaussian closed forms of the analytic boundary (Sec. 3) spend most of
// their FP64 operations in two exponentials and one reciprocal square root
// per pulse.
//
// exp_nonpos_fx keeps Tang's table-driven method (ACM TOMS 15(2), 1989):
// with y = -x >= 0,
//   n = round(64 y / ln2),  s = n ln2/64 - y  (|s| <= ln2/128),
//   exp(x) = 2^(-n/64) e^s = 2^k 2^(j/64) (1 + p(s)),  -n = 64 k + j,
// p the degree-5 Taylor polynomial of e^s - 1 (truncation below 4e-17), but
// takes y, the reduction, the polynomial and the product with 2^(j/64) in
// fixed point:
//   Y = round(y 2^53) (exact for |x| >= 1/2), ln2/64 split into its integer
//   part on 2^53 and 16 more bits, so s is formed on 2^69 with an error
//   below n 2^-70 <= 6e-17; the polynomial and the table 2^(j/64) on 2^62,
//   each product the high 64 bits of a 128-bit product;
// and assembles the binary64 result from the 63-bit mantissa with one
// rounding (half up).  The error is within about 1.5 units in the last place:
// the final rounding, the rounding of y to 2^-54 for |x| < 1/2, and the
// fixed-point steps (a few 2^-62).  x <= -704 (and -inf) gives 0, as results
// below 2^-1015 are flushed; NaN propagates.  The callers pass x = -a s^2
// with a > 0; x > 0 falls back to the library exp.
//
// sqrt_pair_fx writes y = g 4^k with g in [1, 4), refines z = 1/sqrt(g) from
// the single-precision estimate by two Newton steps z (3 - g z^2) / 2 on 2^62
// (the estimate's 2^-22 error squares twice), and forms sqrt(y) = g z 2^k and
// 1/(2 sqrt(y)) = z 2^(-k-1), each rounded once: within 0.53 units in the
// last place.  Non-finite or non-positive y falls back to the library
// functions.
//
// The file includes nothing: the CUDA intrinsics it names come from the
// translation units that include it.
#pragma once

namespace mpw {

// round(2^(j/64) 2^62), j = 0..63
static __device__ const long long g_exp2_q62[64] = {
    4611686018427387904ll, 4661903986662671290ll, 4712668792719003884ll, 4763986391269842979ll,
    4815862801830788490ll, 4868304109465667592ll, 4921316465500308116ll, 4974906088244084429ll,
    5029079263719320435ll, 5083842346398635251ll, 5139201759950318048ll, 5195163997991819502ll,
    5251735624851448219ll, 5308923276338361494ll, 5366733660520940721ll, 5425173558513642752ll,
    5484249825272419512ll, 5543969390398799154ll, 5604339258952723100ll, 5665366512274234280ll,
    5727058308814112983ll, 5789421884973557729ll, 5852464555953009676ll, 5916193716610220111ll,
    5980616842327661685ll, 6045741489889385141ll, 6111575298367424380ll, 6178125990017853852ll,
    6245401371186603363ll, 6313409333225136570ll, 6382157853416100552ll, 6451654995909055045ll,
    6521908912666391106ll, 6592927844419550153ll, 6664720121635655541ll, 6737294165494670078ll,
    6810658488877194079ll, 6884821697363019841ll, 6959792490240559659ll, 7035579661527265796ll,
    7112192101001162095ll, 7189638795243608238ll, 7267928828693418961ll, 7347071384712461870ll,
    7427075746662858866ll, 7507951298995917514ll, 7589707528352920109ll, 7672354024677899536ll,
    7755900482342532474ll, 7840356701283281883ll, 7925732588150922155ll, 8012038157472581778ll,
    8099283532826439817ll, 8187478948029213993ll, 8276634748336579668ll, 8366761391656660532ll,
    8457869449776733335ll, 8549969609603290562ll, 8643072674415606502ll, 8737189565132953757ll,
    8832331321595618838ll, 8928509103859867100ll, 9025734193507008925ll, 9124017994966720698ll};

// The binary64 of M 2^(E - 62) for M in [2^61, 2^63): 53 bits rounded half
// up.  Adding the mantissa with its leading bit to the exponent field one
// below also takes a carry out of the rounding into the exponent.
__device__ __forceinline__ double fx_to_double(long long M, int E) {
  const bool top = M >= (1ll << 62);
  const int sh = top ? 10 : 9;
  const long long r53 = ((M >> (sh - 1)) + 1) >> 1;
  const long long biased = (top ? 1023 : 1022) + E;
  return __longlong_as_double(((biased - 1) << 52) + r53);
}

__device__ __forceinline__ double exp_nonpos_fx(double x) {
  const long long bits = __double_as_longlong(x);
  const long long mag = bits & 0x7fffffffffffffffll;
  if (mag > 0x7ff0000000000000ll) return x;      // NaN
  if (mag >= 0x4086000000000000ll) return 0.0;   // |x| >= 704 (or infinite)
  if (bits > 0) return exp(x);                   // x > 0: not a case of the callers
  // Y = |x| 2^53 (< 2^62.5), rounded; |x| = mant 2^(e - 1075)
  const int e = (int)(mag >> 52);
  const long long mant = (mag & 0xfffffffffffffll) | 0x10000000000000ll;
  long long Y = 0;
  if (e >= 1022) {
    Y = mant << (e - 1022);                      // e - 1022 <= 10
  } else if (e > 1022 - 54) {
    const int sh = 1022 - e;                     // 1..53
    Y = ((mant >> (sh - 1)) + 1) >> 1;
  }                                              // else |x| < 2^-55 (or 0): Y = 0, the result is 1
  // n = round(Y (64/ln2) / 2^53) with 64/ln2 on 2^56
  const long long n = (long long)((__umul64hi((unsigned long long)Y, 6653256548922161246ull) + (1ull << 44)) >> 45);
  // s = n ln2/64 - y on 2^69: ln2/64 2^53 = 97551793252583 + 48342 / 2^16
  const long long D = Y - n * 97551793252583ll;               // |D| < 2^46
  const long long S = n * 48342ll - (D << 16);
  const long long s = S >> 7;                    // on 2^62, |s| < 2^55
  // p = s + s^2 (1/2 + s (1/6 + s (1/24 + s/120))) on 2^62
  long long q = 192153584101141163ll + (__mul64hi(s, 38430716820228233ll) << 2);
  q = 768614336404564651ll + (__mul64hi(s, q) << 2);
  q = (1ll << 61) + (__mul64hi(s, q) << 2);
  const long long p = s + (__mul64hi(__mul64hi(s, s) << 2, q) << 2);
  // 2^(j/64) (1 + p) on 2^62, in [2^61, 2^63)
  const long long m = -n;
  const long long T = __ldg(&g_exp2_q62[m & 63]);
  const long long M = T + (__mul64hi(T, p) << 2);
  return fx_to_double(M, (int)(m >> 6));  // times 2^k, k = floor(m / 64)
}

__device__ __forceinline__ void sqrt_pair_fx(double y, double& root, double& half_inv) {
  const long long bits = __double_as_longlong(y);
  const int e = (int)(bits >> 52);  // y > 0: the sign bit is clear
  if (bits <= 0 || e == 0 || e == 0x7ff) {  // y <= 0, subnormal, infinite or NaN
    root = sqrt(y);
    half_inv = 0.5 / root;
    return;
  }
  const int E = e - 1023, odd = E & 1, k = (E - odd) >> 1;
  const long long frac = bits & 0xfffffffffffffll;
  const long long g = (frac | 0x10000000000000ll) << (9 + odd);  // g on 2^61
  // estimate of 1/sqrt(g) from the binary32 of g, then on 2^62
  const float zf = rsqrtf(__int_as_float(((127 + odd) << 23) | (int)(frac >> 29)));
  const int zb = __float_as_int(zf);
  long long z = (long long)((zb & 0x7fffff) | 0x800000) << (((zb >> 23) & 0xff) - 88);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const long long z2 = __mul64hi(z, z) << 2;           // z^2 on 2^62
    const long long gz2 = __mul64hi(g, z2) << 3;         // g z^2 on 2^62
    const long long h = 3 * (1ll << 61) - (gz2 >> 1);    // (3 - g z^2) / 2 on 2^62
    z = __mul64hi(z, h) << 2;
  }
  half_inv = fx_to_double(z, -k - 1);
  // g z = sqrt(g) in [1, 2) on 2^59, taken to 2^61 (below 2^62 with room
  // for the truncation errors), that is M / 2^62 = sqrt(g) / 2
  root = fx_to_double(__mul64hi(g, z) << 2, k + 1);
}

}  // namespace mpw
