// Host build of the fixed-point exp and square root of the analytic
// boundary (csrc/mpw_fxmath.cuh) with plain C++ stand-ins for the CUDA
// intrinsics it names.  Prints the largest errors, in units in the last
// place, against the long double exp and sqrt over seeded arguments, then
// the special cases.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>

#define __device__
#define __forceinline__ inline
static inline long long __double_as_longlong(double x) {
  long long r;
  std::memcpy(&r, &x, 8);
  return r;
}
static inline double __longlong_as_double(long long x) {
  double r;
  std::memcpy(&r, &x, 8);
  return r;
}
static inline long long __mul64hi(long long a, long long b) { return (long long)(((__int128)a * b) >> 64); }
static inline unsigned long long __umul64hi(unsigned long long a, unsigned long long b) {
  return (unsigned long long)(((unsigned __int128)a * b) >> 64);
}
template <class T>
static inline T __ldg(const T* p) {
  return *p;
}
static inline float __int_as_float(int x) {
  float r;
  std::memcpy(&r, &x, 4);
  return r;
}
static inline int __float_as_int(float x) {
  int r;
  std::memcpy(&r, &x, 4);
  return r;
}
// the device estimate is within about 2 units of binary32; this one is
// rounded down in the last bit to stand in for an estimate that is not
// correctly rounded
static inline float rsqrtf(float x) { return __int_as_float(__float_as_int(1.0f / std::sqrt(x)) ^ 1); }
using std::exp;
using std::sqrt;
#include "../../paper_2002_00088_gb300/csrc/mpw_fxmath.cuh"

int main(int argc, char** argv) {
  const long count = argc > 1 ? std::atol(argv[1]) : 1000000;
  std::mt19937_64 g(20020088);
  std::uniform_real_distribution<double> u(0.0, 1.0);
  double worst = 0.0, wx = 0.0;
  auto check = [&](double x) {
    const double a = mpw::exp_nonpos_fx(x);
    const long double r = expl((long double)x);
    const double ulp = std::ldexp(1.0, std::ilogb((double)r) - 52);
    const double err = (double)fabsl((long double)a - r) / ulp;
    if (err > worst) worst = err, wx = x;
  };
  for (long i = 0; i < count; ++i) {
    check(-u(g) * 703.9);                              // whole range
    check(-u(g) * 60.0);                               // the Gaussian tails that matter
    check(-std::ldexp(u(g), -(int)(u(g) * 60.0)));     // small |x|, down to 2^-60
    check(-(double)(i % 65000) * 0.0108304892 + 1e-7 * (u(g) - 0.5));  // near multiples of ln2/64
  }
  std::printf("worst_ulp %.6f at %.17g\n", worst, wx);
  // sqrt and 1/(2 sqrt) over the squared distances of the closed forms
  double wr = 0.0, wi = 0.0, xr = 0.0, xi = 0.0;
  auto check_sqrt = [&](double y) {
    double r, h;
    mpw::sqrt_pair_fx(y, r, h);
    const long double R = sqrtl((long double)y), H = 0.5L / R;
    const double er = (double)fabsl((long double)r - R) / std::ldexp(1.0, std::ilogb((double)R) - 52);
    const double ei = (double)fabsl((long double)h - H) / std::ldexp(1.0, std::ilogb((double)H) - 52);
    if (er > wr) wr = er, xr = y;
    if (ei > wi) wi = ei, xi = y;
  };
  for (long i = 0; i < count; ++i) {
    check_sqrt(std::ldexp(1.0 + u(g), (int)(u(g) * 80.0) - 40));
    check_sqrt(u(g) * 12.0 + 1e-10);
    check_sqrt(4.0 * (1.0 - std::ldexp(u(g), -40)));  // just below a power of 4
  }
  for (double y : {1e-10, 1.0, 4.0, 2.0, 0.25, 3.9999999999999996, 1.0000000000000002, 1e300, 1e-300})
    check_sqrt(y);
  std::printf("worst_sqrt_ulp %.6f at %.17g\n", wr, xr);
  std::printf("worst_half_inv_ulp %.6f at %.17g\n", wi, xi);
  {
    double r, h;
    mpw::sqrt_pair_fx(4.0, r, h);
    std::printf("sqrt4 %.17g %.17g\n", r, h);
    mpw::sqrt_pair_fx(NAN, r, h);
    std::printf("sqrtnan %d\n", (int)(std::isnan(r) && std::isnan(h)));
  }
  std::printf("zero %.17g\n", mpw::exp_nonpos_fx(0.0));
  std::printf("negzero %.17g\n", mpw::exp_nonpos_fx(-0.0));
  std::printf("tiny %.17g\n", mpw::exp_nonpos_fx(-1e-300));
  std::printf("m704 %.17g\n", mpw::exp_nonpos_fx(-704.0));
  std::printf("minf %.17g\n", mpw::exp_nonpos_fx(-INFINITY));
  std::printf("nan %d\n", (int)std::isnan(mpw::exp_nonpos_fx(NAN)));
  std::printf("m703 %.17g %.17g\n", mpw::exp_nonpos_fx(-703.99), (double)expl((long double)-703.99));
  return 0;
}
