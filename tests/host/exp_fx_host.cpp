// Host build of the fixed-point exponential of the analytic boundary
// (csrc/mpw_exp.cuh) with plain C++ stand-ins for the four CUDA intrinsics
// it names.  Prints the largest error, in units in the last place, against
// the long double exp over seeded arguments, then the special cases.
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
using std::exp;
#include "../../paper_2002_00088_gb300/csrc/mpw_exp.cuh"

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
  std::printf("zero %.17g\n", mpw::exp_nonpos_fx(0.0));
  std::printf("negzero %.17g\n", mpw::exp_nonpos_fx(-0.0));
  std::printf("tiny %.17g\n", mpw::exp_nonpos_fx(-1e-300));
  std::printf("m704 %.17g\n", mpw::exp_nonpos_fx(-704.0));
  std::printf("minf %.17g\n", mpw::exp_nonpos_fx(-INFINITY));
  std::printf("nan %d\n", (int)std::isnan(mpw::exp_nonpos_fx(NAN)));
  std::printf("m703 %.17g %.17g\n", mpw::exp_nonpos_fx(-703.99), (double)expl((long double)-703.99));
  return 0;
}
