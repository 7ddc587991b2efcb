// mpw_device.cuh -- device helpers shared by the libmpw kernels: closed-form
// solutions, 1-D Lagrange weights, the direct tensor-product interpolation and
// the enumeration of hollow-box shells.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "mpw_fxmath.cuh"
#include "mpw_index.cuh"
#include "mpw_internal.cuh"

namespace mpw {

// Closed forms (Sec. 3): spherical Gaussian pulse pairs, plane-wave sums and
// the static harmonic basis.  psi = [g(t+r) - g(t-r)] / (2r) with
// g(s) = A s exp(-s^2/w^2) solves the wave equation with psi(0) = A
// exp(-r^2/w^2), Pi(0) = 0; Pi is its time derivative.  Near r = 0 the
// quotient is replaced by its Taylor expansion g'(t) + r^2 g'''(t)/6.
// One Gaussian pulse pair at squared distance r2 from its centre (a = 1/w^2).
__device__ __forceinline__ void gauss_pulse(double A, double a, double r2, double t, double& ps, double& pv) {
  if (r2 < 1e-10) {  // r < 1e-5: Taylor series in r of the same expression
    const double r2_6 = r2 / 6.0;
    const double e = A * exp(-a * t * t), t2 = t * t;
    const double g1 = e * (1.0 - 2.0 * a * t2);
    const double g2 = e * (4.0 * a * a * t2 * t - 6.0 * a * t);
    const double g3 = e * (-6.0 * a + 24.0 * a * a * t2 - 8.0 * a * a * a * t2 * t2);
    const double g4 = e * (60.0 * a * a * t - 80.0 * a * a * a * t2 * t + 16.0 * a * a * a * a * t2 * t2 * t);
    ps += g1 + r2_6 * g3;
    pv += g2 + r2_6 * g4;
    return;
  }
  double r, inv;  // r and 1/(2r)
  sqrt_pair_fx(r2, r, inv);
  const double sp = t + r, sm = t - r;
  const double qp = -a * sp * sp, qm = -a * sm * sm;
  const double ep = exp_nonpos_fx(qp), em = exp_nonpos_fx(qm), ia = A * inv;
  ps += (ep * sp - em * sm) * ia;
  pv += (ep * (1.0 + 2.0 * qp) - em * (1.0 + 2.0 * qm)) * ia;
}

// Sum of Gaussian pulses (params 5 per pulse), accumulated into ps, pv.
// apre (may be null): 1/width^2 of every pulse, precomputed.
__device__ __forceinline__ void gauss_sum(const double* __restrict__ P, const float4* __restrict__ screen,
                                          const double* __restrict__ apre, int count, double t, double x, double y,
                                          double z, double& ps, double& pv) {
  const float xf = (float)x, yf = (float)y, zf = (float)z, tf = fabsf((float)t) * 1.000001f;
  for (int q = 0; q < count; ++q) {
    if (screen) {
      const float4 s = screen[q];
      const float ex = xf - s.x, ey = yf - s.y, ez = zf - s.z, lim = tf + s.w;
      if (ex * ex + ey * ey + ez * ez > lim * lim) continue;
    }
    const double* g = P + 5 * q;
    const double dx = x - g[2], dy = y - g[3], dz = z - g[4];
    const double a = apre ? apre[q] : 1.0 / (g[1] * g[1]);
    gauss_pulse(g[0], a, dx * dx + dy * dy + dz * dz, t, ps, pv);
  }
}

// Constant plus plane waves (params C, then 5 per wave), accumulated.
__device__ __forceinline__ void plane_sum(const double* __restrict__ P, int count, double t, double x, double y,
                                          double z, double& ps, double& pv) {
  ps += P[0];
  for (int q = 0; q < count; ++q) {
    const double* wv = P + 1 + 5 * q;
    const double kk = sqrt(wv[1] * wv[1] + wv[2] * wv[2] + wv[3] * wv[3]);
    double sn, cs;
    sincos(wv[1] * x + wv[2] * y + wv[3] * z - kk * t + wv[4], &sn, &cs);
    ps += wv[0] * sn;
    pv -= wv[0] * kk * cs;
  }
}

// The closed forms of mpw_set_analytic (kinds GAUSS_SUM 0, PLANE_SUM 1,
// HARMONIC_POLY 2, PLANE_GAUSS 3) at time t and point (x, y, z).
__device__ __forceinline__ void closed_form(int kind, const double* __restrict__ P, const float4* __restrict__ screen,
                                            const double* __restrict__ apre, int count, double t, double x, double y,
                                            double z, double& ps, double& pv) {
  ps = 0.0;
  pv = 0.0;
  if (kind == 0) {
    gauss_sum(P, screen, apre, count, t, x, y, z, ps, pv);
  } else if (kind == 1) {
    plane_sum(P, count, t, x, y, z, ps, pv);
  } else if (kind == 3) {
    // one plane wave plus the pulses: the wave equation is linear
    plane_sum(P, 1, t, x, y, z, ps, pv);
    gauss_sum(P + 6, screen, apre, count, t, x, y, z, ps, pv);
  } else {
    const double basis[14] = {1.0,
                              x,
                              y,
                              z,
                              x * y,
                              y * z,
                              z * x,
                              x * x - y * y,
                              y * y - z * z,
                              x * y * z,
                              x * (x * x - 3.0 * y * y),
                              y * (y * y - 3.0 * z * z),
                              z * (z * z - 3.0 * x * x),
                              (x * x - y * y) * (x * x - y * y) - 4.0 * x * x * y * y};
    for (int q = 0; q < count && q < 14; ++q) ps += P[q] * basis[q];
  }
}

__device__ __forceinline__ int wrap_index(int i, int n) { return ((i % n) + n) % n; }

// ---------------------------------------------------------------------------
// 1-D Lagrange weights of the window that starts two nodes below
// i_c = floor(s) (Sec. 2.4, Eq. Pijk).  With u = s - i_c and node offsets
// o_m = m - 2, w_m = prod_{q != m} (u - o_q) / prod_{q != m} (o_m - o_q); the
// numerators come from prefix and suffix products.
template <int P>
__device__ __forceinline__ int lagrange_weights(double s, double* w) {
  const double fl = floor(s);
  const double u = s - fl;
  double d[P], pre[P + 1], suf[P + 1];
#pragma unroll
  for (int m = 0; m < P; ++m) d[m] = u - (double)(m - 2);
  pre[0] = 1.0;
  suf[P] = 1.0;
#pragma unroll
  for (int m = 0; m < P; ++m) pre[m + 1] = pre[m] * d[m];
#pragma unroll
  for (int m = P - 1; m >= 0; --m) suf[m] = suf[m + 1] * d[m];
  if (P == 6) {
    const double inv[6] = {-1.0 / 120.0, 1.0 / 24.0, -1.0 / 12.0, 1.0 / 12.0, -1.0 / 24.0, 1.0 / 120.0};
#pragma unroll
    for (int m = 0; m < P; ++m) w[m] = pre[m] * suf[m + 1] * inv[m];
  } else {
    const double inv[5] = {1.0 / 24.0, -1.0 / 6.0, 1.0 / 4.0, -1.0 / 6.0, 1.0 / 24.0};
#pragma unroll
    for (int m = 0; m < P; ++m) w[m] = pre[m] * suf[m + 1] * inv[m];
  }
  return (int)fl - 2;
}

// Tensor-product interpolation of both fields of a donor box at the numeric
// position (x, y, z).  The window must lie inside the donor interior; returns
// false (point skipped) otherwise.
template <int P, typename ST>
__device__ __forceinline__ bool interp_point(const ST* __restrict__ src, const Geom& g, double x, double y, double z,
                             double& o0, double& o1) {
  double wx[P], wy[P], wz[P];
  const int sx = lagrange_weights<P>((x - g.lo[0]) / g.h[0] - 0.5, wx);
  const int sy = lagrange_weights<P>((y - g.lo[1]) / g.h[1] - 0.5, wy);
  const int sz = lagrange_weights<P>((z - g.lo[2]) / g.h[2] - 0.5, wz);
  if (sx < 0 || sy < 0 || sz < 0 || sx + P > g.n[0] || sy + P > g.n[1] || sz + P > g.n[2]) return false;
  const ST* s0 = src;
  const ST* s1 = src + g.vol;
  double a0 = 0.0, a1 = 0.0;
#pragma unroll
  for (int c = 0; c < P; ++c) {
    double b0 = 0.0, b1 = 0.0;
#pragma unroll
    for (int b = 0; b < P; ++b) {
      const long long row = g.at(sx, sy + b, sz + c);
      double r0 = 0.0, r1 = 0.0;
#pragma unroll
      for (int a = 0; a < P; ++a) {
        r0 = fma(wx[a], (double)s0[row + a], r0);
        r1 = fma(wx[a], (double)s1[row + a], r1);
      }
      b0 = fma(wy[b], r0, b0);
      b1 = fma(wy[b], r1, b1);
    }
    a0 = fma(wz[c], b0, a0);
    a1 = fma(wz[c], b1, a1);
  }
  o0 = a0;
  o1 = a1;
  return true;
}


// ---------------------------------------------------------------------------
// Spherical shells (numeric r, theta, phi; phi periodic over [0, 2 pi)).
// Cartesian patch frame of the shell point (r, theta, phi).
__device__ __forceinline__ void sph_to_cart(double r, double th, double ph, double x[3]) {
  double st, ct, sp, cp;
  sincos(th, &st, &ct);
  sincos(ph, &sp, &cp);
  x[0] = r * st * cp;
  x[1] = r * st * sp;
  x[2] = r * ct;
}

// (r, theta, phi) of a point of the Cartesian patch frame.
__device__ __forceinline__ void cart_to_sph(const double x[3], double q[3]) {
  const double r = sqrt((x[0] * x[0] + x[1] * x[1]) + x[2] * x[2]);
  const double c = r > 0.0 ? fmin(fmax(x[2] / r, -1.0), 1.0) : 1.0;
  double ph = atan2(x[1], x[0]);
  if (ph < 0.0) ph += 2.0 * 3.14159265358979323846;
  q[0] = r;
  q[1] = acos(c);
  q[2] = ph;
}

// Tensor-product interpolation on a shell at numeric (r, theta, phi): the r
// and theta windows must lie in the interior, the phi window wraps.
template <int P, typename ST>
__device__ __forceinline__ bool interp_point_shell(const ST* __restrict__ src, const Geom& g, double r, double th,
                                                   double ph, double& o0, double& o1) {
  double wx[P], wy[P], wz[P];
  const int sx = lagrange_weights<P>((r - g.lo[0]) / g.h[0] - 0.5, wx);
  const int sy = lagrange_weights<P>((th - g.lo[1]) / g.h[1] - 0.5, wy);
  const int sz = lagrange_weights<P>((ph - g.lo[2]) / g.h[2] - 0.5, wz);
  if (sx < 0 || sy < 0 || sx + P > g.n[0] || sy + P > g.n[1]) return false;
  const ST* s0 = src;
  const ST* s1 = src + g.vol;
  double a0 = 0.0, a1 = 0.0;
#pragma unroll 1
  for (int c = 0; c < P; ++c) {
    const int kz = wrap_index(sz + c, g.n[2]);
    double b0 = 0.0, b1 = 0.0;
#pragma unroll
    for (int b = 0; b < P; ++b) {
      const long long row = g.at(sx, sy + b, kz);
      double r0 = 0.0, r1 = 0.0;
#pragma unroll
      for (int a = 0; a < P; ++a) {
        r0 = fma(wx[a], (double)s0[row + a], r0);
        r1 = fma(wx[a], (double)s1[row + a], r1);
      }
      b0 = fma(wy[b], r0, b0);
      b1 = fma(wy[b], r1, b1);
    }
    a0 = fma(wz[c], b0, a0);
    a1 = fma(wz[c], b1, a1);
  }
  o0 = a0;
  o1 = a1;
  return true;
}

// ---------------------------------------------------------------------------
// Patch maps X_B = R X' + X0 (Sec. 2.4, numeric -> background).  The cover
// flags are discrete decisions taken on these positions, so the two helpers
// below round every operation as written (no contraction): the same
// operations in the same order on the host give the same bits.
// Cell-centred node lo + (i + 1/2) h.
__device__ __forceinline__ double node_rn(double lo, int i, double h) {
  return __dadd_rn(lo, __dmul_rn((double)i + 0.5, h));
}

// X' = R^T (X_B - X0), R row-major.
__device__ __forceinline__ void to_local_rn(const double* __restrict__ R, const double* __restrict__ X0, double xb,
                                            double yb, double zb, double xl[3]) {
  const double d0 = __dsub_rn(xb, X0[0]), d1 = __dsub_rn(yb, X0[1]), d2 = __dsub_rn(zb, X0[2]);
#pragma unroll
  for (int a = 0; a < 3; ++a)
    xl[a] = __dadd_rn(__dadd_rn(__dmul_rn(R[a], d0), __dmul_rn(R[3 + a], d1)), __dmul_rn(R[6 + a], d2));
}

// X_B = R X' + X0, rounded as written (the closed-form initial data of a
// rotating patch is then sampled at the oracle's very positions).
__device__ __forceinline__ void to_background_rn(const double* __restrict__ R, const double* __restrict__ X0, double x,
                                                 double y, double z, double xb[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
    xb[a] = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(R[3 * a], x), __dmul_rn(R[3 * a + 1], y)), __dmul_rn(R[3 * a + 2], z)),
                      X0[a]);
}

// General affine position M x + c (interpolation only: rounding here moves a
// point by ulps, which the interpolant absorbs).
__device__ __forceinline__ void affine(const double* __restrict__ M, const double* __restrict__ c, double x, double y,
                                       double z, double& ox, double& oy, double& oz) {
  ox = fma(M[0], x, fma(M[1], y, fma(M[2], z, c[0])));
  oy = fma(M[3], x, fma(M[4], y, fma(M[5], z, c[1])));
  oz = fma(M[6], x, fma(M[7], y, fma(M[8], z, c[2])));
}

}  // namespace mpw
