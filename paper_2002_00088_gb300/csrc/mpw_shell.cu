// mpw_shell.cu -- fused RHS + RK4 stage on spherical-shell local patches (the
// paper's spherical local patch, Sec. 3.3), plain FP64, one thread per point.
//
// Numeric coordinates (r, theta, phi); the flat metric in spherical
// coordinates (appendix, with g_phiphi = r^2 sin^2 theta) turns the two-field
// system of the Cartesian patches into
//   K_psi = Pi + w . D psi + KO(psi)
//   K_Pi  = lap psi + w . D Pi + KO(Pi)
//   lap u   = u_rr + (2/r) u_r + (u_thth + cot(theta) u_th) / r^2 + u_phph / (r^2 sin^2 theta)
//   w . D u = w_r u_r + (w_th / r) u_th + (w_ph / (r sin theta)) u_ph
// with w_r, w_th, w_ph the frame velocity on the unit vectors r^, theta^,
// phi^, every derivative the 4th-order centred difference along its index
// axis, and KO per axis over that axis' physical spacing (h_r, r h_theta,
// r sin(theta) h_phi).  The stage combination is that of the Cartesian
// kernel (Table 1, Eqs. k1-k4).
#include <cuda_runtime.h>

#include "mpw_device.cuh"
#include "mpw_fixed.cuh"
#include "mpw_internal.cuh"

namespace mpw {

namespace {

constexpr int SHELL_THREADS = 256;

__device__ __forceinline__ double fd1(const double* u, long long s, double h) {
  return (u[-2 * s] - 8.0 * u[-s] + 8.0 * u[s] - u[2 * s]) / (12.0 * h);
}
__device__ __forceinline__ double fd2(const double* u, long long s, double h) {
  return (-u[-2 * s] + 16.0 * u[-s] - 30.0 * u[0] + 16.0 * u[s] - u[2 * s]) / (12.0 * h * h);
}
__device__ __forceinline__ double fko(const double* u, long long s, double L, double eps) {
  return (eps / 64.0) * (u[-3 * s] - 6.0 * u[-2 * s] + 15.0 * u[-s] - 20.0 * u[0] + 15.0 * u[s] - 6.0 * u[2 * s] +
                         u[3 * s]) /
         L;
}

}  // namespace

__global__ void __launch_bounds__(SHELL_THREADS) k_rhs_shell(const __grid_constant__ ShellArgs A) {
  const long long b = blockIdx.x;
  int p = 0;
  while (p + 1 < A.np && b >= A.p[p + 1].block0) ++p;
  const ShellPatch& S = A.p[p];
  const Geom& g = S.g;
  const long long idx = (b - S.block0) * SHELL_THREADS + threadIdx.x;
  const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
  int e0 = 0, e1 = 0;
  if (idx < N) {
    const int i = (int)(idx % g.n[0]);
    const int j = (int)((idx / g.n[0]) % g.n[1]);
    const int k = (int)(idx / ((long long)g.n[0] * g.n[1]));
    const double r = g.lo[0] + (i + 0.5) * g.h[0], th = g.lo[1] + (j + 0.5) * g.h[1],
                 ph = g.lo[2] + (k + 0.5) * g.h[2];
    double sn, cs, sp, cp;
    sincos(th, &sn, &cs);
    sincos(ph, &sp, &cp);
    const long long c = g.at(i, j, k);
    const long long st[3] = {1, g.px, g.plane};
    double wr = 0.0, wt = 0.0, wp = 0.0;
    if (S.moving) {
      const double x[3] = {r * sn * cp, r * sn * sp, r * cs};
      double w[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) w[a] = S.w0[a] + S.W[3 * a] * x[0] + S.W[3 * a + 1] * x[1] + S.W[3 * a + 2] * x[2];
      wr = w[0] * sn * cp + w[1] * sn * sp + w[2] * cs;
      wt = w[0] * cs * cp + w[1] * cs * sp - w[2] * sn;
      wp = -w[0] * sp + w[1] * cp;
    }
    const double Lr = g.h[0], Lt = r * g.h[1], Lp = r * sn * g.h[2];
    double K[2];
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const double* u = S.Y + f * g.vol + c;
      double k_f = fko(u, st[0], Lr, A.ko_eps) + fko(u, st[1], Lt, A.ko_eps) + fko(u, st[2], Lp, A.ko_eps);
      if (S.moving)
        k_f += wr * fd1(u, st[0], g.h[0]) + (wt / r) * fd1(u, st[1], g.h[1]) + (wp / (r * sn)) * fd1(u, st[2], g.h[2]);
      K[f] = k_f;
    }
    const double* ps = S.Y + c;
    const double lap = fd2(ps, st[0], g.h[0]) + (2.0 / r) * fd1(ps, st[0], g.h[0]) +
                       (fd2(ps, st[1], g.h[1]) + (cs / sn) * fd1(ps, st[1], g.h[1])) / (r * r) +
                       fd2(ps, st[2], g.h[2]) / (r * r * sn * sn);
    const double Ks = S.Y[g.vol + c] + K[0], Kp = lap + K[1];
    // RK4 stage combination
    double os, op;
    if (A.stage == 3) {
      os = fma(A.alpha, Ks, S.ACC[c]);
      op = fma(A.alpha, Kp, S.ACC[c + g.vol]);
    } else {
      const double us = S.U[c], up = S.U[c + g.vol];
      const double as = A.stage == 0 ? us : S.ACC[c], ap = A.stage == 0 ? up : S.ACC[c + g.vol];
      os = fma(A.alpha, Ks, us);
      op = fma(A.alpha, Kp, up);
      S.ACC[c] = fma(A.beta, Ks, as);
      S.ACC[c + g.vol] = fma(A.beta, Kp, ap);
    }
    S.OUT[c] = os;
    S.OUT[c + g.vol] = op;
    e0 = biased_exponent(os);
    e1 = biased_exponent(op);
  }
  // exponent slots of the output buffer (the fixed-point scale of the fills
  // that read this shell)
  e0 = __reduce_max_sync(0xffffffffu, e0);
  e1 = __reduce_max_sync(0xffffffffu, e1);
  if ((threadIdx.x & 31) == 0) {
    if (e0) atomicMax(&A.expo[S.patch * EXP_SLOTS_PER_PATCH + A.out_buf * 2], e0);
    if (e1) atomicMax(&A.expo[S.patch * EXP_SLOTS_PER_PATCH + A.out_buf * 2 + 1], e1);
  }
}

void launch_rhs_shell(const ShellArgs& a, long long blocks, void* stream) {
  if (blocks <= 0) return;
  k_rhs_shell<<<(unsigned)blocks, SHELL_THREADS, 0, (cudaStream_t)stream>>>(a);
}

}  // namespace mpw
