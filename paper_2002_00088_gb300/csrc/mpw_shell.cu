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

// Centred-difference combinations with their 1/h factors applied by the
// caller: 12 h D1, 12 h^2 D2 and the sixth difference of KO.
__device__ __forceinline__ double s1(const double* u, long long s) { return (u[-2 * s] - u[2 * s]) + 8.0 * (u[s] - u[-s]); }
__device__ __forceinline__ double s2(const double* u, long long s) {
  return 16.0 * (u[-s] + u[s]) - (u[-2 * s] + u[2 * s]) - 30.0 * u[0];
}
__device__ __forceinline__ double s6(const double* u, long long s) {
  return (u[-3 * s] + u[3 * s]) - 6.0 * (u[-2 * s] + u[2 * s]) + 15.0 * (u[-s] + u[s]) - 20.0 * u[0];
}

}  // namespace

// The node tables (see ShellPatch) replace every transcendental and every
// division of the point loop: GB300 runs FP64 at a small fraction of its
// integer rate, and a division is a Newton sequence there.
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
    const double* T = S.tab;
    const double r = T[i], ir = T[g.n[0] + i];
    const double* Tt = T + 2 * g.n[0];
    const double sn = Tt[j], cs = Tt[g.n[1] + j], isn = Tt[2 * g.n[1] + j];
    const double* Tp = Tt + 3 * g.n[1];
    const double sp = Tp[k], cp = Tp[g.n[2] + k];
    const long long c = g.at(i, j, k);
    const long long st[3] = {1, g.px, g.plane};
    // 1/(12 h), 1/(12 h^2) per axis, and the KO factor eps / (64 L)
    const double d1[3] = {S.id1[0], S.id1[1], S.id1[2]};
    const double ko[3] = {S.iko[0], S.iko[1] * ir, S.iko[2] * ir * isn};
    double wr = 0.0, wt = 0.0, wp = 0.0;
    if (S.moving) {
      const double x[3] = {r * sn * cp, r * sn * sp, r * cs};
      double w[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) w[a] = S.w0[a] + S.W[3 * a] * x[0] + S.W[3 * a + 1] * x[1] + S.W[3 * a + 2] * x[2];
      wr = (w[0] * sn * cp + w[1] * sn * sp + w[2] * cs) * d1[0];
      wt = (w[0] * cs * cp + w[1] * cs * sp - w[2] * sn) * ir * d1[1];
      wp = (-w[0] * sp + w[1] * cp) * ir * isn * d1[2];
    }
    double K[2];
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const double* u = S.Y + f * g.vol + c;
      double k_f = ko[0] * s6(u, st[0]) + ko[1] * s6(u, st[1]) + ko[2] * s6(u, st[2]);
      if (S.moving) k_f += wr * s1(u, st[0]) + wt * s1(u, st[1]) + wp * s1(u, st[2]);
      K[f] = k_f;
    }
    const double* ps = S.Y + c;
    const double ir2 = ir * ir;
    const double lap = S.id2[0] * s2(ps, st[0]) + 2.0 * ir * d1[0] * s1(ps, st[0]) +
                       ir2 * (S.id2[1] * s2(ps, st[1]) + cs * isn * d1[1] * s1(ps, st[1])) +
                       ir2 * isn * isn * S.id2[2] * s2(ps, st[2]);
    const double Ks = S.Y[g.vol + c] + K[0], Kp = lap + K[1];
    // RK4 stage combination
    double os, op;
    if (A.stage == 3) {
      os = fma(S.alpha, Ks, S.ACC[c]);
      op = fma(S.alpha, Kp, S.ACC[c + g.vol]);
    } else {
      const double us = S.U[c], up = S.U[c + g.vol];
      const double as = A.stage == 0 ? us : S.ACC[c], ap = A.stage == 0 ? up : S.ACC[c + g.vol];
      os = fma(S.alpha, Ks, us);
      op = fma(S.alpha, Kp, up);
      S.ACC[c] = fma(S.beta, Ks, as);
      S.ACC[c + g.vol] = fma(S.beta, Kp, ap);
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
    if (e0) atomicMax(&S.expo[S.patch * EXP_SLOTS_PER_PATCH + A.out_buf * 2], e0);
    if (e1) atomicMax(&S.expo[S.patch * EXP_SLOTS_PER_PATCH + A.out_buf * 2 + 1], e1);
  }
}

void launch_rhs_shell(const ShellArgs& a, long long blocks, void* stream) {
  if (blocks <= 0) return;
  k_rhs_shell<<<(unsigned)blocks, SHELL_THREADS, 0, (cudaStream_t)stream>>>(a);
}

}  // namespace mpw
