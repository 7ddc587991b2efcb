// mpw_rhs.cu -- fused RHS + RK4 stage kernel (Sec. 2.2-2.3) for every patch
// of one substage, in one launch.
//
// Per live point (4th-order centred differences, KO with n = 5, frame
// velocity w of a translating patch):
//   K_psi = Pi + w . D1 psi + KO(psi)
//   K_Pi  = sum_a D2_a psi + w . D1 Pi + KO(Pi)
// then the RK4 stage combination (Table 1, Eqs. k1-k4):
//   stage 0: ACC = U + dt/6 K,  OUT = U + dt/2 K
//   stage 1: ACC += dt/3 K,     OUT = U + dt/2 K
//   stage 2: ACC += dt/3 K,     OUT = U + dt K
//   stage 3:                    OUT(=U) = ACC + dt/6 K
//
// Traversal: a CTA owns a TX x TY column tile and marches zc planes; the z
// neighbours of its own column live in a 7-deep register queue, the x/y
// neighbours of the current plane in shared memory (halo 3, star stencil).
//
// Arithmetic (template FIXED):
//   true  -- stencil inputs are converted once, on load, to exact int64 fixed
//            point at the scale of their buffer's tracked maximum exponent
//            (mpw_fixed.cuh); all stencil sums are exact integer sums, the
//            coefficients are applied as 64x64->128 high products, and K is
//            rounded once to binary64.  Only the stage combination uses the
//            FP64 pipe (4 FMAs per point).  A CTA whose input buffer holds a
//            non-finite live value falls back to the FP64 formulas, so NaN and
//            Inf propagate as in IEEE arithmetic.
//   false -- native FP64 throughout (the reference GPU path).
#include <cuda_runtime.h>

#include <cstdint>

#include "mpw_fixed.cuh"
#include "mpw_internal.cuh"

namespace mpw {

namespace {

// Term multipliers of one CTA (fixed-point path).
struct Terms {
  long long ms[7];  // K_psi: Pi_0, KO_x..z(psi) (or aggregated in [1]), D1_x..z(psi)
  long long mp[9];  // K_Pi : D2_x..z(psi) (or aggregated in [0]), KO_x..z(Pi) (or [3]), D1_x..z(Pi)
  int Ss, Sp;       // output scales of K_psi and K_Pi
  int Es, Ep;       // input scales (biased exponents) of psi and Pi
  int fixed;        // 0: FP64 fallback for this CTA
};

__device__ void setup_terms(Terms& T, const RhsPatch& P, int Es_raw, int Ep_raw, bool want_fixed) {
  T.fixed = want_fixed && Es_raw < EXP_NONFINITE && Ep_raw < EXP_NONFINITE;
  if (!T.fixed) return;
  const int Es = max(Es_raw, 64), Ep = max(Ep_raw, 64);
  T.Es = Es;
  T.Ep = Ep;
  double cs[7], cp[9];
  int es[7], ep[9];
  cs[0] = 1.0;
  es[0] = Ep;
  for (int a = 0; a < 3; ++a) {
    cs[1 + a] = P.iso ? (a == 0 ? P.cko[0] : 0.0) : P.cko[a];
    es[1 + a] = Es;
    cs[4 + a] = P.c1[a];
    es[4 + a] = Es;
    cp[a] = P.iso ? (a == 0 ? P.c2[0] : 0.0) : P.c2[a];
    ep[a] = Es;
    cp[3 + a] = P.iso ? (a == 0 ? P.cko[0] : 0.0) : P.cko[a];
    ep[3 + a] = Ep;
    cp[6 + a] = P.c1[a];
    ep[6 + a] = Ep;
  }
  int Ss = -100000, Sp = -100000;
  for (int t = 0; t < 7; ++t) Ss = max(Ss, term_scale(cs[t], es[t]));
  for (int t = 0; t < 9; ++t) Sp = max(Sp, term_scale(cp[t], ep[t]));
  T.Ss = Ss;
  T.Sp = Sp;
  for (int t = 0; t < 7; ++t) T.ms[t] = term_multiplier(cs[t], es[t], Ss);
  for (int t = 0; t < 9; ++t) T.mp[t] = term_multiplier(cp[t], ep[t], Sp);
}

__device__ __forceinline__ int slot(int patch, int buf, int field) {
  return patch * EXP_SLOTS_PER_PATCH + buf * 2 + field;
}

}  // namespace

template <int TX, int TY, bool FIXED>
__global__ void __launch_bounds__(TX* TY, RHS_MIN_BLOCKS) k_rhs(const __grid_constant__ RhsArgs A) {
  __shared__ long long sm[2][TY + 6][TX + 6];
  __shared__ Terms T;
  const int b = blockIdx.x;
  int p = 0;
  while (p + 1 < A.np && b >= A.p[p + 1].block0) ++p;
  const RhsPatch& Pt = A.p[p];
  const Geom& g = Pt.g;
  if (threadIdx.x == 0)
    setup_terms(T, Pt, A.expo[slot(p, Pt.in_buf, 0)], A.expo[slot(p, Pt.in_buf, 1)], FIXED);
  int lb = b - Pt.block0;
  const int tx = lb % Pt.tiles_x;
  lb /= Pt.tiles_x;
  const int ty = lb % Pt.tiles_y;
  const int tz = lb / Pt.tiles_y;
  const int li = threadIdx.x % TX, lj = threadIdx.x / TX;
  const int i0 = tx * TX, j0 = ty * TY;
  const int i = i0 + li, j = j0 + lj;
  const int z0 = tz * Pt.zc, z1 = min(z0 + Pt.zc, g.n[2]);
  const bool in_box = (i < g.n[0] + NG) && (j < g.n[1] + NG);
  const bool in_xy = (i < g.n[0]) && (j < g.n[1]);
  bool check_flags = false;
  if (Pt.is_global) {
    for (int q = 0; q < A.nbox; ++q) {
      const Box& bx = A.box[q];
      if (bx.lo[0] <= i0 + TX - 1 && bx.hi[0] >= i0 && bx.lo[1] <= j0 + TY - 1 && bx.hi[1] >= j0 &&
          bx.lo[2] <= z1 - 1 && bx.hi[2] >= z0)
        check_flags = true;
    }
  }
  __syncthreads();
  const bool fx = FIXED && T.fixed;
  const int Es = T.Es, Ep = T.Ep;
  auto load = [&](const double* base, long long c, int E) -> long long {
    const double v = base[c];
    return fx ? to_fixed(v, E) : __double_as_longlong(v);
  };
  const double* Ys = Pt.Y;
  const double* Yp = Pt.Y + g.vol;
  long long qs[7], qp[7];
#pragma unroll
  for (int o = 0; o < 6; ++o) {
    qs[o] = 0;
    qp[o] = 0;
    if (in_box) {
      const long long c = g.at(i, j, z0 - NG + o);
      qs[o] = load(Ys, c, Es);
      qp[o] = load(Yp, c, Ep);
    }
  }
  // halo assignment: threads [0, 6 TX) load the y halo, [6 TX, 6 TX + 6 TY) the x halo
  const int t = threadIdx.x;
  int hi_ = -100, hj = -100, hsi = 0, hsj = 0;
  if (t < 6 * TX) {
    const int rr = t / TX, cc = t % TX;
    hsj = rr < 3 ? rr : TY + rr;
    hsi = cc + 3;
    hi_ = i0 + cc;
    hj = j0 + (rr < 3 ? rr - 3 : TY + rr - 3);
  } else if (t < 6 * TX + 6 * TY) {
    const int u = t - 6 * TX, rr = u / 6, cc = u % 6;
    hsj = rr + 3;
    hsi = cc < 3 ? cc : TX + cc;
    hj = j0 + rr;
    hi_ = i0 + (cc < 3 ? cc - 3 : TX + cc - 3);
  }
  const bool h_ok = hi_ >= -NG && hi_ < g.n[0] + NG && hj >= -NG && hj < g.n[1] + NG;
  constexpr int SY = TX + 6;
  int emax_s = 0, emax_p = 0;
  // software pipeline: the raw values of plane z+3 (own column) and of the
  // halo of plane z are loaded one iteration ahead
  double nx_s = 0.0, nx_p = 0.0, nh_s = 0.0, nh_p = 0.0;
  if (in_box && z0 < z1) {
    const long long c = g.at(i, j, z0 + NG);
    nx_s = Ys[c];
    nx_p = Yp[c];
  }
  if (h_ok && z0 < z1) {
    const long long c = g.at(hi_, hj, z0);
    nh_s = Ys[c];
    nh_p = Yp[c];
  }
  for (int z = z0; z < z1; ++z) {
    const long long cz = g.at(i, j, z);
    // operands of the stage combination and the cover flag, issued early
    double ua_s = 0.0, ua_p = 0.0, ub_s = 0.0, ub_p = 0.0;
    int fl = FLAG_LIVE;
    if (in_xy) {
      if (A.stage == 0) {
        ua_s = Ys[cz];
        ua_p = Yp[cz];
      } else {
        ub_s = Pt.ACC[cz];
        ub_p = Pt.ACC[cz + g.vol];
        if (A.stage != 3) {
          ua_s = Pt.U[cz];
          ua_p = Pt.U[cz + g.vol];
        }
      }
      if (check_flags) fl = A.flags[((long long)z * g.n[1] + j) * g.n[0] + i] & 3;
    }
    const long long hs_v = fx ? to_fixed(nh_s, Es) : __double_as_longlong(nh_s);
    const long long hp_v = fx ? to_fixed(nh_p, Ep) : __double_as_longlong(nh_p);
    qs[6] = fx ? to_fixed(nx_s, Es) : __double_as_longlong(nx_s);
    qp[6] = fx ? to_fixed(nx_p, Ep) : __double_as_longlong(nx_p);
    if (z + 1 < z1) {
      if (in_box) {
        const long long c = g.at(i, j, z + 1 + NG);
        nx_s = Ys[c];
        nx_p = Yp[c];
      }
      if (h_ok) {
        const long long c = g.at(hi_, hj, z + 1);
        nh_s = Ys[c];
        nh_p = Yp[c];
      }
    }
    __syncthreads();
    sm[0][lj + 3][li + 3] = qs[3];
    sm[1][lj + 3][li + 3] = qp[3];
    if (h_ok) {
      sm[0][hsj][hsi] = hs_v;
      sm[1][hsj][hsi] = hp_v;
    }
    __syncthreads();
    const bool live = in_xy && (fl == FLAG_LIVE || fl == FLAG_REVIVED);
    if (live) {
      const long long* rs = &sm[0][lj + 3][li + 3];
      const long long* rp = &sm[1][lj + 3][li + 3];
      double Ks, Kp;
      if (fx) {
        // ---- exact integer stencil sums
        const long long u0 = qs[3], v0 = qp[3];
        const long long xs1 = rs[-1] + rs[1], xs2 = rs[-2] + rs[2], xs3 = rs[-3] + rs[3];
        const long long ys1 = rs[-SY] + rs[SY], ys2 = rs[-2 * SY] + rs[2 * SY], ys3 = rs[-3 * SY] + rs[3 * SY];
        const long long zs1 = qs[2] + qs[4], zs2 = qs[1] + qs[5], zs3 = qs[0] + qs[6];
        const long long xp1 = rp[-1] + rp[1], xp2 = rp[-2] + rp[2], xp3 = rp[-3] + rp[3];
        const long long yp1 = rp[-SY] + rp[SY], yp2 = rp[-2 * SY] + rp[2 * SY], yp3 = rp[-3 * SY] + rp[3 * SY];
        const long long zp1 = qp[2] + qp[4], zp2 = qp[1] + qp[5], zp3 = qp[0] + qp[6];
        long long ks, kp;
        if (Pt.iso) {
          const long long S1 = xs1 + ys1 + zs1, S2 = xs2 + ys2 + zs2, S3 = xs3 + ys3 + zs3;
          const long long P1 = xp1 + yp1 + zp1, P2 = xp2 + yp2 + zp2, P3 = xp3 + yp3 + zp3;
          const long long d2 = 16 * S1 - S2 - 90 * u0;
          const long long kos = S3 - 6 * S2 + 15 * S1 - 60 * u0;
          const long long kop = P3 - 6 * P2 + 15 * P1 - 60 * v0;
          ks = mulhi(v0, T.ms[0]) + mulhi(kos, T.ms[1]);
          kp = mulhi(d2, T.mp[0]) + mulhi(kop, T.mp[3]);
        } else {
          ks = mulhi(v0, T.ms[0]) + mulhi(xs3 - 6 * xs2 + 15 * xs1 - 20 * u0, T.ms[1]) +
               mulhi(ys3 - 6 * ys2 + 15 * ys1 - 20 * u0, T.ms[2]) +
               mulhi(zs3 - 6 * zs2 + 15 * zs1 - 20 * u0, T.ms[3]);
          kp = mulhi(16 * xs1 - xs2 - 30 * u0, T.mp[0]) + mulhi(16 * ys1 - ys2 - 30 * u0, T.mp[1]) +
               mulhi(16 * zs1 - zs2 - 30 * u0, T.mp[2]) + mulhi(xp3 - 6 * xp2 + 15 * xp1 - 20 * v0, T.mp[3]) +
               mulhi(yp3 - 6 * yp2 + 15 * yp1 - 20 * v0, T.mp[4]) +
               mulhi(zp3 - 6 * zp2 + 15 * zp1 - 20 * v0, T.mp[5]);
        }
        if (Pt.moving) {
          ks += mulhi(8 * (rs[1] - rs[-1]) - (rs[2] - rs[-2]), T.ms[4]) +
                mulhi(8 * (rs[SY] - rs[-SY]) - (rs[2 * SY] - rs[-2 * SY]), T.ms[5]) +
                mulhi(8 * (qs[4] - qs[2]) - (qs[5] - qs[1]), T.ms[6]);
          kp += mulhi(8 * (rp[1] - rp[-1]) - (rp[2] - rp[-2]), T.mp[6]) +
                mulhi(8 * (rp[SY] - rp[-SY]) - (rp[2 * SY] - rp[-2 * SY]), T.mp[7]) +
                mulhi(8 * (qp[4] - qp[2]) - (qp[5] - qp[1]), T.mp[8]);
        }
        Ks = fixed_to_double(ks, T.Ss);
        Kp = fixed_to_double(kp, T.Sp);
      } else {
        // ---- native FP64
        auto D = [](long long v) { return __longlong_as_double(v); };
        const double u0 = D(qs[3]), v0 = D(qp[3]);
        const double xs1 = D(rs[-1]) + D(rs[1]), xs2 = D(rs[-2]) + D(rs[2]), xs3 = D(rs[-3]) + D(rs[3]);
        const double ys1 = D(rs[-SY]) + D(rs[SY]), ys2 = D(rs[-2 * SY]) + D(rs[2 * SY]),
                     ys3 = D(rs[-3 * SY]) + D(rs[3 * SY]);
        const double zs1 = D(qs[2]) + D(qs[4]), zs2 = D(qs[1]) + D(qs[5]), zs3 = D(qs[0]) + D(qs[6]);
        const double xp1 = D(rp[-1]) + D(rp[1]), xp2 = D(rp[-2]) + D(rp[2]), xp3 = D(rp[-3]) + D(rp[3]);
        const double yp1 = D(rp[-SY]) + D(rp[SY]), yp2 = D(rp[-2 * SY]) + D(rp[2 * SY]),
                     yp3 = D(rp[-3 * SY]) + D(rp[3 * SY]);
        const double zp1 = D(qp[2]) + D(qp[4]), zp2 = D(qp[1]) + D(qp[5]), zp3 = D(qp[0]) + D(qp[6]);
        const double d2 = Pt.c2[0] * (16.0 * xs1 - xs2 - 30.0 * u0) + Pt.c2[1] * (16.0 * ys1 - ys2 - 30.0 * u0) +
                          Pt.c2[2] * (16.0 * zs1 - zs2 - 30.0 * u0);
        const double kos = Pt.cko[0] * (xs3 - 6.0 * xs2 + 15.0 * xs1 - 20.0 * u0) +
                           Pt.cko[1] * (ys3 - 6.0 * ys2 + 15.0 * ys1 - 20.0 * u0) +
                           Pt.cko[2] * (zs3 - 6.0 * zs2 + 15.0 * zs1 - 20.0 * u0);
        const double kop = Pt.cko[0] * (xp3 - 6.0 * xp2 + 15.0 * xp1 - 20.0 * v0) +
                           Pt.cko[1] * (yp3 - 6.0 * yp2 + 15.0 * yp1 - 20.0 * v0) +
                           Pt.cko[2] * (zp3 - 6.0 * zp2 + 15.0 * zp1 - 20.0 * v0);
        Ks = v0 + kos;
        Kp = d2 + kop;
        if (Pt.moving) {
          Ks += Pt.c1[0] * (8.0 * (D(rs[1]) - D(rs[-1])) - (D(rs[2]) - D(rs[-2]))) +
                Pt.c1[1] * (8.0 * (D(rs[SY]) - D(rs[-SY])) - (D(rs[2 * SY]) - D(rs[-2 * SY]))) +
                Pt.c1[2] * (8.0 * (D(qs[4]) - D(qs[2])) - (D(qs[5]) - D(qs[1])));
          Kp += Pt.c1[0] * (8.0 * (D(rp[1]) - D(rp[-1])) - (D(rp[2]) - D(rp[-2]))) +
                Pt.c1[1] * (8.0 * (D(rp[SY]) - D(rp[-SY])) - (D(rp[2 * SY]) - D(rp[-2 * SY]))) +
                Pt.c1[2] * (8.0 * (D(qp[4]) - D(qp[2])) - (D(qp[5]) - D(qp[1])));
        }
      }
      // ---- RK4 stage combination (FP64)
      const long long c = cz;
      double os, op;
      if (A.stage == 3) {
        os = fma(A.alpha, Ks, ub_s);
        op = fma(A.alpha, Kp, ub_p);
      } else {
        const double as = A.stage == 0 ? ua_s : ub_s;
        const double ap = A.stage == 0 ? ua_p : ub_p;
        os = fma(A.alpha, Ks, ua_s);
        op = fma(A.alpha, Kp, ua_p);
        Pt.ACC[c] = fma(A.beta, Ks, as);
        Pt.ACC[c + g.vol] = fma(A.beta, Kp, ap);
      }
      Pt.OUT[c] = os;
      Pt.OUT[c + g.vol] = op;
      emax_s = max(emax_s, biased_exponent(os));
      emax_p = max(emax_p, biased_exponent(op));
    }
#pragma unroll
    for (int o = 0; o < 6; ++o) {
      qs[o] = qs[o + 1];
      qp[o] = qp[o + 1];
    }
  }
  // exponent bookkeeping of the output buffer (consumed by the next substage)
  emax_s = __reduce_max_sync(0xffffffffu, emax_s);
  emax_p = __reduce_max_sync(0xffffffffu, emax_p);
  if ((threadIdx.x & 31) == 0) {
    if (emax_s) atomicMax(&A.expo[slot(p, Pt.out_buf, 0)], emax_s);
    if (emax_p) atomicMax(&A.expo[slot(p, Pt.out_buf, 1)], emax_p);
  }
}

void launch_rhs(const RhsArgs& a, int blocks, bool fixed, void* stream) {
  if (fixed)
    k_rhs<RHS_TX, RHS_TY, true><<<blocks, RHS_TX * RHS_TY, 0, (cudaStream_t)stream>>>(a);
  else
    k_rhs<RHS_TX, RHS_TY, false><<<blocks, RHS_TX * RHS_TY, 0, (cudaStream_t)stream>>>(a);
}

}  // namespace mpw
