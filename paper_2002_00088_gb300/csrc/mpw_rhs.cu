// mpw_rhs.cu -- fused RHS + RK4 stage kernel (Sec. 2.2-2.3) for every patch
// of one substage, in one launch.
//
// Per live point (4th-order centred differences, KO with n = 5, frame
// velocity w: constant on a translating patch, w(X') = Omega n x X' + R^T V
// on a rotating one):
//   K_psi = Pi + w . D1 psi + KO(psi)
//   K_Pi  = sum_a D2_a psi + w . D1 Pi + KO(Pi)
// then the RK4 stage combination (Table 1, Eqs. k1-k4):
//   stage 0: ACC = U + dt/6 K,  OUT = U + dt/2 K
//   stage 1: ACC += dt/3 K,     OUT = U + dt/2 K
//   stage 2: ACC += dt/3 K,     OUT = U + dt K
//   stage 3:                    OUT(=U) = ACC + dt/6 K
//
// Traversal: a CTA owns a 32 x 8 column tile and marches zc planes.  The raw
// input tile of each plane (with its x/y halo) and the stage operands arrive
// by TMA (cp.async.bulk.tensor) several planes ahead; each value is converted
// once, the z neighbours of a thread's own column then live in a 7-deep
// register queue and the x/y neighbours in a small ring of converted planes in
// shared memory (halo 3, star stencil).
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
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mpw_fixed.cuh"
#include "mpw_internal.cuh"
#include "mpw_tma.cuh"

namespace mpw {

namespace {

// Term multipliers of one CTA (fixed-point path).
struct Terms {
  long long ms[7];  // K_psi: Pi_0, KO_x..z(psi) (or aggregated in [1]), D1_x..z(psi)
  long long mp[9];  // K_Pi : D2_x..z(psi) (or aggregated in [0]), KO_x..z(Pi) (or [3]), D1_x..z(Pi)
  long long gs[3][3], gp[3][3];  // rotating frame: D1 multipliers per unit of i, j, k (psi, Pi)
  int Ss, Sp;       // output scales of K_psi and K_Pi
  int Es, Ep;       // input scales (biased exponents) of psi and Pi
  int fixed;        // 0: FP64 fallback for this CTA
  double fa[2], fb[2];  // stage coefficients alpha, beta applied to K (psi, Pi), scaled by 2^S
};

__device__ void setup_terms(Terms& T, const RhsPatch& P, int Es_raw, int Ep_raw, bool want_fixed, double alpha,
                            double beta) {
  T.fa[0] = T.fa[1] = alpha;
  T.fb[0] = T.fb[1] = beta;
  T.fixed = want_fixed && Es_raw < EXP_NONFINITE && Ep_raw < EXP_NONFINITE;
  if (!T.fixed) return;
  const int Es = max(Es_raw, 64), Ep = max(Ep_raw, 64);
  T.Es = Es;
  T.Ep = Ep;
  double cs[7], cp[9];
  int es[7], ep[9];
  // D1 coefficients for the scales: c1 itself, or on a rotating patch the
  // largest |c1_a| over the patch (c1 is then affine in the indices, so its
  // extremes sit at the corners)
  double c1m[3] = {P.c1[0], P.c1[1], P.c1[2]};
  if (P.rot)
    for (int a = 0; a < 3; ++a) {
      c1m[a] = fabs(P.c1[a]);
      for (int c = 0; c < 8; ++c) {
        double v = P.c1[a];
        for (int b = 0; b < 3; ++b) v += P.c1g[a][b] * (((c >> b) & 1) ? P.g.n[b] - 1 : 0);
        c1m[a] = fmax(c1m[a], fabs(v));
      }
    }
  cs[0] = 1.0;
  es[0] = Ep;
  for (int a = 0; a < 3; ++a) {
    cs[1 + a] = P.iso ? (a == 0 ? P.cko[0] : 0.0) : P.cko[a];
    es[1 + a] = Es;
    cs[4 + a] = c1m[a];
    es[4 + a] = Es;
    cp[a] = P.iso ? (a == 0 ? P.c2[0] : 0.0) : P.c2[a];
    ep[a] = Es;
    cp[3 + a] = P.iso ? (a == 0 ? P.cko[0] : 0.0) : P.cko[a];
    ep[3 + a] = Ep;
    cp[6 + a] = c1m[a];
    ep[6 + a] = Ep;
  }
  int Ss = -100000, Sp = -100000;
  for (int t = 0; t < 7; ++t) Ss = max(Ss, term_scale(cs[t], es[t]));
  for (int t = 0; t < 9; ++t) Sp = max(Sp, term_scale(cp[t], ep[t]));
  T.Ss = Ss;
  T.Sp = Sp;
  for (int t = 0; t < 7; ++t) T.ms[t] = term_multiplier(cs[t], es[t], Ss);
  for (int t = 0; t < 9; ++t) T.mp[t] = term_multiplier(cp[t], ep[t], Sp);
  // rotating frame: D1 multipliers of c1 at cell (0, 0, 0), and their steps
  // per index (thread 0 of every CTA runs this: the FP64 work stays off the
  // translating patches)
  if (P.rot)
    for (int a = 0; a < 3; ++a) {
      T.ms[4 + a] = term_multiplier(P.c1[a], Es, Ss);
      T.mp[6 + a] = term_multiplier(P.c1[a], Ep, Sp);
      for (int b = 0; b < 3; ++b) {
        T.gs[a][b] = term_multiplier(P.c1g[a][b], Es, Ss);
        T.gp[a][b] = term_multiplier(P.c1g[a][b], Ep, Sp);
      }
    }
  // K = k 2^S with k the exact int64 sum: the stage updates use alpha 2^S and
  // beta 2^S (exact scalings), or the FP64 path when they would leave the
  // normal range
  if (Ss < -960 || Sp < -960 || Ss > 960 || Sp > 960) {
    T.fixed = 0;
    return;
  }
  T.fa[0] = scalbn(alpha, Ss);
  T.fb[0] = scalbn(beta, Ss);
  T.fa[1] = scalbn(alpha, Sp);
  T.fb[1] = scalbn(beta, Sp);
}

__device__ __forceinline__ int slot(int patch, int buf, int field) {
  return patch * EXP_SLOTS_PER_PATCH + buf * 2 + field;
}

}  // namespace

// ---------------------------------------------------------------------------
// TMA pipeline.  Iteration z of a CTA consumes one ring slot holding the raw
// tile (with halo) of input plane z+3 and the stage operands u and ACC of
// plane z; slots are refilled RHS_DEPTH iterations ahead by one elected
// thread with cp.async.bulk.tensor, completion tracked by one mbarrier per
// slot.  Every wait is bounded: a wait that runs out sets ERR_TIMEOUT in the
// error word, the CTA drains its own copies (again bounded) and returns.
#ifndef MPW_RHS_DEPTH
#define MPW_RHS_DEPTH 4
#endif
constexpr int RHS_DEPTH = MPW_RHS_DEPTH;  // planes in flight per CTA
constexpr int BOX_X = RHS_TX + 8, BOX_Y = RHS_TY + 6;
constexpr int TILE_DOUBLES = BOX_X * BOX_Y * 2;
constexpr int PT_DOUBLES = RHS_TX * RHS_TY * 2;
constexpr int SLOT_DOUBLES = TILE_DOUBLES + 2 * PT_DOUBLES;  // tile | u | ACC
constexpr int CONV_PLANE = (RHS_TY + 6) * (RHS_TX + 6);      // one field of a converted plane
constexpr int CONV_SLOTS = 4;
constexpr size_t RHS_SMEM = 1024 + sizeof(double) * RHS_DEPTH * SLOT_DOUBLES +
                            sizeof(long long) * CONV_SLOTS * 2 * CONV_PLANE + 8 * RHS_DEPTH;
// Issue the loads of iteration zz (tile of input plane zz+3, u and ACC of
// plane zz) into slot s.
__device__ __forceinline__ void issue_slot(const RhsPatch& Pt, int stage, double* slot, unsigned bar, int i0, int j0,
                                           int zz) {
  const unsigned bytes = sizeof(double) * (TILE_DOUBLES + (stage < 3 ? PT_DOUBLES : 0) + (stage > 0 ? PT_DOUBLES : 0));
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  bar_expect_tx(bar, bytes);
  // tile: columns from interior i0 - 4 (padded column i0 + xoff - 4), rows from interior j0 - 3 (padded row j0)
  tma_load_4d(smem_u32(slot), &Pt.ymap, i0 + Pt.g.xoff - 4, j0, zz + 3 + NG, 0, bar);
  if (stage < 3) tma_load_4d(smem_u32(slot + TILE_DOUBLES), &Pt.umap, i0 + Pt.g.xoff, j0 + NG, zz + NG, 0, bar);
  if (stage > 0) tma_load_4d(smem_u32(slot + TILE_DOUBLES + PT_DOUBLES), &Pt.amap, i0 + Pt.g.xoff, j0 + NG, zz + NG, 0, bar);
}

// Body of the kernel for block b of the launch described by A (A may sit in
// kernel parameter space or, for a batched launch, in global memory).
template <int TX, int TY, bool FIXED, bool ROT>
__device__ __forceinline__ void rhs_body(const RhsArgs& A, const int b) {
  static_assert(TX == RHS_TX && TY == RHS_TY, "TMA boxes are sized for RHS_TX x RHS_TY tiles");
  extern __shared__ unsigned char smem_dyn[];
  __shared__ Terms T;
  __shared__ int s_abort;
  constexpr int SY = TX + 6;
  // 1 KB-aligned carve-up of the dynamic shared memory
  const unsigned long long base = (reinterpret_cast<unsigned long long>(smem_dyn) + 1023ull) & ~1023ull;
  double* slots = reinterpret_cast<double*>(base);
  long long* conv = reinterpret_cast<long long*>(slots + RHS_DEPTH * SLOT_DOUBLES);
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(conv + CONV_SLOTS * 2 * CONV_PLANE);
  int p = 0;
  while (p + 1 < A.np && b >= A.p[p + 1].block0) ++p;
  const RhsPatch& Pt = A.p[p];
  const Geom& g = Pt.g;
  int lb = b - Pt.block0;
  const int tx = lb % Pt.tiles_x;
  lb /= Pt.tiles_x;
  const int ty = lb % Pt.tiles_y;
  const int tz = lb / Pt.tiles_y;
  const int li = threadIdx.x % TX, lj = threadIdx.x / TX;
  const int i0 = tx * TX, j0 = ty * TY;
  const int i = i0 + li, j = j0 + lj;
  const int z0 = tz * Pt.zc, z1 = min(z0 + Pt.zc, g.n[2]);
  if (threadIdx.x == 0) {
    // input scale: live values and the ghost values the fill wrote
    const int Es = max(A.expo[slot(p, Pt.in_buf, 0)], A.expo[slot(p, Pt.in_buf, 0) + EXP_GHOST]);
    const int Ep = max(A.expo[slot(p, Pt.in_buf, 1)], A.expo[slot(p, Pt.in_buf, 1) + EXP_GHOST]);
    setup_terms(T, Pt, Es, Ep, FIXED, A.alpha, A.beta);
    s_abort = 0;
    for (int s = 0; s < RHS_DEPTH; ++s) bar_init(smem_u32(&bars[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int s = 0; s < RHS_DEPTH && z0 + s < z1; ++s)
      issue_slot(Pt, A.stage, slots + s * SLOT_DOUBLES, smem_u32(&bars[s]), i0, j0, z0 + s);
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
  // halo assignment: threads [0, 6 TX) carry the y halo, [6 TX, 6 TX + 6 TY) the x halo
  const int t = threadIdx.x;
  int hi_ = -100, hj = -100, hoff = 0;
  if (t < 6 * TX) {
    const int rr = t / TX, cc = t % TX;
    hoff = (rr < 3 ? rr : TY + rr) * SY + cc + 3;
    hi_ = i0 + cc;
    hj = j0 + (rr < 3 ? rr - 3 : TY + rr - 3);
  } else if (t < 6 * TX + 6 * TY) {
    const int u = t - 6 * TX, rr = u / 6, cc = u % 6;
    hoff = (rr + 3) * SY + (cc < 3 ? cc : TX + cc);
    hj = j0 + rr;
    hi_ = i0 + (cc < 3 ? cc - 3 : TX + cc - 3);
  }
  const bool h_ok = hi_ >= -NG && hi_ < g.n[0] + NG && hj >= -NG && hj < g.n[1] + NG;
  const int own = (lj + 3) * SY + li + 3;
  // positions in a raw tile slot (x from interior i0 - 4, y from interior j0 - 3)
  const int own_raw = (lj + 3) * BOX_X + li + 4;
  const int halo_raw = (hj - j0 + 3) * BOX_X + (hi_ - i0 + 4);
  const bool fx = FIXED && T.fixed;
  const int Es = T.Es, Ep = T.Ep;
  const double* Ys = Pt.Y;
  const double* Yp = Pt.Y + g.vol;
  auto cvt = [&](double v, int E) -> long long { return fx ? to_fixed(v, E) : __double_as_longlong(v); };
  auto conv_of = [&](int zz) -> long long* { return conv + ((zz - z0) & (CONV_SLOTS - 1)) * 2 * CONV_PLANE; };
  // prologue: planes z0-3 .. z0+2 by plain loads (queue), z0 .. z0+2 also into the converted ring
  long long qs[7], qp[7];
#pragma unroll
  for (int o = 0; o < 6; ++o) {
    const int zz = z0 - NG + o;
    qs[o] = 0;
    qp[o] = 0;
    if (in_box) {
      const long long c = g.at(i, j, zz);
      qs[o] = cvt(Ys[c], Es);
      qp[o] = cvt(Yp[c], Ep);
    }
    if (o >= NG && zz < z1) {
      long long* cv = conv_of(zz);
      cv[own] = qs[o];
      cv[CONV_PLANE + own] = qp[o];
      if (h_ok) {
        const long long c = g.at(hi_, hj, zz);
        cv[hoff] = cvt(Ys[c], Es);
        cv[CONV_PLANE + hoff] = cvt(Yp[c], Ep);
      }
    }
  }
  int emax_s = 0, emax_p = 0;
  for (int z = z0; z < z1; ++z) {
    const int it = z - z0;
    const int s = it % RHS_DEPTH;
    const double* sl = slots + s * SLOT_DOUBLES;
    const unsigned bar = smem_u32(&bars[s]);
    int fl = FLAG_LIVE;
    if (in_xy && check_flags) fl = A.flags[((long long)z * g.n[1] + j) * g.n[0] + i] & 3;
    if (!bar_wait(bar, (unsigned)(it / RHS_DEPTH) & 1u)) s_abort = 1;
    // raw values of this iteration
    const double rs_own = sl[own_raw], rp_own = sl[BOX_X * BOX_Y + own_raw];
    double rs_h = 0.0, rp_h = 0.0;
    if (h_ok) {
      rs_h = sl[halo_raw];
      rp_h = sl[BOX_X * BOX_Y + halo_raw];
    }
    const int pt = lj * TX + li;
    double ua_s = 0.0, ua_p = 0.0, ub_s = 0.0, ub_p = 0.0;
    if (A.stage < 3) {
      ua_s = sl[TILE_DOUBLES + pt];
      ua_p = sl[TILE_DOUBLES + TX * TY + pt];
    }
    if (A.stage > 0) {
      ub_s = sl[TILE_DOUBLES + PT_DOUBLES + pt];
      ub_p = sl[TILE_DOUBLES + PT_DOUBLES + TX * TY + pt];
    }
    __syncthreads();
    if (s_abort) {
      // drain this CTA's copies still in flight (bounded), report, leave
      if (threadIdx.x == 0) {
        atomicOr(A.err, ERR_TIMEOUT);
        for (int k = it; k < it + RHS_DEPTH && z0 + k < z1; ++k)
          bar_wait(smem_u32(&bars[k % RHS_DEPTH]), (unsigned)(k / RHS_DEPTH) & 1u);
      }
      return;
    }
    if (threadIdx.x == 0 && z + RHS_DEPTH < z1)
      issue_slot(Pt, A.stage, slots + s * SLOT_DOUBLES, bar, i0, j0, z + RHS_DEPTH);
    // plane z+3 enters the queue (its converted plane is stored after the compute)
    qs[6] = cvt(rs_own, Es);
    qp[6] = cvt(rp_own, Ep);
    // every thread computes (points outside the patch or not live read valid
    // shared memory and store nothing), so the block has no divergent branch
    const bool live = in_xy && (fl == FLAG_LIVE || fl == FLAG_REVIVED);
    {
      const long long* rs = conv_of(z) + own;
      const long long* rp = rs + CONV_PLANE;
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
        if (ROT && Pt.rot) {
          // multipliers of c1_a(i, j, z), affine in the indices
          long long m[6];
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            m[a] = T.ms[4 + a] + T.gs[a][0] * i + T.gs[a][1] * j + T.gs[a][2] * z;
            m[3 + a] = T.mp[6 + a] + T.gp[a][0] * i + T.gp[a][1] * j + T.gp[a][2] * z;
          }
          ks += mulhi(8 * (rs[1] - rs[-1]) - (rs[2] - rs[-2]), m[0]) +
                mulhi(8 * (rs[SY] - rs[-SY]) - (rs[2 * SY] - rs[-2 * SY]), m[1]) +
                mulhi(8 * (qs[4] - qs[2]) - (qs[5] - qs[1]), m[2]);
          kp += mulhi(8 * (rp[1] - rp[-1]) - (rp[2] - rp[-2]), m[3]) +
                mulhi(8 * (rp[SY] - rp[-SY]) - (rp[2 * SY] - rp[-2 * SY]), m[4]) +
                mulhi(8 * (qp[4] - qp[2]) - (qp[5] - qp[1]), m[5]);
        } else if (Pt.moving) {
          ks += mulhi(8 * (rs[1] - rs[-1]) - (rs[2] - rs[-2]), T.ms[4]) +
                mulhi(8 * (rs[SY] - rs[-SY]) - (rs[2 * SY] - rs[-2 * SY]), T.ms[5]) +
                mulhi(8 * (qs[4] - qs[2]) - (qs[5] - qs[1]), T.ms[6]);
          kp += mulhi(8 * (rp[1] - rp[-1]) - (rp[2] - rp[-2]), T.mp[6]) +
                mulhi(8 * (rp[SY] - rp[-SY]) - (rp[2 * SY] - rp[-2 * SY]), T.mp[7]) +
                mulhi(8 * (qp[4] - qp[2]) - (qp[5] - qp[1]), T.mp[8]);
        }
        Ks = (double)ks;  // K_psi / 2^Ss, rounded once
        Kp = (double)kp;
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
          double c1[3] = {Pt.c1[0], Pt.c1[1], Pt.c1[2]};
          if (ROT && Pt.rot)
#pragma unroll
            for (int a = 0; a < 3; ++a) c1[a] += Pt.c1g[a][0] * i + Pt.c1g[a][1] * j + Pt.c1g[a][2] * z;
          Ks += c1[0] * (8.0 * (D(rs[1]) - D(rs[-1])) - (D(rs[2]) - D(rs[-2]))) +
                c1[1] * (8.0 * (D(rs[SY]) - D(rs[-SY])) - (D(rs[2 * SY]) - D(rs[-2 * SY]))) +
                c1[2] * (8.0 * (D(qs[4]) - D(qs[2])) - (D(qs[5]) - D(qs[1])));
          Kp += c1[0] * (8.0 * (D(rp[1]) - D(rp[-1])) - (D(rp[2]) - D(rp[-2]))) +
                c1[1] * (8.0 * (D(rp[SY]) - D(rp[-SY])) - (D(rp[2 * SY]) - D(rp[-2 * SY]))) +
                c1[2] * (8.0 * (D(qp[4]) - D(qp[2])) - (D(qp[5]) - D(qp[1])));
        }
      }
      // ---- RK4 stage combination (FP64)
      const long long cz = g.at(i, j, z);
      const double fa_s = fx ? T.fa[0] : A.alpha, fa_p = fx ? T.fa[1] : A.alpha;
      const double fb_s = fx ? T.fb[0] : A.beta, fb_p = fx ? T.fb[1] : A.beta;
      double os, op;
      if (A.stage == 3) {
        os = fma(fa_s, Ks, ub_s);
        op = fma(fa_p, Kp, ub_p);
      } else {
        const double as = A.stage == 0 ? ua_s : ub_s;
        const double ap = A.stage == 0 ? ua_p : ub_p;
        os = fma(fa_s, Ks, ua_s);
        op = fma(fa_p, Kp, ua_p);
        if (live) {
          Pt.ACC[cz] = fma(fb_s, Ks, as);
          Pt.ACC[cz + g.vol] = fma(fb_p, Kp, ap);
        }
      }
      if (live) {
        Pt.OUT[cz] = os;
        Pt.OUT[cz + g.vol] = op;
        emax_s = max(emax_s, biased_exponent(os));
        emax_p = max(emax_p, biased_exponent(op));
      }
    }
    // plane z+3 into the converted ring (read from iteration z+3 on)
    {
      long long* cv = conv_of(z + NG);
      cv[own] = qs[6];
      cv[CONV_PLANE + own] = qp[6];
      if (h_ok) {
        cv[hoff] = cvt(rs_h, Es);
        cv[CONV_PLANE + hoff] = cvt(rp_h, Ep);
      }
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

template <int TX, int TY, bool FIXED, bool ROT>
__global__ void __launch_bounds__(TX* TY, RHS_MIN_BLOCKS) k_rhs(const __grid_constant__ RhsArgs A) {
  rhs_body<TX, TY, FIXED, ROT>(A, blockIdx.x);
}

// Batched launch over independent instances: instance i owns the blocks
// [blk0[i], blk0[i + 1]) and its arguments As[i] (in global memory).
__device__ __forceinline__ int batch_instance(const int* __restrict__ blk0, int ninst) {
  int lo = 0, hi = ninst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((int)blockIdx.x >= blk0[mid]) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int TX, int TY, bool FIXED, bool ROT>
__global__ void __launch_bounds__(TX* TY, RHS_MIN_BLOCKS) k_rhs_batch(const RhsArgs* __restrict__ As,
                                                                      const int* __restrict__ blk0, int ninst) {
  const int i = batch_instance(blk0, ninst);
  rhs_body<TX, TY, FIXED, ROT>(As[i], blockIdx.x - blk0[i]);
}

// Host: TMA maps of one field buffer (4-D: x, y, plane, field).
bool encode_rhs_map(CUtensorMap* map, const void* base, const Geom& g, bool tile, bool f32) {
  // looked up once (thread-safe initialisation of a function-local static)
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  if (!encode) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)g.px, (cuuint64_t)g.py, (cuuint64_t)(g.n[2] + 2 * NG), 2};
  const cuuint64_t es = f32 ? 4 : 8;
  const cuuint64_t strides[3] = {(cuuint64_t)g.px * es, (cuuint64_t)g.plane * es, (cuuint64_t)g.vol * es};
  const cuuint32_t box[4] = {(cuuint32_t)(tile ? BOX_X : RHS_TX), (cuuint32_t)(tile ? BOX_Y : RHS_TY), 1, 2};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = encode(map, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4,
                            const_cast<void*>(base), dims, strides, box,
                            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <bool FIXED, bool ROT>
static void launch_rhs_batch_t(const RhsArgs* d_args, const int* d_blk0, int ninst, int blocks, cudaStream_t s) {
  cudaFuncSetAttribute(k_rhs_batch<RHS_TX, RHS_TY, FIXED, ROT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)RHS_SMEM);
  k_rhs_batch<RHS_TX, RHS_TY, FIXED, ROT><<<blocks, RHS_TX * RHS_TY, RHS_SMEM, s>>>(d_args, d_blk0, ninst);
}

void launch_rhs_batch(const RhsArgs* d_args, const int* d_blk0, int ninst, int blocks, bool fixed, bool rot,
                      void* stream) {
  const cudaStream_t s = (cudaStream_t)stream;
  if (fixed)
    rot ? launch_rhs_batch_t<true, true>(d_args, d_blk0, ninst, blocks, s)
        : launch_rhs_batch_t<true, false>(d_args, d_blk0, ninst, blocks, s);
  else
    rot ? launch_rhs_batch_t<false, true>(d_args, d_blk0, ninst, blocks, s)
        : launch_rhs_batch_t<false, false>(d_args, d_blk0, ninst, blocks, s);
}

template <bool FIXED, bool ROT>
static void launch_rhs_t(const RhsArgs& a, int blocks, cudaStream_t s) {
  cudaFuncSetAttribute(k_rhs<RHS_TX, RHS_TY, FIXED, ROT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)RHS_SMEM);
  k_rhs<RHS_TX, RHS_TY, FIXED, ROT><<<blocks, RHS_TX * RHS_TY, RHS_SMEM, s>>>(a);
}

void launch_rhs(const RhsArgs& a, int blocks, bool fixed, bool rot, void* stream) {
  const cudaStream_t s = (cudaStream_t)stream;
  if (fixed)
    rot ? launch_rhs_t<true, true>(a, blocks, s) : launch_rhs_t<true, false>(a, blocks, s);
  else
    rot ? launch_rhs_t<false, true>(a, blocks, s) : launch_rhs_t<false, false>(a, blocks, s);
}

}  // namespace mpw
