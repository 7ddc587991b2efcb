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
    if (!bar_wait(bar, (unsigned)(it / RHS_DEPTH) & 1u, A.wait_limit)) s_abort = 1;
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

// ---------------------------------------------------------------------------
// Fixed-point body for translating frames on isotropic patches (constant w,
// equal spacing on every axis): the common case.  Same traversal, TMA
// pipeline and arithmetic model as rhs_body<FIXED>, with the integer work cut
// down:
//  - conversion of x to q = x 2^(1074-E) within one unit for the buffer's
//    largest biased exponent E (|q| < 2^52): the significand shifted right
//    once, the sign applied as a one's complement (to_fixed52);
//  - stencil sums formed around the centre, T_m = sum_axes (u_m + u_-m) - 6 u0,
//    so that D2 = 16 T1 - T2 and KO = T3 - 6 T2 + 15 T1 need no multiple of u0
//    (the weights of each stencil sum to zero);
//  - the real coefficients as 64 x 64 high products built from three 32-bit
//    partial products of a signed-digit split of the per-CTA multiplier
//    (hi_pos, hi_any), within three units of the output scale 2^S;
//  - per-CTA constants in registers, pointers advanced per plane.
// Rotating frames and anisotropic patches keep rhs_body<FIXED, ROT>; a CTA
// whose input is not finite or whose scales leave the binary64 range takes
// rhs_body<false>.

// Per-CTA constants of the fixed-point body.  A multiplier M (|M| < 2^61)
// is held as M = hi 2^32 + lo with lo in [-2^31, 2^31).
struct FxTerms {
  int ok;
  int E1s, E1p;          // conversion exponents of psi and Pi
  int v0[2];             // K_psi: Pi_0
  int kos[2];            // K_psi: KO(psi), all axes
  int d2[2];             // K_Pi : D2(psi), all axes
  int kop[2];            // K_Pi : KO(Pi), all axes
  int d1s[3][2];         // K_psi: D1(psi) per axis (moving patch)
  int d1p[3][2];         // K_Pi : D1(Pi) per axis
  double fa[2], fb[2];   // alpha 2^S, beta 2^S (psi, Pi)
};

// q = x 2^(1074-E1) to within one unit (the magnitude truncated, then the
// sign applied as a one's complement: -q - 1 for negative x), for a binary64
// x whose biased exponent is at most E1 (|q| < 2^52); values of larger
// exponent (non-live cells only) and values below 2^(E1-1086) give 0 or -1.
__device__ __forceinline__ long long to_fixed52(double x, int E1) {
  const int hi = __double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const unsigned mh = ((unsigned)hi & 0xFFFFFu) | 0x100000u;
  const unsigned sh = (unsigned)(E1 + 1 - (int)(((unsigned)hi >> 20) & 0x7FFu));
  const unsigned long long m = ((unsigned long long)mh << 32) | lo;
  unsigned long long t;
  asm("shr.b64 %0, %1, %2;" : "=l"(t) : "l"(m), "r"(sh));  // shift amounts >= 64 give 0
  return (long long)(t ^ (unsigned long long)(long long)(hi >> 31));
}

// M = round(coef 2^(E1 - 1074 - S + 64)) as a signed-digit pair.
__device__ __forceinline__ void fx_multiplier(double coef, int E1, int S, int (&m)[2]) {
  const long long M = coef == 0.0 ? 0ll : __double2ll_rn(scalbn(coef, E1 - 1074 - S + 64));
  const long long h = (M + 0x80000000ll) >> 32;
  m[0] = (int)h;
  m[1] = (int)(M - (h << 32));
}

// Smallest S with |coef| 2^(E1-1074-S+64) < 2^61 (so every multiplier is
// below 2^61); -100000 for coef = 0.
__device__ __forceinline__ int fx_scale(double coef, int E1) {
  return coef == 0.0 ? -100000 : ilogb(coef) + E1 - 1074 + 4;
}

// acc += a M / 2^64 (within 3 units) for |a| < 2^61 and a multiplier M >= 0:
// the partial products ah mh (exact, 64-bit), ah ml and al mh (their high
// words); al ml / 2^64 < 1 is dropped.
__device__ __forceinline__ long long hi_pos(long long a, const int (&m)[2], int& t) {
  const int ah = (int)(a >> 32);
  const unsigned al = (unsigned)a;
  t += __mulhi(ah, m[1]) + (int)__umulhi(al, (unsigned)m[0]);
  return (long long)ah * m[0];
}
// The same for a multiplier of either sign (al is unsigned: its high word
// against a negative mh needs mh added back when al >= 2^31).
__device__ __forceinline__ long long hi_any(long long a, const int (&m)[2], int& t) {
  const int ah = (int)(a >> 32);
  const int al = (int)(unsigned)a;
  t += __mulhi(ah, m[1]) + __mulhi(al, m[0]) + ((al >> 31) & m[0]);
  return (long long)ah * m[0];
}

__device__ void fx_setup(FxTerms& T, const RhsPatch& P, int Es_raw, int Ep_raw, double alpha, double beta) {
  T.ok = Es_raw < EXP_NONFINITE && Ep_raw < EXP_NONFINITE;
  if (!T.ok) return;
  const int Es = max(Es_raw, 64), Ep = max(Ep_raw, 64);
  T.E1s = Es;
  T.E1p = Ep;
  const double cko = P.cko[0], c2 = P.c2[0];
  int Ss = max(fx_scale(1.0, Ep), fx_scale(cko, Es));
  int Sp = max(fx_scale(c2, Es), fx_scale(cko, Ep));
  if (P.moving)
    for (int a = 0; a < 3; ++a) {
      Ss = max(Ss, fx_scale(P.c1[a], Es));
      Sp = max(Sp, fx_scale(P.c1[a], Ep));
    }
  if (Ss < -960 || Sp < -960 || Ss > 960 || Sp > 960) {
    T.ok = 0;
    return;
  }
  fx_multiplier(1.0, Ep, Ss, T.v0);
  fx_multiplier(cko, Es, Ss, T.kos);
  fx_multiplier(c2, Es, Sp, T.d2);
  fx_multiplier(cko, Ep, Sp, T.kop);
  for (int a = 0; a < 3; ++a) {
    fx_multiplier(P.moving ? P.c1[a] : 0.0, Es, Ss, T.d1s[a]);
    fx_multiplier(P.moving ? P.c1[a] : 0.0, Ep, Sp, T.d1p[a]);
  }
  T.fa[0] = scalbn(alpha, Ss);
  T.fb[0] = scalbn(beta, Ss);
  T.fa[1] = scalbn(alpha, Sp);
  T.fb[1] = scalbn(beta, Sp);
}

// Two-plane pipeline of the fixed-point body.  Iteration k of a CTA
// computes the output planes zb = z0 + 2k and zb + 1; its slot holds, in two
// halves laid out like one RHS_DEPTH slot each, the raw tiles (with halo) of
// input planes zb + 3 and zb + 4 and the stage operands u and ACC of planes
// zb and zb + 1.  FX_DEPTH slots are in flight (four planes ahead).  The
// z-neighbours live in an 8-deep register queue (planes zb - 3 .. zb + 4),
// the x/y neighbours in a ring of FX_CONV converted planes: iteration k
// reads planes zb and zb + 1 and, after its barrier, writes zb + 3 and zb + 4
// into the slots of zb - 2 and zb - 1 (plane p sits in slot (p - z0) mod 5),
// which iteration k - 1 read last; so one CTA barrier per iteration orders
// every write after the last read of its slot, and every read after the
// write (planes zb + 3, zb + 4 are read from iteration k + 1 on).
constexpr int FX_DEPTH = 2;
constexpr int FX_SLOT = 2 * SLOT_DOUBLES;
constexpr int FX_CONV = 5;
constexpr size_t FX_SMEM = 128 + sizeof(double) * FX_DEPTH * FX_SLOT +
                           sizeof(long long) * FX_CONV * 2 * CONV_PLANE + 8 * FX_DEPTH;

// Loads of iteration slot (output planes zb and, when nq = 2, zb + 1): one
// transaction count for all of them on the slot's barrier.
__device__ __forceinline__ void issue_pair(const RhsPatch& Pt, int stage, double* slot, unsigned bar, int i0, int j0,
                                           int zb, int nq) {
  const unsigned per = sizeof(double) * (TILE_DOUBLES + (stage < 3 ? PT_DOUBLES : 0) + (stage > 0 ? PT_DOUBLES : 0));
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  bar_expect_tx(bar, per * nq);
  for (int q = 0; q < nq; ++q) {
    double* sq = slot + q * SLOT_DOUBLES;
    const int zz = zb + q;
    tma_load_4d(smem_u32(sq), &Pt.ymap, i0 + Pt.g.xoff - 4, j0, zz + 3 + NG, 0, bar);
    if (stage < 3) tma_load_4d(smem_u32(sq + TILE_DOUBLES), &Pt.umap, i0 + Pt.g.xoff, j0 + NG, zz + NG, 0, bar);
    if (stage > 0)
      tma_load_4d(smem_u32(sq + TILE_DOUBLES + PT_DOUBLES), &Pt.amap, i0 + Pt.g.xoff, j0 + NG, zz + NG, 0, bar);
  }
}

// Multipliers of the stencil terms of one CTA, in registers (the D1
// multipliers of a moving patch are read from shared memory where used).
struct FxMul {
  int v0[2], kos[2], d2[2], kop[2];
};

// K_psi / 2^Ss and K_Pi / 2^Sp of the point whose z column is q[C-3 .. C+3]
// and whose converted x/y neighbours sit around rs (psi) and rp (Pi).
template <bool MOVING, int C>
__device__ __forceinline__ void fx_point(const long long (&qs)[8], const long long (&qp)[8], const long long* rs,
                                         const long long* rp, const FxMul& M, const FxTerms& T, long long& ks,
                                         long long& kp) {
  constexpr int SY = RHS_TX + 6;
  const long long u0 = qs[C], v0 = qp[C];
  int ts = 0, tp = 0;
  const long long u6 = 6 * u0, v6 = 6 * v0;
  const long long T1 = (rs[-1] + rs[1] + rs[-SY]) + (rs[SY] + qs[C - 1] + qs[C + 1]) - u6;
  const long long T2 = (rs[-2] + rs[2] + rs[-2 * SY]) + (rs[2 * SY] + qs[C - 2] + qs[C + 2]) - u6;
  const long long T3 = (rs[-3] + rs[3] + rs[-3 * SY]) + (rs[3 * SY] + qs[C - 3] + qs[C + 3]) - u6;
  const long long P1 = (rp[-1] + rp[1] + rp[-SY]) + (rp[SY] + qp[C - 1] + qp[C + 1]) - v6;
  const long long P2 = (rp[-2] + rp[2] + rp[-2 * SY]) + (rp[2 * SY] + qp[C - 2] + qp[C + 2]) - v6;
  const long long P3 = (rp[-3] + rp[3] + rp[-3 * SY]) + (rp[3 * SY] + qp[C - 3] + qp[C + 3]) - v6;
  const long long T16 = T1 * 16;
  const long long d2 = T16 - T2;
  const long long kos = T3 - 6 * T2 + (T16 - T1);
  const long long kop = P3 - 6 * P2 + 15 * P1;
  ks = hi_pos(v0, M.v0, ts) + hi_pos(kos, M.kos, ts);
  kp = hi_pos(d2, M.d2, tp) + hi_pos(kop, M.kop, tp);
  if (MOVING) {
    ks += (long long)ts;
    kp += (long long)tp;
    ts = 0;
    tp = 0;
    const long long dsx = 8 * (rs[1] - rs[-1]) - (rs[2] - rs[-2]);
    const long long dsy = 8 * (rs[SY] - rs[-SY]) - (rs[2 * SY] - rs[-2 * SY]);
    const long long dsz = 8 * (qs[C + 1] - qs[C - 1]) - (qs[C + 2] - qs[C - 2]);
    const long long dpx = 8 * (rp[1] - rp[-1]) - (rp[2] - rp[-2]);
    const long long dpy = 8 * (rp[SY] - rp[-SY]) - (rp[2 * SY] - rp[-2 * SY]);
    const long long dpz = 8 * (qp[C + 1] - qp[C - 1]) - (qp[C + 2] - qp[C - 2]);
    ks += hi_any(dsx, T.d1s[0], ts) + hi_any(dsy, T.d1s[1], ts);
    ks += (long long)ts;
    ts = 0;
    ks += hi_any(dsz, T.d1s[2], ts);
    kp += hi_any(dpx, T.d1p[0], tp) + hi_any(dpy, T.d1p[1], tp);
    kp += (long long)tp;
    tp = 0;
    kp += hi_any(dpz, T.d1p[2], tp);
  }
  ks += (long long)ts;
  kp += (long long)tp;
}

template <bool MOVING, int STAGE>
__device__ __forceinline__ void rhs_fx_body(const RhsArgs& A, const RhsPatch& Pt, const int p, int lb,
                                            const FxTerms& T, double* slots, long long* conv,
                                            unsigned long long* bars, int& s_abort) {
  constexpr int TX = RHS_TX, TY = RHS_TY, SY = TX + 6;
  const Geom& g = Pt.g;
  const int tx = lb % Pt.tiles_x;
  lb /= Pt.tiles_x;
  const int ty = lb % Pt.tiles_y;
  const int tz = lb / Pt.tiles_y;
  const int li = threadIdx.x % TX, lj = threadIdx.x / TX;
  const int i0 = tx * TX, j0 = ty * TY;
  const int i = i0 + li, j = j0 + lj;
  const int z0 = tz * Pt.zc, z1 = min(z0 + Pt.zc, g.n[2]);
  const int niter = (z1 - z0 + 1) / 2;
  constexpr int stage = STAGE;
  if (threadIdx.x == 0)
    for (int k = 0; k < FX_DEPTH && k < niter; ++k) {
      const int zb = z0 + 2 * k;
      issue_pair(Pt, stage, slots + k * FX_SLOT, smem_u32(&bars[k]), i0, j0, zb, zb + 1 < z1 ? 2 : 1);
    }
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
  const int own_raw = (lj + 3) * BOX_X + li + 4;
  const int halo_raw = (hj - j0 + 3) * BOX_X + (hi_ - i0 + 4);
  const int E1s = T.E1s, E1p = T.E1p;
  const double* Ys = Pt.Y;
  const long long vol = g.vol, plane = g.plane;
  constexpr int CP2 = 2 * CONV_PLANE;  // one converted plane, both fields
  // prologue: planes z0-3 .. z0+2 by plain loads (queue), z0 .. z0+2 also
  // into ring slots 0 .. 2 (plane zz sits in slot (zz - z0) mod FX_CONV)
  long long qs[8], qp[8];
  {
    const long long c0 = g.at(min(i, g.n[0] + NG - 1), min(j, g.n[1] + NG - 1), z0 - NG);
    const long long ch = h_ok ? g.at(hi_, hj, z0) : 0;
#pragma unroll
    for (int o = 0; o < 6; ++o) {
      const int zz = z0 - NG + o;
      qs[o] = 0;
      qp[o] = 0;
      if (in_box) {
        const long long c = c0 + o * plane;
        qs[o] = to_fixed52(Ys[c], E1s);
        qp[o] = to_fixed52(Ys[c + vol], E1p);
      }
      if (o >= NG && zz < z1) {
        long long* cv = conv + (o - NG) * CP2;
        cv[own] = qs[o];
        cv[CONV_PLANE + own] = qp[o];
        if (h_ok) {
          const long long c = ch + (o - NG) * plane;
          cv[hoff] = to_fixed52(Ys[c], E1s);
          cv[CONV_PLANE + hoff] = to_fixed52(Ys[c + vol], E1p);
        }
      }
    }
    qs[6] = qs[7] = qp[6] = qp[7] = 0;
  }
  FxMul M;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    M.v0[k] = T.v0[k];
    M.kos[k] = T.kos[k];
    M.d2[k] = T.d2[k];
    M.kop[k] = T.kop[k];
  }
  const double fa_s = T.fa[0], fa_p = T.fa[1], fb_s = T.fb[0], fb_p = T.fb[1];
  // output pointers advance two planes per iteration
  const long long c_own = g.at(min(i, g.n[0] - 1), min(j, g.n[1] - 1), z0);
  double* outp = Pt.OUT + c_own;
  double* accp = Pt.ACC + c_own;
  const uint8_t* flagp = A.flags + ((long long)z0 * g.n[1] + min(j, g.n[1] - 1)) * g.n[0] + min(i, g.n[0] - 1);
  const long long fplane = (long long)g.n[0] * g.n[1];
  const int pt = lj * TX + li;
  unsigned emax_s = 0, emax_p = 0;
  int cs = 0;  // ring slot of plane zb
  for (int k = 0; k < niter; ++k) {
    const int zb = z0 + 2 * k;
    const bool two = zb + 1 < z1;
    const int s = k % FX_DEPTH;
    const double* sl = slots + s * FX_SLOT;
    const unsigned bar = smem_u32(&bars[s]);
    int fl0 = FLAG_LIVE, fl1 = FLAG_LIVE;
    if (in_xy && check_flags) {
      fl0 = flagp[0] & 3;
      if (two) fl1 = flagp[fplane] & 3;
    }
    if (!bar_wait(bar, (unsigned)(k / FX_DEPTH) & 1u, A.wait_limit)) s_abort = 1;
    // raw values of input planes zb + 3 (half 0) and zb + 4 (half 1)
    const double* sl1 = sl + SLOT_DOUBLES;
    const double rs0 = sl[own_raw], rp0 = sl[BOX_X * BOX_Y + own_raw];
    double rs1 = 0.0, rp1 = 0.0, hs0 = 0.0, hp0 = 0.0, hs1 = 0.0, hp1 = 0.0;
    if (two) {
      rs1 = sl1[own_raw];
      rp1 = sl1[BOX_X * BOX_Y + own_raw];
    }
    if (h_ok) {
      hs0 = sl[halo_raw];
      hp0 = sl[BOX_X * BOX_Y + halo_raw];
      if (two) {
        hs1 = sl1[halo_raw];
        hp1 = sl1[BOX_X * BOX_Y + halo_raw];
      }
    }
    // stage operands of planes zb (half 0) and zb + 1 (half 1)
    double ua_s0 = 0.0, ua_p0 = 0.0, ub_s0 = 0.0, ub_p0 = 0.0, ua_s1 = 0.0, ua_p1 = 0.0, ub_s1 = 0.0, ub_p1 = 0.0;
    if (stage < 3) {
      ua_s0 = sl[TILE_DOUBLES + pt];
      ua_p0 = sl[TILE_DOUBLES + TX * TY + pt];
      if (two) {
        ua_s1 = sl1[TILE_DOUBLES + pt];
        ua_p1 = sl1[TILE_DOUBLES + TX * TY + pt];
      }
    }
    if (stage > 0) {
      ub_s0 = sl[TILE_DOUBLES + PT_DOUBLES + pt];
      ub_p0 = sl[TILE_DOUBLES + PT_DOUBLES + TX * TY + pt];
      if (two) {
        ub_s1 = sl1[TILE_DOUBLES + PT_DOUBLES + pt];
        ub_p1 = sl1[TILE_DOUBLES + PT_DOUBLES + TX * TY + pt];
      }
    }
    __syncthreads();
    if (s_abort) {
      // drain this CTA's copies still in flight (bounded), report, leave
      if (threadIdx.x == 0) {
        atomicOr(A.err, ERR_TIMEOUT);
        for (int m = k; m < k + FX_DEPTH && m < niter; ++m)
          bar_wait(smem_u32(&bars[m % FX_DEPTH]), (unsigned)(m / FX_DEPTH) & 1u);
      }
      return;
    }
    if (threadIdx.x == 0 && k + FX_DEPTH < niter) {
      const int zn = zb + 2 * FX_DEPTH;
      issue_pair(Pt, stage, slots + s * FX_SLOT, bar, i0, j0, zn, zn + 1 < z1 ? 2 : 1);
    }
    qs[6] = to_fixed52(rs0, E1s);
    qp[6] = to_fixed52(rp0, E1p);
    qs[7] = to_fixed52(rs1, E1s);
    qp[7] = to_fixed52(rp1, E1p);
    // planes zb + 3 and zb + 4 into the ring (read from iterations k + 1 and
    // k + 2); their slots last held planes zb - 2 and zb - 1, which the
    // barrier above retired
    {
      const int c3 = cs + 3 >= FX_CONV ? cs + 3 - FX_CONV : cs + 3;
      const int c4 = cs + 4 >= FX_CONV ? cs + 4 - FX_CONV : cs + 4;
      long long* cv3 = conv + c3 * CP2;
      long long* cv4 = conv + c4 * CP2;
      cv3[own] = qs[6];
      cv3[CONV_PLANE + own] = qp[6];
      cv4[own] = qs[7];
      cv4[CONV_PLANE + own] = qp[7];
      if (h_ok) {
        cv3[hoff] = to_fixed52(hs0, E1s);
        cv3[CONV_PLANE + hoff] = to_fixed52(hp0, E1p);
        cv4[hoff] = to_fixed52(hs1, E1s);
        cv4[CONV_PLANE + hoff] = to_fixed52(hp1, E1p);
      }
    }
    const int cs1 = cs + 1 == FX_CONV ? 0 : cs + 1;
    // ---- output plane zb
    {
      const long long* rs = conv + cs * CP2 + own;
      long long ks, kp;
      fx_point<MOVING, 3>(qs, qp, rs, rs + CONV_PLANE, M, T, ks, kp);
      const double Ks = (double)ks, Kp = (double)kp;
      const bool live = in_xy && (fl0 == FLAG_LIVE || fl0 == FLAG_REVIVED);
      double os, op;
      if (stage == 3) {
        os = fma(fa_s, Ks, ub_s0);
        op = fma(fa_p, Kp, ub_p0);
      } else {
        os = fma(fa_s, Ks, ua_s0);
        op = fma(fa_p, Kp, ua_p0);
        if (live) {
          accp[0] = fma(fb_s, Ks, stage == 0 ? ua_s0 : ub_s0);
          accp[vol] = fma(fb_p, Kp, stage == 0 ? ua_p0 : ub_p0);
        }
      }
      if (live) {
        outp[0] = os;
        outp[vol] = op;
        emax_s = max(emax_s, (unsigned)__double2hiint(os) & 0x7FFFFFFFu);
        emax_p = max(emax_p, (unsigned)__double2hiint(op) & 0x7FFFFFFFu);
      }
    }
    // ---- output plane zb + 1
    if (two) {
      const long long* rs = conv + cs1 * CP2 + own;
      long long ks, kp;
      fx_point<MOVING, 4>(qs, qp, rs, rs + CONV_PLANE, M, T, ks, kp);
      const double Ks = (double)ks, Kp = (double)kp;
      const bool live = in_xy && (fl1 == FLAG_LIVE || fl1 == FLAG_REVIVED);
      double os, op;
      if (stage == 3) {
        os = fma(fa_s, Ks, ub_s1);
        op = fma(fa_p, Kp, ub_p1);
      } else {
        os = fma(fa_s, Ks, ua_s1);
        op = fma(fa_p, Kp, ua_p1);
        if (live) {
          accp[plane] = fma(fb_s, Ks, stage == 0 ? ua_s1 : ub_s1);
          accp[plane + vol] = fma(fb_p, Kp, stage == 0 ? ua_p1 : ub_p1);
        }
      }
      if (live) {
        outp[plane] = os;
        outp[plane + vol] = op;
        emax_s = max(emax_s, (unsigned)__double2hiint(os) & 0x7FFFFFFFu);
        emax_p = max(emax_p, (unsigned)__double2hiint(op) & 0x7FFFFFFFu);
      }
    }
#pragma unroll
    for (int o = 0; o < 6; ++o) {
      qs[o] = qs[o + 2];
      qp[o] = qp[o + 2];
    }
    cs = cs + 2 >= FX_CONV ? cs + 2 - FX_CONV : cs + 2;
    outp += 2 * plane;
    accp += 2 * plane;
    flagp += 2 * fplane;
  }
  // exponent bookkeeping of the output buffer (consumed by the next substage)
  int es = (int)(emax_s >> 20), ep = (int)(emax_p >> 20);
  es = __reduce_max_sync(0xffffffffu, es);
  ep = __reduce_max_sync(0xffffffffu, ep);
  if ((threadIdx.x & 31) == 0) {
    if (es) atomicMax(&A.expo[slot(p, Pt.out_buf, 0)], es);
    if (ep) atomicMax(&A.expo[slot(p, Pt.out_buf, 1)], ep);
  }
}

// The bodies of rhs_body that the fixed-point entry hands CTAs to, kept out
// of line so that they do not share a register allocation with the
// isotropic fixed-point bodies: native FP64 (non-finite input, scales out of
// range), the per-axis fixed-point arithmetic of anisotropic patches and the
// rotating frames.
template <int TX, int TY, bool FIXED, bool ROT>
__device__ __noinline__ void rhs_out_of_line(const RhsArgs& A, const int b) {
  rhs_body<TX, TY, FIXED, ROT>(A, b);
}

// Fixed-point launch entry: per-CTA set-up, then the body for the patch: the
// isotropic fixed-point body of a translating frame (moving or not), or one
// of the out-of-line bodies.  Every launch (with or without rotating patches,
// single or batched) takes the same body for the same patch, so results do
// not depend on what else the launch holds.
template <int TX, int TY, bool ROT>
__device__ __forceinline__ void rhs_fx(const RhsArgs& A, const int b) {
  extern __shared__ unsigned char smem_dyn[];
  __shared__ FxTerms T;
  __shared__ int s_abort;
  const unsigned long long base = (reinterpret_cast<unsigned long long>(smem_dyn) + 127ull) & ~127ull;
  double* slots = reinterpret_cast<double*>(base);
  long long* conv = reinterpret_cast<long long*>(slots + FX_DEPTH * FX_SLOT);
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(conv + FX_CONV * 2 * CONV_PLANE);
  int p = 0;
  while (p + 1 < A.np && b >= A.p[p + 1].block0) ++p;
  const RhsPatch& Pt = A.p[p];
  if (ROT && Pt.rot) {
    rhs_out_of_line<TX, TY, true, ROT>(A, b);
    return;
  }
  if (!Pt.iso) {
    rhs_out_of_line<TX, TY, true, false>(A, b);
    return;
  }
  if (threadIdx.x == 0) {
    const int Es = max(A.expo[slot(p, Pt.in_buf, 0)], A.expo[slot(p, Pt.in_buf, 0) + EXP_GHOST]);
    const int Ep = max(A.expo[slot(p, Pt.in_buf, 1)], A.expo[slot(p, Pt.in_buf, 1) + EXP_GHOST]);
    fx_setup(T, Pt, Es, Ep, A.alpha, A.beta);
    s_abort = 0;
    if (T.ok) {
      for (int s = 0; s < FX_DEPTH; ++s) bar_init(smem_u32(&bars[s]), 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
  }
  __syncthreads();
  if (!T.ok) {
    rhs_out_of_line<TX, TY, false, false>(A, b);
    return;
  }
  const int lb = b - Pt.block0;
  switch (A.stage * 2 + (Pt.moving ? 1 : 0)) {
    case 0: rhs_fx_body<false, 0>(A, Pt, p, lb, T, slots, conv, bars, s_abort); break;
    case 1: rhs_fx_body<true, 0>(A, Pt, p, lb, T, slots, conv, bars, s_abort); break;
    case 2: rhs_fx_body<false, 1>(A, Pt, p, lb, T, slots, conv, bars, s_abort); break;
    case 3: rhs_fx_body<true, 1>(A, Pt, p, lb, T, slots, conv, bars, s_abort); break;
    case 4: rhs_fx_body<false, 2>(A, Pt, p, lb, T, slots, conv, bars, s_abort); break;
    case 5: rhs_fx_body<true, 2>(A, Pt, p, lb, T, slots, conv, bars, s_abort); break;
    case 6: rhs_fx_body<false, 3>(A, Pt, p, lb, T, slots, conv, bars, s_abort); break;
    default: rhs_fx_body<true, 3>(A, Pt, p, lb, T, slots, conv, bars, s_abort); break;
  }
}

template <int TX, int TY, bool FIXED, bool ROT>
__global__ void __launch_bounds__(TX* TY, RHS_MIN_BLOCKS) k_rhs(const __grid_constant__ RhsArgs A) {
  if (FIXED)
    rhs_fx<TX, TY, ROT>(A, blockIdx.x);
  else
    rhs_body<TX, TY, false, ROT>(A, blockIdx.x);
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
  if ((int)blockIdx.x >= blk0[ninst]) return;  // spare block of a padded grid
  const int i = batch_instance(blk0, ninst);
  if (FIXED)
    rhs_fx<TX, TY, ROT>(As[i], blockIdx.x - blk0[i]);
  else
    rhs_body<TX, TY, false, ROT>(As[i], blockIdx.x - blk0[i]);
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

// Dynamic shared memory of the RHS kernels: the larger of the layouts of
// rhs_body (RHS_SMEM) and of the two-plane fixed-point body (FX_SMEM).
constexpr size_t RHS_KERNEL_SMEM = RHS_SMEM > FX_SMEM ? RHS_SMEM : FX_SMEM;

template <bool FIXED, bool ROT>
static void launch_rhs_batch_t(const RhsArgs* d_args, const int* d_blk0, int ninst, int blocks, cudaStream_t s) {
  cudaFuncSetAttribute(k_rhs_batch<RHS_TX, RHS_TY, FIXED, ROT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)RHS_KERNEL_SMEM);
  k_rhs_batch<RHS_TX, RHS_TY, FIXED, ROT><<<blocks, RHS_TX * RHS_TY, RHS_KERNEL_SMEM, s>>>(d_args, d_blk0, ninst);
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
                       (int)RHS_KERNEL_SMEM);
  k_rhs<RHS_TX, RHS_TY, FIXED, ROT><<<blocks, RHS_TX * RHS_TY, RHS_KERNEL_SMEM, s>>>(a);
}

void launch_rhs(const RhsArgs& a, int blocks, bool fixed, bool rot, void* stream) {
  const cudaStream_t s = (cudaStream_t)stream;
  if (fixed)
    rot ? launch_rhs_t<true, true>(a, blocks, s) : launch_rhs_t<true, false>(a, blocks, s);
  else
    rot ? launch_rhs_t<false, true>(a, blocks, s) : launch_rhs_t<false, false>(a, blocks, s);
}

}  // namespace mpw
