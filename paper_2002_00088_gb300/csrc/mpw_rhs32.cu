// mpw_rhs32.cu -- fused RHS + RK4 stage kernel in binary32 storage and
// arithmetic (the FP32 precision of a context created with precision = 32).
//
// Same equations and traversal as k_rhs (Sec. 2.2-2.3, Table 1): a CTA owns a
// 32 x 8 column tile and marches a chunk of planes; the raw input tile of each
// plane (with its halo) and the stage operands arrive by TMA several planes
// ahead; the z neighbours live in a register queue and the x/y neighbours in a
// ring of planes in shared memory.
//
// Rounding.  Every stencil is formed from differences to the centre value,
//   D2 = (16 (d1 + d-1) - (d2 + d-2)) / (12 h^2),
//   KO = (eps/64) ((d3 + d-3) - 6 (d2 + d-2) + 15 (d1 + d-1)) / h,
//   D1 = (8 (d1 - d-1) - (d2 - d-2)) / (12 h),      d_m = u_m - u_0,
// which is the same polynomial as the centred formulas (the weights of each sum
// to zero).  Neighbouring values of a smooth field agree to within a factor of
// two, so the differences are exact in binary32 and the rounding error of a
// stencil scales with the local variation of u, not with |u| / h^2.
//
// Packing.  psi and Pi go through the same stencil sums, so the two fields of a
// point travel as one pair: the ring of planes holds (psi, Pi) pairs, a
// neighbour is one 64-bit shared-memory load, and the differences, sums and
// stage updates are the packed binary32 pair instructions of sm_100 and later
// (add/sub/fma .rn.f32x2), each lane rounded exactly as the scalar operation.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mpw_internal.cuh"
#include "mpw_tma.cuh"

namespace mpw {

namespace {

#ifndef MPW_R32_DEPTH
#define MPW_R32_DEPTH 4
#endif
#ifndef MPW_R32_MINB
#define MPW_R32_MINB 4
#endif
constexpr int R32_DEPTH = MPW_R32_DEPTH;           // planes in flight per CTA
constexpr int R32_MINB = MPW_R32_MINB;             // CTAs per SM the register budget is sized for
constexpr int BX = RHS_TX + 8, BY = RHS_TY + 6;    // TMA tile box (x start rounded down 16 bytes)
constexpr int TILE_F = BX * BY * 2;
constexpr int PT_F = RHS_TX * RHS_TY * 2;
constexpr int SLOT_F = TILE_F + 2 * PT_F;          // tile | u | ACC
constexpr int RING_PLANE = (RHS_TY + 6) * (RHS_TX + 6);
constexpr int RING_SLOTS = 4;
constexpr size_t RHS32_SMEM =
    1024 + sizeof(float) * R32_DEPTH * SLOT_F + 8 * RING_SLOTS * RING_PLANE + 8 * R32_DEPTH;

// Loads of iteration zz (tile of input plane zz+3, u and ACC of plane zz).
__device__ __forceinline__ void issue_slot32(const RhsPatch& Pt, int stage, float* slot, unsigned bar, int i0, int j0,
                                             int zz) {
  const unsigned bytes = sizeof(float) * (TILE_F + (stage < 3 ? PT_F : 0) + (stage > 0 ? PT_F : 0));
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  bar_expect_tx(bar, bytes);
  tma_load_4d(smem_u32(slot), &Pt.ymap, i0 + Pt.g.xoff - 4, j0, zz + 3 + NG, 0, bar);
  if (stage < 3) tma_load_4d(smem_u32(slot + TILE_F), &Pt.umap, i0 + Pt.g.xoff, j0 + NG, zz + NG, 0, bar);
  if (stage > 0) tma_load_4d(smem_u32(slot + TILE_F + PT_F), &Pt.amap, i0 + Pt.g.xoff, j0 + NG, zz + NG, 0, bar);
}

// A (psi, Pi) pair of binary32 values in one 64-bit register: psi in the low
// half.
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float lo(f2 v) { return __uint_as_float((unsigned)(v & 0xFFFFFFFFull)); }
__device__ __forceinline__ float hi(f2 v) { return __uint_as_float((unsigned)(v >> 32)); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// Sums of the differences to the centre along one axis, both fields:
// s1 = d1 + d-1, s2 = d2 + d-2, s3 = d3 + d-3.
struct AxisSums {
  f2 s1, s2, s3;
};

__device__ __forceinline__ AxisSums axis_sums(f2 m3, f2 m2, f2 m1, f2 u0, f2 p1, f2 p2, f2 p3) {
  AxisSums r;
  r.s1 = add2(sub2(m1, u0), sub2(p1, u0));
  r.s2 = add2(sub2(m2, u0), sub2(p2, u0));
  r.s3 = add2(sub2(m3, u0), sub2(p3, u0));
  return r;
}

// First-derivative combination 8 (u1 - u-1) - (u2 - u-2), both fields (u0
// cancels, so no difference form is needed).
__device__ __forceinline__ f2 d1_pair(f2 m2, f2 m1, f2 p1, f2 p2) {
  return fma2(pk(8.0f, 8.0f), sub2(p1, m1), sub2(m2, p2));
}

// KO sixth-difference sum s3 - 6 s2 + 15 s1, both fields.
__device__ __forceinline__ f2 ko_pair(const AxisSums& a) {
  return fma2(pk(15.0f, 15.0f), a.s1, fma2(pk(-6.0f, -6.0f), a.s2, a.s3));
}

}  // namespace

template <bool ROT>
__device__ __forceinline__ void rhs32_body(const RhsArgs& A, const int b) {
  constexpr int TX = RHS_TX, TY = RHS_TY, SY = TX + 6;
  extern __shared__ unsigned char smem32[];
  __shared__ int s_abort;
  const unsigned long long base = (reinterpret_cast<unsigned long long>(smem32) + 1023ull) & ~1023ull;
  float* slots = reinterpret_cast<float*>(base);
  f2* ring = reinterpret_cast<f2*>(slots + R32_DEPTH * SLOT_F);  // [RING_SLOTS][RING_PLANE] (psi, Pi) pairs
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(ring + RING_SLOTS * RING_PLANE);
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
    s_abort = 0;
    for (int s = 0; s < R32_DEPTH; ++s) bar_init(smem_u32(&bars[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int s = 0; s < R32_DEPTH && z0 + s < z1; ++s)
      issue_slot32(Pt, A.stage, slots + s * SLOT_F, smem_u32(&bars[s]), i0, j0, z0 + s);
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
  const int own_raw = (lj + 3) * BX + li + 4;
  const int halo_raw = (hj - j0 + 3) * BX + (hi_ - i0 + 4);
  const float* Ys = reinterpret_cast<const float*>(Pt.Y);
  const float* Yp = Ys + g.vol;
  float* OUT = reinterpret_cast<float*>(Pt.OUT);
  float* ACC = reinterpret_cast<float*>(Pt.ACC);
  // coefficients, rounded once to binary32
  float c1[3], c2[3], ck[3], c1z[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    // a rotating frame's c1 is affine in the indices: this thread's column
    // value, and its step per plane
    c1[a] = (float)((ROT && Pt.rot) ? Pt.c1[a] + Pt.c1g[a][0] * i + Pt.c1g[a][1] * j : Pt.c1[a]);
    c1z[a] = (ROT && Pt.rot) ? (float)Pt.c1g[a][2] : 0.0f;
    c2[a] = (float)Pt.c2[a];
    ck[a] = (float)Pt.cko[a];
  }
  const float alpha = (float)A.alpha, beta = (float)A.beta;
  auto ring_of = [&](int zz) -> f2* { return ring + ((zz - z0) & (RING_SLOTS - 1)) * RING_PLANE; };
  // prologue: planes z0-3 .. z0+2 by plain loads (queue), z0 .. z0+2 also into the ring
  f2 q[7];
#pragma unroll
  for (int o = 0; o < 6; ++o) {
    const int zz = z0 - NG + o;
    q[o] = 0ull;
    if (in_box) {
      const long long c = g.at(i, j, zz);
      q[o] = pk(Ys[c], Yp[c]);
    }
    if (o >= NG && zz < z1) {
      f2* rv = ring_of(zz);
      rv[own] = q[o];
      if (h_ok) {
        const long long c = g.at(hi_, hj, zz);
        rv[hoff] = pk(Ys[c], Yp[c]);
      }
    }
  }
  const f2 alpha2 = pk(alpha, alpha), beta2 = pk(beta, beta);
  for (int z = z0; z < z1; ++z) {
    const int it = z - z0;
    const int s = it % R32_DEPTH;
    const float* sl = slots + s * SLOT_F;
    const unsigned bar = smem_u32(&bars[s]);
    int fl = FLAG_LIVE;
    if (in_xy && check_flags) fl = A.flags[((long long)z * g.n[1] + j) * g.n[0] + i] & 3;
    if (!bar_wait(bar, (unsigned)(it / R32_DEPTH) & 1u, A.wait_limit)) s_abort = 1;
    const float rs_own = sl[own_raw], rp_own = sl[BX * BY + own_raw];
    float rs_h = 0.0f, rp_h = 0.0f;
    if (h_ok) {
      rs_h = sl[halo_raw];
      rp_h = sl[BX * BY + halo_raw];
    }
    const int pt = lj * TX + li;
    f2 ua = 0ull, ub = 0ull;
    if (A.stage < 3) ua = pk(sl[TILE_F + pt], sl[TILE_F + TX * TY + pt]);
    if (A.stage > 0) ub = pk(sl[TILE_F + PT_F + pt], sl[TILE_F + PT_F + TX * TY + pt]);
    __syncthreads();
    if (s_abort) {
      if (threadIdx.x == 0) {
        atomicOr(A.err, ERR_TIMEOUT);
        for (int k = it; k < it + R32_DEPTH && z0 + k < z1; ++k)
          bar_wait(smem_u32(&bars[k % R32_DEPTH]), (unsigned)(k / R32_DEPTH) & 1u);
      }
      return;
    }
    if (threadIdx.x == 0 && z + R32_DEPTH < z1)
      issue_slot32(Pt, A.stage, slots + s * SLOT_F, bar, i0, j0, z + R32_DEPTH);
    q[6] = pk(rs_own, rp_own);
    const bool live = in_xy && (fl == FLAG_LIVE || fl == FLAG_REVIVED);
    {
      const f2* r = ring_of(z) + own;
      const f2 u0 = q[3];
      const AxisSums sx = axis_sums(r[-3], r[-2], r[-1], u0, r[1], r[2], r[3]);
      const AxisSums sy = axis_sums(r[-3 * SY], r[-2 * SY], r[-SY], u0, r[SY], r[2 * SY], r[3 * SY]);
      const AxisSums sz = axis_sums(q[0], q[1], q[2], u0, q[4], q[5], q[6]);
      // KO of both fields (KO_psi, KO_Pi) and D2 of psi
      f2 ko;
      float d2;
      if (Pt.iso) {
        AxisSums S;
        S.s1 = add2(add2(sx.s1, sy.s1), sz.s1);
        S.s2 = add2(add2(sx.s2, sy.s2), sz.s2);
        S.s3 = add2(add2(sx.s3, sy.s3), sz.s3);
        ko = fma2(pk(ck[0], ck[0]), ko_pair(S), 0ull);
        d2 = c2[0] * fmaf(16.0f, lo(S.s1), -lo(S.s2));
      } else {
        ko = fma2(pk(ck[2], ck[2]), ko_pair(sz),
                  fma2(pk(ck[1], ck[1]), ko_pair(sy), fma2(pk(ck[0], ck[0]), ko_pair(sx), 0ull)));
        d2 = c2[0] * fmaf(16.0f, lo(sx.s1), -lo(sx.s2)) + c2[1] * fmaf(16.0f, lo(sy.s1), -lo(sy.s2)) +
             c2[2] * fmaf(16.0f, lo(sz.s1), -lo(sz.s2));
      }
      // K = (Pi + KO_psi, D2 psi + KO_Pi) (+ w . D1 of both fields on a moving patch)
      f2 K = add2(ko, pk(hi(u0), d2));
      if (Pt.moving) {
        const f2 dx = d1_pair(r[-2], r[-1], r[1], r[2]);
        const f2 dy = d1_pair(r[-2 * SY], r[-SY], r[SY], r[2 * SY]);
        const f2 dz = d1_pair(q[1], q[2], q[4], q[5]);
        float w[3] = {c1[0], c1[1], c1[2]};
        if (ROT)
#pragma unroll
          for (int a = 0; a < 3; ++a) w[a] = fmaf(c1z[a], (float)z, w[a]);
        K = fma2(pk(w[2], w[2]), dz, fma2(pk(w[1], w[1]), dy, fma2(pk(w[0], w[0]), dx, K)));
      }
      const long long cz = g.at(i, j, z);
      if (live) {
        if (A.stage == 3) {
          const f2 o = fma2(alpha2, K, ub);
          OUT[cz] = lo(o);
          OUT[cz + g.vol] = hi(o);
        } else {
          const f2 o = fma2(alpha2, K, ua);
          const f2 acc = fma2(beta2, K, A.stage == 0 ? ua : ub);
          ACC[cz] = lo(acc);
          ACC[cz + g.vol] = hi(acc);
          OUT[cz] = lo(o);
          OUT[cz + g.vol] = hi(o);
        }
      }
    }
    // plane z+3 into the ring (read from iteration z+3 on)
    {
      f2* rv = ring_of(z + NG);
      rv[own] = q[6];
      if (h_ok) rv[hoff] = pk(rs_h, rp_h);
    }
#pragma unroll
    for (int o = 0; o < 6; ++o) q[o] = q[o + 1];
  }
}

// ---------------------------------------------------------------------------
// Two-plane body for translating frames on isotropic patches (the common
// case; rotating frames and anisotropic patches keep rhs32_body).  The same
// arithmetic per point as rhs32_body, in the same order, so the results are
// bit for bit those of rhs32_body; what changes is the traversal:
// iteration k computes the output planes zb = z0 + 2k and zb + 1 from an
// 8-deep register queue (planes zb - 3 .. zb + 4) and a ring of R32_CONV
// planes, and its slot holds, in two halves laid out like one R32_DEPTH slot
// each, the raw tiles of input planes zb + 3, zb + 4 and the stage operands
// of planes zb, zb + 1.  After the iteration's barrier, planes zb + 3 and
// zb + 4 go into the ring slots of zb - 2 and zb - 1 (plane p in slot
// (p - z0) mod 5), which iteration k - 1 read last.  Compiled once per
// substage and per moving / static patch; pointers advance per plane.
constexpr int R32_PAIR_DEPTH = 2;
constexpr int R32_PAIR_SLOT = 2 * SLOT_F;
constexpr int R32_CONV = 5;
constexpr size_t RHS32_PAIR_SMEM =
    128 + sizeof(float) * R32_PAIR_DEPTH * R32_PAIR_SLOT + 8 * R32_CONV * RING_PLANE + 8 * R32_PAIR_DEPTH;

__device__ __forceinline__ void issue_pair32(const RhsPatch& Pt, int stage, float* slot, unsigned bar, int i0, int j0,
                                             int zb, int nq) {
  const unsigned per = sizeof(float) * (TILE_F + (stage < 3 ? PT_F : 0) + (stage > 0 ? PT_F : 0));
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  bar_expect_tx(bar, per * nq);
  for (int q = 0; q < nq; ++q) {
    float* sq = slot + q * SLOT_F;
    const int zz = zb + q;
    tma_load_4d(smem_u32(sq), &Pt.ymap, i0 + Pt.g.xoff - 4, j0, zz + 3 + NG, 0, bar);
    if (stage < 3) tma_load_4d(smem_u32(sq + TILE_F), &Pt.umap, i0 + Pt.g.xoff, j0 + NG, zz + NG, 0, bar);
    if (stage > 0) tma_load_4d(smem_u32(sq + TILE_F + PT_F), &Pt.amap, i0 + Pt.g.xoff, j0 + NG, zz + NG, 0, bar);
  }
}

// K of one isotropic point (z column q[C-3 .. C+3], x/y neighbours around r),
// exactly as rhs32_body forms it.
template <bool MOVING, int C>
__device__ __forceinline__ f2 pair_point(const f2 (&q)[8], const f2* r, float ck, float c2, const float (&c1)[3]) {
  constexpr int SY = RHS_TX + 6;
  const f2 u0 = q[C];
  const AxisSums sx = axis_sums(r[-3], r[-2], r[-1], u0, r[1], r[2], r[3]);
  const AxisSums sy = axis_sums(r[-3 * SY], r[-2 * SY], r[-SY], u0, r[SY], r[2 * SY], r[3 * SY]);
  const AxisSums sz = axis_sums(q[C - 3], q[C - 2], q[C - 1], u0, q[C + 1], q[C + 2], q[C + 3]);
  AxisSums S;
  S.s1 = add2(add2(sx.s1, sy.s1), sz.s1);
  S.s2 = add2(add2(sx.s2, sy.s2), sz.s2);
  S.s3 = add2(add2(sx.s3, sy.s3), sz.s3);
  const f2 ko = fma2(pk(ck, ck), ko_pair(S), 0ull);
  const float d2 = c2 * fmaf(16.0f, lo(S.s1), -lo(S.s2));
  f2 K = add2(ko, pk(hi(u0), d2));
  if (MOVING) {
    const f2 dx = d1_pair(r[-2], r[-1], r[1], r[2]);
    const f2 dy = d1_pair(r[-2 * SY], r[-SY], r[SY], r[2 * SY]);
    const f2 dz = d1_pair(q[C - 2], q[C - 1], q[C + 1], q[C + 2]);
    K = fma2(pk(c1[2], c1[2]), dz, fma2(pk(c1[1], c1[1]), dy, fma2(pk(c1[0], c1[0]), dx, K)));
  }
  return K;
}

template <bool MOVING, int STAGE>
__device__ __forceinline__ void rhs32_pair_body(const RhsArgs& A, const RhsPatch& Pt, int lb, float* slots, f2* ring,
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
  if (threadIdx.x == 0)
    for (int k = 0; k < R32_PAIR_DEPTH && k < niter; ++k) {
      const int zb = z0 + 2 * k;
      issue_pair32(Pt, STAGE, slots + k * R32_PAIR_SLOT, smem_u32(&bars[k]), i0, j0, zb, zb + 1 < z1 ? 2 : 1);
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
  const int own_raw = (lj + 3) * BX + li + 4;
  const int halo_raw = (hj - j0 + 3) * BX + (hi_ - i0 + 4);
  const float* Ys = reinterpret_cast<const float*>(Pt.Y);
  const long long vol = g.vol, plane = g.plane;
  const float ck = (float)Pt.cko[0], c2 = (float)Pt.c2[0];
  float c1[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) c1[a] = (float)Pt.c1[a];
  const f2 alpha2 = pk((float)A.alpha, (float)A.alpha), beta2 = pk((float)A.beta, (float)A.beta);
  // prologue: planes z0-3 .. z0+2 by plain loads (queue), z0 .. z0+2 also
  // into ring slots 0 .. 2
  f2 q[8];
  {
    const long long c0 = g.at(min(i, g.n[0] + NG - 1), min(j, g.n[1] + NG - 1), z0 - NG);
    const long long ch = h_ok ? g.at(hi_, hj, z0) : 0;
#pragma unroll
    for (int o = 0; o < 6; ++o) {
      const int zz = z0 - NG + o;
      q[o] = 0ull;
      if (in_box) {
        const long long c = c0 + o * plane;
        q[o] = pk(Ys[c], Ys[c + vol]);
      }
      if (o >= NG && zz < z1) {
        f2* rv = ring + (o - NG) * RING_PLANE;
        rv[own] = q[o];
        if (h_ok) {
          const long long c = ch + (o - NG) * plane;
          rv[hoff] = pk(Ys[c], Ys[c + vol]);
        }
      }
    }
    q[6] = q[7] = 0ull;
  }
  const long long c_own = g.at(min(i, g.n[0] - 1), min(j, g.n[1] - 1), z0);
  float* outp = reinterpret_cast<float*>(Pt.OUT) + c_own;
  float* accp = reinterpret_cast<float*>(Pt.ACC) + c_own;
  const uint8_t* flagp = A.flags + ((long long)z0 * g.n[1] + min(j, g.n[1] - 1)) * g.n[0] + min(i, g.n[0] - 1);
  const long long fplane = (long long)g.n[0] * g.n[1];
  const int pt = lj * TX + li;
  int cs = 0;  // ring slot of plane zb
  for (int k = 0; k < niter; ++k) {
    const int zb = z0 + 2 * k;
    const bool two = zb + 1 < z1;
    const int s = k % R32_PAIR_DEPTH;
    const float* sl = slots + s * R32_PAIR_SLOT;
    const float* sl1 = sl + SLOT_F;
    const unsigned bar = smem_u32(&bars[s]);
    int fl0 = FLAG_LIVE, fl1 = FLAG_LIVE;
    if (in_xy && check_flags) {
      fl0 = flagp[0] & 3;
      if (two) fl1 = flagp[fplane] & 3;
    }
    if (!bar_wait(bar, (unsigned)(k / R32_PAIR_DEPTH) & 1u, A.wait_limit)) s_abort = 1;
    const f2 n0 = pk(sl[own_raw], sl[BX * BY + own_raw]);
    const f2 n1 = two ? pk(sl1[own_raw], sl1[BX * BY + own_raw]) : 0ull;
    f2 h0 = 0ull, h1 = 0ull;
    if (h_ok) {
      h0 = pk(sl[halo_raw], sl[BX * BY + halo_raw]);
      if (two) h1 = pk(sl1[halo_raw], sl1[BX * BY + halo_raw]);
    }
    f2 ua0 = 0ull, ub0 = 0ull, ua1 = 0ull, ub1 = 0ull;
    if (STAGE < 3) {
      ua0 = pk(sl[TILE_F + pt], sl[TILE_F + TX * TY + pt]);
      if (two) ua1 = pk(sl1[TILE_F + pt], sl1[TILE_F + TX * TY + pt]);
    }
    if (STAGE > 0) {
      ub0 = pk(sl[TILE_F + PT_F + pt], sl[TILE_F + PT_F + TX * TY + pt]);
      if (two) ub1 = pk(sl1[TILE_F + PT_F + pt], sl1[TILE_F + PT_F + TX * TY + pt]);
    }
    __syncthreads();
    if (s_abort) {
      if (threadIdx.x == 0) {
        atomicOr(A.err, ERR_TIMEOUT);
        for (int m = k; m < k + R32_PAIR_DEPTH && m < niter; ++m)
          bar_wait(smem_u32(&bars[m % R32_PAIR_DEPTH]), (unsigned)(m / R32_PAIR_DEPTH) & 1u);
      }
      return;
    }
    if (threadIdx.x == 0 && k + R32_PAIR_DEPTH < niter) {
      const int zn = zb + 2 * R32_PAIR_DEPTH;
      issue_pair32(Pt, STAGE, slots + s * R32_PAIR_SLOT, bar, i0, j0, zn, zn + 1 < z1 ? 2 : 1);
    }
    q[6] = n0;
    q[7] = n1;
    {
      const int c3 = cs + 3 >= R32_CONV ? cs + 3 - R32_CONV : cs + 3;
      const int c4 = cs + 4 >= R32_CONV ? cs + 4 - R32_CONV : cs + 4;
      f2* rv3 = ring + c3 * RING_PLANE;
      f2* rv4 = ring + c4 * RING_PLANE;
      rv3[own] = n0;
      rv4[own] = n1;
      if (h_ok) {
        rv3[hoff] = h0;
        rv4[hoff] = h1;
      }
    }
    const int cs1 = cs + 1 == R32_CONV ? 0 : cs + 1;
    {
      const f2 K = pair_point<MOVING, 3>(q, ring + cs * RING_PLANE + own, ck, c2, c1);
      if (in_xy && (fl0 == FLAG_LIVE || fl0 == FLAG_REVIVED)) {
        if (STAGE == 3) {
          const f2 o = fma2(alpha2, K, ub0);
          outp[0] = lo(o);
          outp[vol] = hi(o);
        } else {
          const f2 o = fma2(alpha2, K, ua0);
          const f2 acc = fma2(beta2, K, STAGE == 0 ? ua0 : ub0);
          accp[0] = lo(acc);
          accp[vol] = hi(acc);
          outp[0] = lo(o);
          outp[vol] = hi(o);
        }
      }
    }
    if (two) {
      const f2 K = pair_point<MOVING, 4>(q, ring + cs1 * RING_PLANE + own, ck, c2, c1);
      if (in_xy && (fl1 == FLAG_LIVE || fl1 == FLAG_REVIVED)) {
        if (STAGE == 3) {
          const f2 o = fma2(alpha2, K, ub1);
          outp[plane] = lo(o);
          outp[plane + vol] = hi(o);
        } else {
          const f2 o = fma2(alpha2, K, ua1);
          const f2 acc = fma2(beta2, K, STAGE == 0 ? ua1 : ub1);
          accp[plane] = lo(acc);
          accp[plane + vol] = hi(acc);
          outp[plane] = lo(o);
          outp[plane + vol] = hi(o);
        }
      }
    }
#pragma unroll
    for (int o = 0; o < 6; ++o) q[o] = q[o + 2];
    cs = cs + 2 >= R32_CONV ? cs + 2 - R32_CONV : cs + 2;
    outp += 2 * plane;
    accp += 2 * plane;
    flagp += 2 * fplane;
  }
}

template <bool ROT>
__device__ __noinline__ void rhs32_out_of_line(const RhsArgs& A, const int b) {
  rhs32_body<ROT>(A, b);
}

// Launch entry: the two-plane body for isotropic translating patches, the
// single-plane body (out of line) for rotating frames and anisotropic
// patches; the same body for the same patch in every launch.
template <bool ROT>
__device__ __forceinline__ void rhs32_entry(const RhsArgs& A, const int b) {
  extern __shared__ unsigned char smem32[];
  __shared__ int s_abort2;
  int p = 0;
  while (p + 1 < A.np && b >= A.p[p + 1].block0) ++p;
  const RhsPatch& Pt = A.p[p];
  if ((ROT && Pt.rot) || !Pt.iso) {
    rhs32_out_of_line<ROT>(A, b);
    return;
  }
  const unsigned long long base = (reinterpret_cast<unsigned long long>(smem32) + 127ull) & ~127ull;
  float* slots = reinterpret_cast<float*>(base);
  f2* ring = reinterpret_cast<f2*>(slots + R32_PAIR_DEPTH * R32_PAIR_SLOT);
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(ring + R32_CONV * RING_PLANE);
  if (threadIdx.x == 0) {
    s_abort2 = 0;
    for (int s = 0; s < R32_PAIR_DEPTH; ++s) bar_init(smem_u32(&bars[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  const int lb = b - Pt.block0;
  switch (A.stage * 2 + (Pt.moving ? 1 : 0)) {
    case 0: rhs32_pair_body<false, 0>(A, Pt, lb, slots, ring, bars, s_abort2); break;
    case 1: rhs32_pair_body<true, 0>(A, Pt, lb, slots, ring, bars, s_abort2); break;
    case 2: rhs32_pair_body<false, 1>(A, Pt, lb, slots, ring, bars, s_abort2); break;
    case 3: rhs32_pair_body<true, 1>(A, Pt, lb, slots, ring, bars, s_abort2); break;
    case 4: rhs32_pair_body<false, 2>(A, Pt, lb, slots, ring, bars, s_abort2); break;
    case 5: rhs32_pair_body<true, 2>(A, Pt, lb, slots, ring, bars, s_abort2); break;
    case 6: rhs32_pair_body<false, 3>(A, Pt, lb, slots, ring, bars, s_abort2); break;
    default: rhs32_pair_body<true, 3>(A, Pt, lb, slots, ring, bars, s_abort2); break;
  }
}

// Dynamic shared memory of the binary32 RHS kernels: the larger of the two layouts.
constexpr size_t RHS32_KERNEL_SMEM = RHS32_SMEM > RHS32_PAIR_SMEM ? RHS32_SMEM : RHS32_PAIR_SMEM;

template <bool ROT>
__global__ void __launch_bounds__(RHS_TX* RHS_TY, R32_MINB) k_rhs32(const __grid_constant__ RhsArgs A) {
  rhs32_entry<ROT>(A, blockIdx.x);
}

// Batched launch: instance i owns blocks [blk0[i], blk0[i + 1]), arguments As[i].
template <bool ROT>
__global__ void __launch_bounds__(RHS_TX* RHS_TY, R32_MINB) k_rhs32_batch(const RhsArgs* __restrict__ As,
                                                                          const int* __restrict__ blk0, int ninst) {
  if ((int)blockIdx.x >= blk0[ninst]) return;  // spare block of a padded grid
  int lo = 0, hi = ninst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((int)blockIdx.x >= blk0[mid]) lo = mid; else hi = mid - 1;
  }
  rhs32_entry<ROT>(As[lo], blockIdx.x - blk0[lo]);
}

template <bool ROT>
static void launch_rhs32_batch_t(const RhsArgs* d_args, const int* d_blk0, int ninst, int blocks, cudaStream_t s) {
  cudaFuncSetAttribute(k_rhs32_batch<ROT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RHS32_KERNEL_SMEM);
  k_rhs32_batch<ROT><<<blocks, RHS_TX * RHS_TY, RHS32_KERNEL_SMEM, s>>>(d_args, d_blk0, ninst);
}

void launch_rhs32_batch(const RhsArgs* d_args, const int* d_blk0, int ninst, int blocks, bool rot, void* stream) {
  rot ? launch_rhs32_batch_t<true>(d_args, d_blk0, ninst, blocks, (cudaStream_t)stream)
      : launch_rhs32_batch_t<false>(d_args, d_blk0, ninst, blocks, (cudaStream_t)stream);
}

template <bool ROT>
static void launch_rhs32_t(const RhsArgs& a, int blocks, cudaStream_t s) {
  cudaFuncSetAttribute(k_rhs32<ROT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RHS32_KERNEL_SMEM);
  k_rhs32<ROT><<<blocks, RHS_TX * RHS_TY, RHS32_KERNEL_SMEM, s>>>(a);
}

void launch_rhs32(const RhsArgs& a, int blocks, bool rot, void* stream) {
  rot ? launch_rhs32_t<true>(a, blocks, (cudaStream_t)stream) : launch_rhs32_t<false>(a, blocks, (cudaStream_t)stream);
}

}  // namespace mpw
