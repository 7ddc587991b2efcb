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
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mpw_internal.cuh"
#include "mpw_tma.cuh"

namespace mpw {

namespace {

constexpr int R32_DEPTH = 4;                       // planes in flight per CTA
constexpr int R32_MINB = 4;                        // CTAs per SM the register budget is sized for
constexpr int BX = RHS_TX + 8, BY = RHS_TY + 6;    // TMA tile box (x start rounded down 16 bytes)
constexpr int TILE_F = BX * BY * 2;
constexpr int PT_F = RHS_TX * RHS_TY * 2;
constexpr int SLOT_F = TILE_F + 2 * PT_F;          // tile | u | ACC
constexpr int RING_PLANE = (RHS_TY + 6) * (RHS_TX + 6);
constexpr int RING_SLOTS = 4;
constexpr size_t RHS32_SMEM =
    1024 + sizeof(float) * R32_DEPTH * SLOT_F + sizeof(float) * RING_SLOTS * 2 * RING_PLANE + 8 * R32_DEPTH;

// Loads of iteration zz (tile of input plane zz+3, u and ACC of plane zz).
__device__ __forceinline__ void issue_slot32(const RhsPatch& Pt, int stage, float* slot, unsigned bar, int i0, int j0,
                                             int zz) {
  const unsigned bytes = sizeof(float) * (TILE_F + (stage < 3 ? PT_F : 0) + (stage > 0 ? PT_F : 0));
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  bar_expect_tx(bar, bytes);
  tma_load_4d(smem_u32(slot), &Pt.ymap, i0, j0, zz + 3 + NG, 0, bar);
  if (stage < 3) tma_load_4d(smem_u32(slot + TILE_F), &Pt.umap, i0 + XOFF, j0 + NG, zz + NG, 0, bar);
  if (stage > 0) tma_load_4d(smem_u32(slot + TILE_F + PT_F), &Pt.amap, i0 + XOFF, j0 + NG, zz + NG, 0, bar);
}

// Sums of the differences to the centre along one axis: s1 = d1 + d-1,
// s2 = d2 + d-2, s3 = d3 + d-3 and the first-derivative combination.
struct AxisSums {
  float s1, s2, s3, d1;
};

__device__ __forceinline__ AxisSums axis_sums(float m3, float m2, float m1, float u0, float p1, float p2, float p3) {
  const float a1 = m1 - u0, b1 = p1 - u0, a2 = m2 - u0, b2 = p2 - u0;
  AxisSums r;
  r.s1 = a1 + b1;
  r.s2 = a2 + b2;
  r.s3 = (m3 - u0) + (p3 - u0);
  r.d1 = 8.0f * (b1 - a1) - (b2 - a2);
  return r;
}

}  // namespace

__global__ void __launch_bounds__(RHS_TX* RHS_TY, R32_MINB) k_rhs32(const __grid_constant__ RhsArgs A) {
  constexpr int TX = RHS_TX, TY = RHS_TY, SY = TX + 6;
  extern __shared__ unsigned char smem32[];
  __shared__ int s_abort;
  const unsigned long long base = (reinterpret_cast<unsigned long long>(smem32) + 1023ull) & ~1023ull;
  float* slots = reinterpret_cast<float*>(base);
  float* ring = slots + R32_DEPTH * SLOT_F;
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(ring + RING_SLOTS * 2 * RING_PLANE);
  const int b = blockIdx.x;
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
  float c1[3], c2[3], ck[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    c1[a] = (float)Pt.c1[a];
    c2[a] = (float)Pt.c2[a];
    ck[a] = (float)Pt.cko[a];
  }
  const float alpha = (float)A.alpha, beta = (float)A.beta;
  auto ring_of = [&](int zz) -> float* { return ring + ((zz - z0) & (RING_SLOTS - 1)) * 2 * RING_PLANE; };
  // prologue: planes z0-3 .. z0+2 by plain loads (queue), z0 .. z0+2 also into the ring
  float qs[7], qp[7];
#pragma unroll
  for (int o = 0; o < 6; ++o) {
    const int zz = z0 - NG + o;
    qs[o] = 0.0f;
    qp[o] = 0.0f;
    if (in_box) {
      const long long c = g.at(i, j, zz);
      qs[o] = Ys[c];
      qp[o] = Yp[c];
    }
    if (o >= NG && zz < z1) {
      float* rv = ring_of(zz);
      rv[own] = qs[o];
      rv[RING_PLANE + own] = qp[o];
      if (h_ok) {
        const long long c = g.at(hi_, hj, zz);
        rv[hoff] = Ys[c];
        rv[RING_PLANE + hoff] = Yp[c];
      }
    }
  }
  for (int z = z0; z < z1; ++z) {
    const int it = z - z0;
    const int s = it % R32_DEPTH;
    const float* sl = slots + s * SLOT_F;
    const unsigned bar = smem_u32(&bars[s]);
    int fl = FLAG_LIVE;
    if (in_xy && check_flags) fl = A.flags[((long long)z * g.n[1] + j) * g.n[0] + i] & 3;
    if (!bar_wait(bar, (unsigned)(it / R32_DEPTH) & 1u)) s_abort = 1;
    const float rs_own = sl[own_raw], rp_own = sl[BX * BY + own_raw];
    float rs_h = 0.0f, rp_h = 0.0f;
    if (h_ok) {
      rs_h = sl[halo_raw];
      rp_h = sl[BX * BY + halo_raw];
    }
    const int pt = lj * TX + li;
    float ua_s = 0.0f, ua_p = 0.0f, ub_s = 0.0f, ub_p = 0.0f;
    if (A.stage < 3) {
      ua_s = sl[TILE_F + pt];
      ua_p = sl[TILE_F + TX * TY + pt];
    }
    if (A.stage > 0) {
      ub_s = sl[TILE_F + PT_F + pt];
      ub_p = sl[TILE_F + PT_F + TX * TY + pt];
    }
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
    qs[6] = rs_own;
    qp[6] = rp_own;
    const bool live = in_xy && (fl == FLAG_LIVE || fl == FLAG_REVIVED);
    {
      const float* rs = ring_of(z) + own;
      const float* rp = rs + RING_PLANE;
      const float u0 = qs[3], v0 = qp[3];
      const AxisSums sx = axis_sums(rs[-3], rs[-2], rs[-1], u0, rs[1], rs[2], rs[3]);
      const AxisSums sy = axis_sums(rs[-3 * SY], rs[-2 * SY], rs[-SY], u0, rs[SY], rs[2 * SY], rs[3 * SY]);
      const AxisSums sz = axis_sums(qs[0], qs[1], qs[2], u0, qs[4], qs[5], qs[6]);
      const AxisSums px = axis_sums(rp[-3], rp[-2], rp[-1], v0, rp[1], rp[2], rp[3]);
      const AxisSums py = axis_sums(rp[-3 * SY], rp[-2 * SY], rp[-SY], v0, rp[SY], rp[2 * SY], rp[3 * SY]);
      const AxisSums pz = axis_sums(qp[0], qp[1], qp[2], v0, qp[4], qp[5], qp[6]);
      float Ks, Kp;
      if (Pt.iso) {
        const float S1 = sx.s1 + sy.s1 + sz.s1, S2 = sx.s2 + sy.s2 + sz.s2, S3 = sx.s3 + sy.s3 + sz.s3;
        const float P1 = px.s1 + py.s1 + pz.s1, P2 = px.s2 + py.s2 + pz.s2, P3 = px.s3 + py.s3 + pz.s3;
        Ks = v0 + ck[0] * (S3 - 6.0f * S2 + 15.0f * S1);
        Kp = c2[0] * (16.0f * S1 - S2) + ck[0] * (P3 - 6.0f * P2 + 15.0f * P1);
      } else {
        Ks = v0 + ck[0] * (sx.s3 - 6.0f * sx.s2 + 15.0f * sx.s1) + ck[1] * (sy.s3 - 6.0f * sy.s2 + 15.0f * sy.s1) +
             ck[2] * (sz.s3 - 6.0f * sz.s2 + 15.0f * sz.s1);
        Kp = c2[0] * (16.0f * sx.s1 - sx.s2) + c2[1] * (16.0f * sy.s1 - sy.s2) + c2[2] * (16.0f * sz.s1 - sz.s2) +
             ck[0] * (px.s3 - 6.0f * px.s2 + 15.0f * px.s1) + ck[1] * (py.s3 - 6.0f * py.s2 + 15.0f * py.s1) +
             ck[2] * (pz.s3 - 6.0f * pz.s2 + 15.0f * pz.s1);
      }
      if (Pt.moving) {
        Ks += c1[0] * sx.d1 + c1[1] * sy.d1 + c1[2] * sz.d1;
        Kp += c1[0] * px.d1 + c1[1] * py.d1 + c1[2] * pz.d1;
      }
      const long long cz = g.at(i, j, z);
      if (A.stage == 3) {
        if (live) {
          OUT[cz] = fmaf(alpha, Ks, ub_s);
          OUT[cz + g.vol] = fmaf(alpha, Kp, ub_p);
        }
      } else {
        const float as = A.stage == 0 ? ua_s : ub_s;
        const float ap = A.stage == 0 ? ua_p : ub_p;
        if (live) {
          ACC[cz] = fmaf(beta, Ks, as);
          ACC[cz + g.vol] = fmaf(beta, Kp, ap);
          OUT[cz] = fmaf(alpha, Ks, ua_s);
          OUT[cz + g.vol] = fmaf(alpha, Kp, ua_p);
        }
      }
    }
    // plane z+3 into the ring (read from iteration z+3 on)
    {
      float* rv = ring_of(z + NG);
      rv[own] = qs[6];
      rv[RING_PLANE + own] = qp[6];
      if (h_ok) {
        rv[hoff] = rs_h;
        rv[RING_PLANE + hoff] = rp_h;
      }
    }
#pragma unroll
    for (int o = 0; o < 6; ++o) {
      qs[o] = qs[o + 1];
      qp[o] = qp[o + 1];
    }
  }
}

void launch_rhs32(const RhsArgs& a, int blocks, void* stream) {
  cudaFuncSetAttribute(k_rhs32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RHS32_SMEM);
  k_rhs32<<<blocks, RHS_TX * RHS_TY, RHS32_SMEM, (cudaStream_t)stream>>>(a);
}

}  // namespace mpw
