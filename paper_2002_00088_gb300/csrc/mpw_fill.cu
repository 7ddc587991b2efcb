// mpw_fill.cu -- ghost-zone fill of one RK4 substage (Sec. 2.4), one launch:
//   * the global outer ghost shell: analytic closed form at the substage time
//     (Sec. 3) or periodic wrap -- one thread per point;
//   * Local-to-Global (Sec. 2.4.2): the global effective-ghost shell under each
//     local patch, interpolated from that patch;
//   * Global-to-Local (Sec. 2.4.1): every local ghost shell, interpolated from
//     the global patch.
// The three target sets are disjoint and each reads only data the others do
// not write (the buffer makes every interpolation donor a live cell).
//
// Interpolation is the tensor-product Lagrange sum of Eq. (Pijk).  Under
// rigid translation the three 1-D weight sets of a target depend only on its
// index along the respective axis, so the sum factors: a CTA takes a tile of
// targets that is a box, stages the donor block that the tile's windows cover
// in shared memory and contracts one axis after the other (separable passes,
// cheapest order first).  A tile whose donor block exceeds the shared-memory
// budget or the donor interior is evaluated point by point with the direct
// sum instead.
//
// Fixed-point passes (FillArgs::fixed).  GB300 issues FP64 FMAs at a small
// fraction of its integer rate, so by default the passes run on integers:
// the donor block is put on the scale of its own largest exponent E
// (q = round(x 2^(1075-E)), |q| < 2^53, then a = 64 q), the weights on
// 2^59 (every weight of these windows has |w| <= 1), and each product is
// formed from three 32 x 32 -> 64 partial products of the values split at
// bit 31 (the low x low product is dropped).  One pass maps values below
// 2^60 to values below Lambda 2^60 with Lambda = 1.39, the largest Lebesgue
// constant of the P = 5 and 6 windows, so the three passes stay inside int64;
// each pass adds an error below one unit of q, so the result is within a few
// units in the last place of the block's largest value.  A block holding a
// non-finite value takes the FP64 passes, which propagate it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "mpw_device.cuh"
#include "mpw_fixed.cuh"
#include "mpw_internal.cuh"

namespace mpw {

// Shared-memory budget of one CTA of the separable path, per field (both
// fields are contracted together): the block after the thin-axis pass and
// the block after the second pass.  The final values reuse the first.
constexpr int CAP_R1 = 4608;
constexpr int CAP_R2 = 1792;
constexpr int MAXT = 32;      // largest tile extent along a wide axis
constexpr int MAXT0 = NG;     // targets along the thin axis (slab walls are NG thick)
constexpr int MAXD = 16;      // largest donor extent along the thin axis
constexpr int FILL_THREADS = 256;
constexpr size_t FILL_SMEM = sizeof(double) * 2 * (CAP_R1 + CAP_R2) +
                             (sizeof(double) + sizeof(int2)) * (3 * MAXT * 6 + MAXT0 * MAXD) + sizeof(int) * 3 * MAXT;

namespace {

// Warp- then CTA-level maximum of two exponents, reported with one atomicMax
// per field by the first thread.
__device__ void report_block_max(int* slot2, int e0, int e1) {
  __shared__ int red[2];
  if (threadIdx.x == 0) red[0] = red[1] = 0;
  __syncthreads();
  e0 = __reduce_max_sync(0xffffffffu, e0);
  e1 = __reduce_max_sync(0xffffffffu, e1);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&red[0], e0);
    atomicMax(&red[1], e1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (red[0]) atomicMax(&slot2[0], red[0]);
    if (red[1]) atomicMax(&slot2[1], red[1]);
  }
}

// Position of target index i along axis a in the donor's index units.
// The buffer whose exponent slots scale a segment's donor values: the one
// being filled, or for the global patch an override (the hybrid step's
// prescribed stage states, laid out in other buffers).
__device__ __forceinline__ int donor_buf(const FillArgs& A, const InterpSeg& S) {
  return S.dpatch == 0 && A.gdonor_use ? A.gdonor_buf : A.y_buf;
}

__device__ __forceinline__ double donor_index(const InterpSeg& S, int a, int i) {
  return ((S.gt.lo[a] + (i + 0.5) * S.gt.h[a] + S.shift[a]) - S.gd.lo[a]) / S.gd.h[a] - 0.5;
}

// v = hi 2^31 + lo with 0 <= lo < 2^31 (|v| < 2^62).
__device__ __forceinline__ int2 split31(long long v) {
  return make_int2((int)(v & 0x7FFFFFFFll), (int)(v >> 31));
}

// Fixed-point multiply-add of a split value and a split weight on 2^59:
// accumulates the high x high, high x low and low x high partial products.
struct Acc3 {
  long long hh = 0, hl = 0, lh = 0;
  __device__ __forceinline__ void mac(int2 a, int2 b) {
    hh += (long long)a.y * b.y;
    hl += (long long)a.y * b.x;
    lh += (long long)a.x * b.y;
  }
  // sum of a w over the accumulated terms (the low x low products, each
  // below 2^62 / 2^59 = 8 units, are dropped)
  __device__ __forceinline__ long long value() const { return hh * 8 + (hl >> 28) + (lh >> 28); }
};

// One separable pass over both fields: contract axis AX of the blocks `in`
// (extents din, x fastest, field f at in + f * in_stride) against the 1-D
// weights of the tile's targets along AX.  ws holds the absolute window
// starts, off the block origin along AX, w the P weights per target.  FX
// is the arithmetic: M_FP64 (double entries), M_FIXED (int2 entries, split
// output; FINAL keeps the last output whole as long long) or M_FP32 (float
// entries and weights).
enum { M_FP64 = 0, M_FIXED = 1, M_FP32 = 2 };

template <int P, int AX, int MODE, bool FINAL>
__device__ __forceinline__ void contract_axis(const void* __restrict__ in, int in_stride, void* __restrict__ out,
                                              int out_stride, const int din[3], int T, const void* __restrict__ w,
                                              const int* __restrict__ ws, int off) {
  const int d0 = AX == 0 ? T : din[0], d1 = AX == 1 ? T : din[1], d2 = AX == 2 ? T : din[2];
  const int s1 = din[0], s2 = din[0] * din[1];
  const int st = AX == 0 ? 1 : (AX == 1 ? s1 : s2);
  const int n = d0 * d1 * d2;
  BlockWalk<FILL_THREADS> wk(threadIdx.x, d0, d1, d2);
  for (int e = threadIdx.x; e < 2 * n; e += FILL_THREADS, wk.next()) {
    const int f = wk.f;
    const int r = e - f * n;
    int o0 = wk.o0, o1 = wk.o1, o2 = wk.o2;
    const int t = AX == 0 ? o0 : (AX == 1 ? o1 : o2);
    const int c = ws[t] - off;
    if (AX == 0) o0 = c;
    if (AX == 1) o1 = c;
    if (AX == 2) o2 = c;
    const int src = f * in_stride + o0 + o1 * s1 + o2 * s2;
    if (MODE == M_FIXED) {
      const int2* a = static_cast<const int2*>(in) + src;
      const int2* wt = static_cast<const int2*>(w) + t * 6;
      Acc3 acc;
#pragma unroll
      for (int m = 0; m < P; ++m) acc.mac(a[m * st], wt[m]);
      if (FINAL)
        static_cast<long long*>(out)[f * out_stride + r] = acc.value();
      else
        static_cast<int2*>(out)[f * out_stride + r] = split31(acc.value());
    } else if (MODE == M_FP32) {
      const float* a = static_cast<const float*>(in) + src;
      const float* wt = static_cast<const float*>(w) + t * 6;
      float acc = 0.0f;
#pragma unroll
      for (int m = 0; m < P; ++m) acc = fmaf(wt[m], a[m * st], acc);
      static_cast<float*>(out)[f * out_stride + r] = acc;
    } else {
      const double* a = static_cast<const double*>(in) + src;
      const double* wt = static_cast<const double*>(w) + t * 6;
      double acc = 0.0;
#pragma unroll
      for (int m = 0; m < P; ++m) acc = fma(wt[m], a[m * st], acc);
      static_cast<double*>(out)[f * out_stride + r] = acc;
    }
  }
}

template <int P, int MODE, bool FINAL>
__device__ __forceinline__ void contract(const void* in, int in_stride, void* out, int out_stride, const int din[3],
                                         int ax, int T, const void* w, const int* ws, int off) {
  if (ax == 0)
    contract_axis<P, 0, MODE, FINAL>(in, in_stride, out, out_stride, din, T, w, ws, off);
  else if (ax == 1)
    contract_axis<P, 1, MODE, FINAL>(in, in_stride, out, out_stride, din, T, w, ws, off);
  else
    contract_axis<P, 2, MODE, FINAL>(in, in_stride, out, out_stride, din, T, w, ws, off);
}

// Thin-axis pass fused with the donor load: one thread per donor pencil
// along the thin axis a0 (both fields), holding its nk values in registers
// and contracting them against the band matrix of the tile's targets along
// a0 (row t: the P weights of target t at its window offset, zeros
// elsewhere).  Output: the block with extent T0 along a0 and the donor
// extents along the other axes, x fastest.
template <int P, int MODE, typename ST>
__device__ __forceinline__ void thin_pass(const InterpSeg& S, int a0, const int D0[3], const int Dn[3], int T0,
                                          const void* __restrict__ band, int Es, int Ep, void* __restrict__ out) {
  const int a1 = a0 == 0 ? 1 : 0, a2 = a0 == 2 ? 1 : 2;
  const int n1 = Dn[a1], n2 = Dn[a2], nk = Dn[a0];
  const long long st0 = a0 == 0 ? 1 : (a0 == 1 ? (long long)S.gd.px : S.gd.plane);
  // strides of the output block (extent T0 along a0)
  int ext[3] = {Dn[0], Dn[1], Dn[2]};
  ext[a0] = T0;
  const int ostr[3] = {1, ext[0], ext[0] * ext[1]};
  const int npen = n1 * n2;
  auto pencil = [&](int e, int& f, int& obase) -> const ST* {
    f = e >= npen;
    const int p = e - f * npen;
    const int c1 = p % n1, c2 = p / n1;
    int o[3];
    o[a0] = D0[a0];
    o[a1] = D0[a1] + c1;
    o[a2] = D0[a2] + c2;
    obase = c1 * ostr[a1] + c2 * ostr[a2] + f * CAP_R1;
    return reinterpret_cast<const ST*>(S.D) + f * S.gd.vol + S.gd.at(o[0], o[1], o[2]);
  };
  if (MODE == M_FIXED) {
    // software-pipelined: the next pencil's donors are in flight while this
    // one is converted and contracted
    ST raw[MAXD];
    int f, obase;
    if ((int)threadIdx.x < 2 * npen) {
      const ST* src = pencil(threadIdx.x, f, obase);
#pragma unroll
      for (int k = 0; k < MAXD; ++k) raw[k] = k < nk ? src[k * st0] : (ST)0;
    }
    const int2* bq = static_cast<const int2*>(band);
    for (int e = threadIdx.x; e < 2 * npen; e += FILL_THREADS) {
      pencil(e, f, obase);
      ST nxt[MAXD];
      const int en = e + FILL_THREADS;
      if (en < 2 * npen) {
        int fn, on;
        const ST* src = pencil(en, fn, on);
#pragma unroll
        for (int k = 0; k < MAXD; ++k) nxt[k] = k < nk ? src[k * st0] : (ST)0;
      }
      const int E = f ? Ep : Es;
      int2 v[MAXD];
#pragma unroll
      for (int k = 0; k < MAXD; ++k) v[k] = split31(k < nk ? to_fixed((double)raw[k], E) * 64 : 0);
#pragma unroll
      for (int t = 0; t < MAXT0; ++t) {
        if (t >= T0) break;
        Acc3 acc;
#pragma unroll
        for (int k = 0; k < MAXD; ++k)
          if (k < nk) acc.mac(v[k], bq[t * MAXD + k]);
        static_cast<int2*>(out)[obase + t * ostr[a0]] = split31(acc.value());
      }
#pragma unroll
      for (int k = 0; k < MAXD; ++k) raw[k] = nxt[k];
    }
    return;
  }
  for (int e = threadIdx.x; e < 2 * npen; e += FILL_THREADS) {
    const int f = e >= npen;
    const int p = e - f * npen;
    const int c1 = p % n1, c2 = p / n1;
    int o[3];
    o[a0] = D0[a0];
    o[a1] = D0[a1] + c1;
    o[a2] = D0[a2] + c2;
    const ST* src = reinterpret_cast<const ST*>(S.D) + f * S.gd.vol + S.gd.at(o[0], o[1], o[2]);
    const int obase = c1 * ostr[a1] + c2 * ostr[a2] + f * CAP_R1;
    if (MODE == M_FP32) {
      float v[MAXD];
#pragma unroll
      for (int k = 0; k < MAXD; ++k) v[k] = k < nk ? (float)src[k * st0] : 0.0f;
      const float* bf = static_cast<const float*>(band);
#pragma unroll
      for (int t = 0; t < MAXT0; ++t) {
        if (t >= T0) break;
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k < MAXD; ++k)
          if (k < nk) acc = fmaf(bf[t * MAXD + k], v[k], acc);
        static_cast<float*>(out)[obase + t * ostr[a0]] = acc;
      }
    } else if (MODE == M_FIXED) {
      const int E = f ? Ep : Es;
      int2 v[MAXD];
#pragma unroll
      for (int k = 0; k < MAXD; ++k) v[k] = split31(k < nk ? to_fixed((double)src[k * st0], E) * 64 : 0);
      const int2* bq = static_cast<const int2*>(band);
#pragma unroll
      for (int t = 0; t < MAXT0; ++t) {
        if (t >= T0) break;
        Acc3 acc;
#pragma unroll
        for (int k = 0; k < MAXD; ++k)
          if (k < nk) acc.mac(v[k], bq[t * MAXD + k]);
        static_cast<int2*>(out)[obase + t * ostr[a0]] = split31(acc.value());
      }
    } else {
      double v[MAXD];
#pragma unroll
      for (int k = 0; k < MAXD; ++k) v[k] = k < nk ? (double)src[k * st0] : 0.0;
      const double* bd = static_cast<const double*>(band);
#pragma unroll
      for (int t = 0; t < MAXT0; ++t) {
        if (t >= T0) break;
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < MAXD; ++k)
          if (k < nk) acc = fma(bd[t * MAXD + k], v[k], acc);
        static_cast<double*>(out)[obase + t * ostr[a0]] = acc;
      }
    }
  }
}

// Donor position of the target point with target numeric coordinates
// (x, y, z): a shift under translation, an affine map under rotation.
__device__ __forceinline__ void donor_position(const InterpSeg& S, double x, double y, double z, double& px,
                                               double& py, double& pz) {
  if (S.kind == SEG_SHELL) {
    px = x + S.shift[0], py = y + S.shift[1], pz = z + S.shift[2];
  } else {
    affine(S.M, S.shift, x, y, z, px, py, pz);
  }
}

// Position of target cell (i, j, k) in the donor's index units, per axis,
// from the segment's affine index map (rotated segments).
__device__ __forceinline__ void donor_indices(const InterpSeg& S, int i, int j, int k, double sidx[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
    sidx[a] = fma(S.sidx[a][0], (double)i, fma(S.sidx[a][1], (double)j, fma(S.sidx[a][2], (double)k, S.sidx[a][3])));
}

// (a b) / 2^56 and (a b) / 2^61, rounded toward minus infinity, from the
// 128-bit product (the quotients must fit in int64).
__device__ __forceinline__ long long mul56(long long a, long long b) {
  return (long long)(((unsigned long long)__mul64hi(a, b) << 8) | ((unsigned long long)(a * b) >> 56));
}
__device__ __forceinline__ long long mul61(long long a, long long b) {
  return (long long)(((unsigned long long)__mul64hi(a, b) << 3) | ((unsigned long long)(a * b) >> 61));
}

// 1-D Lagrange weights of Eq. (Pijk) on 2^59 (split) for the window that
// starts two nodes below floor(s), in int64 arithmetic (the FP64 pipe of
// GB300 issues at a small fraction of the integer rate): u = s - floor(s) on
// 2^56, the numerators prod_{q != m} (u - o_q) from prefix and suffix
// products, and the division by the integer D_m = prod_{q != m} (o_m - o_q)
// as a product with round(2^64 / D_m).  Every factor is at most 3 in
// magnitude and every product at most 36, so all values fit; the
// truncations leave each weight within about 2^-52 of its exact value.
template <int P>
__device__ __forceinline__ int lagrange_fixed(double s, int2 (&w)[P]) {
  constexpr long long K6[6] = {-153722867280912930ll, 768614336404564651ll, -1537228672809129301ll,
                               1537228672809129301ll, -768614336404564651ll, 153722867280912930ll};
  constexpr long long K5[5] = {768614336404564651ll, -3074457345618258603ll, 4611686018427387904ll,
                               -3074457345618258603ll, 768614336404564651ll};
  const double fl = floor(s);
  constexpr long long one = 1ll << 56;
  const long long U = __double2ll_rz((s - fl) * 0x1p56);
  long long d[P], pre[P + 1], suf[P + 1];
#pragma unroll
  for (int m = 0; m < P; ++m) d[m] = U - (long long)(m - 2) * one;
  pre[0] = one;
  suf[P] = one;
#pragma unroll
  for (int m = 0; m < P; ++m) pre[m + 1] = mul56(pre[m], d[m]);
#pragma unroll
  for (int m = P - 1; m >= 0; --m) suf[m] = mul56(suf[m + 1], d[m]);
#pragma unroll
  for (int m = 0; m < P; ++m) w[m] = split31(mul61(mul56(pre[m], suf[m + 1]), P == 6 ? K6[m] : K5[m]));
  return (int)fl - 2;
}

// Fixed-point tensor sum of one point under a rotated map (Eq. Pijk with
// the separable passes' arithmetic: x rows, then y, then z, each an Acc3
// contraction against weights on 2^59).  fetch(f, x, y, z) returns the
// donor at window-relative offsets as a split fixed-point value; out[f] is
// on the scale of the donor values.
// The field and plane loops stay rolled: the unrolled 6 x 6 x 6 sum of both
// fields is large enough to thrash the instruction cache next to the other
// fill paths.
template <int P, typename Fetch>
__device__ __forceinline__ void contract_point_fixed(const int2 (&wx)[P], const int2 (&wy)[P], const int2 (&wz)[P],
                                                     Fetch fetch, long long out[2]) {
#pragma unroll 1
  for (int f = 0; f < 2; ++f) {
    Acc3 az;
#pragma unroll 1
    for (int c = 0; c < P; ++c) {
      Acc3 ay;
#pragma unroll
      for (int b = 0; b < P; ++b) {
        Acc3 ax;
#pragma unroll
        for (int a = 0; a < P; ++a) ax.mac(fetch(f, a, b, c), wx[a]);
        ay.mac(split31(ax.value()), wy[b]);
      }
      az.mac(split31(ay.value()), wz[c]);
    }
    out[f] = az.value();
  }
}

// 1-D weights of the three axes on 2^59 (split), and the window starts.
template <int P>
__device__ __forceinline__ void fixed_weights(const double sidx[3], int2 (&wx)[P], int2 (&wy)[P], int2 (&wz)[P],
                                              int st[3]) {
  st[0] = lagrange_fixed<P>(sidx[0], wx);
  st[1] = lagrange_fixed<P>(sidx[1], wy);
  st[2] = lagrange_fixed<P>(sidx[2], wz);
}

// Direct tensor sums (Eq. Pijk) point by point for the targets of a tile;
// reports uninterpolable points.
template <int P, typename ST>
__device__ __noinline__ void direct_points(const FillArgs& A, const InterpSeg& S, const int org[3], const int T[3], int emax[2]) {
  ST* Tt = reinterpret_cast<ST*>(S.T);
  const int ntar = T[0] * T[1] * T[2];
  for (int e = threadIdx.x; e < ntar; e += FILL_THREADS) {
    const int x = e % T[0], y = (e / T[0]) % T[1], z = e / (T[0] * T[1]);
    const int i = org[0] + x, j = org[1] + y, k = org[2] + z;
    double v0, v1, px, py, pz;
    donor_position(S, S.gt.lo[0] + (i + 0.5) * S.gt.h[0], S.gt.lo[1] + (j + 0.5) * S.gt.h[1],
                   S.gt.lo[2] + (k + 0.5) * S.gt.h[2], px, py, pz);
    if (!interp_point<P>(reinterpret_cast<const ST*>(S.D), S.gd, px, py, pz, v0, v1)) {
      atomicOr(A.err, ERR_UNFILLED);
      continue;
    }
    const long long c = S.gt.at(i, j, k);
    Tt[c] = (ST)v0;
    Tt[c + S.gt.vol] = (ST)v1;
    emax[0] = max(emax[0], biased_exponent(v0));
    emax[1] = max(emax[1], biased_exponent(v1));
  }
}

// Local-to-Global of one global cell (i, j, k) under a rotating map:
// fixed point with the donors gathered and converted on the fly, or the
// direct FP64 sum (binary32 storage, native FP64, non-finite donors).
template <int P, typename ST>
__device__ __forceinline__ void l2g_point(const FillArgs& A, const InterpSeg& S, int i, int j, int k, int& e0,
                                          int& e1) {
  constexpr bool F32 = sizeof(ST) == 4;
  const int* dslot = A.expo + S.dpatch * EXP_SLOTS_PER_PATCH + donor_buf(A, S) * 2;
  const bool fx = !F32 && A.fixed && dslot[0] < EXP_NONFINITE && dslot[1] < EXP_NONFINITE;
  if (fx) {
    double sidx[3];
    donor_indices(S, i, j, k, sidx);
    int2 wx[P], wy[P], wz[P];
    int st[3];
    fixed_weights<P>(sidx, wx, wy, wz, st);
    if (st[0] < 0 || st[1] < 0 || st[2] < 0 || st[0] + P > S.gd.n[0] || st[1] + P > S.gd.n[1] ||
        st[2] + P > S.gd.n[2]) {
      atomicOr(A.err, ERR_UNFILLED);
      return;
    }
    const int E[2] = {max(dslot[0], 64), max(dslot[1], 64)};
    const double* D = reinterpret_cast<const double*>(S.D);
    const long long base = S.gd.at(st[0], st[1], st[2]);
    long long out[2];
    contract_point_fixed<P>(wx, wy, wz, [&](int f, int a, int b, int c) {
      return split31(to_fixed(D[f * S.gd.vol + base + c * S.gd.plane + b * S.gd.px + a], E[f]) * 64);
    }, out);
    const double v0 = (double)out[0] * __longlong_as_double((long long)(E[0] - 58) << 52);
    const double v1 = (double)out[1] * __longlong_as_double((long long)(E[1] - 58) << 52);
    double* Tt = reinterpret_cast<double*>(S.T);
    const long long c = S.gt.at(i, j, k);
    Tt[c] = v0;
    Tt[c + S.gt.vol] = v1;
    e0 = max(e0, biased_exponent(v0));
    e1 = max(e1, biased_exponent(v1));
    return;
  }
  double v0, v1, px, py, pz;
  donor_position(S, S.gt.lo[0] + (i + 0.5) * S.gt.h[0], S.gt.lo[1] + (j + 0.5) * S.gt.h[1],
                 S.gt.lo[2] + (k + 0.5) * S.gt.h[2], px, py, pz);
  if (!interp_point<P>(reinterpret_cast<const ST*>(S.D), S.gd, px, py, pz, v0, v1)) {
    atomicOr(A.err, ERR_UNFILLED);
    return;
  }
  ST* Tt = reinterpret_cast<ST*>(S.T);
  const long long c = S.gt.at(i, j, k);
  Tt[c] = (ST)v0;
  Tt[c + S.gt.vol] = (ST)v1;
  e0 = max(e0, biased_exponent(v0));
  e1 = max(e1, biased_exponent(v1));
}

// Fixed-point tensor sum at donor index coordinates sidx, the donors gathered
// and converted on the fly; WRAP: the third axis is periodic (a shell's
// azimuth).  False when the window leaves the donor interior.
template <int P, bool WRAP>
__device__ __forceinline__ bool gather_fixed(const InterpSeg& S, const double sidx[3], const int E[2], double& v0,
                                             double& v1) {
  int2 wx[P], wy[P], wz[P];
  int st[3];
  fixed_weights<P>(sidx, wx, wy, wz, st);
  if (st[0] < 0 || st[1] < 0 || st[0] + P > S.gd.n[0] || st[1] + P > S.gd.n[1]) return false;
  if (!WRAP && (st[2] < 0 || st[2] + P > S.gd.n[2])) return false;
  const double* D = reinterpret_cast<const double*>(S.D);
  long long out[2];
  contract_point_fixed<P>(wx, wy, wz, [&](int f, int a, int b, int c) {
    const int kz = WRAP ? wrap_index(st[2] + c, S.gd.n[2]) : st[2] + c;
    return split31(to_fixed(D[f * S.gd.vol + S.gd.at(st[0] + a, st[1] + b, kz)], E[f]) * 64);
  }, out);
  v0 = (double)out[0] * __longlong_as_double((long long)(E[0] - 58) << 52);
  v1 = (double)out[1] * __longlong_as_double((long long)(E[1] - 58) << 52);
  return true;
}

// The same sum from the donor's fixed-point mirror (no conversion per tap);
// false when the window leaves the mirrored box (or, without WRAP, the donor
// interior).
template <int P, bool WRAP>
__device__ __forceinline__ bool gather_mirror(const InterpSeg& S, const double sidx[3], const int E[2], double& v0,
                                              double& v1) {
  int2 wx[P], wy[P], wz[P];
  int st[3];
  fixed_weights<P>(sidx, wx, wy, wz, st);
  if (st[0] < 0 || st[1] < 0 || st[0] + P > S.gd.n[0] || st[1] + P > S.gd.n[1]) return false;
  if (!WRAP && (st[2] < 0 || st[2] + P > S.gd.n[2])) return false;
  const Box& b = S.mbox;
  const int mx = b.hi[0] - b.lo[0] + 1, my = b.hi[1] - b.lo[1] + 1, mz = b.hi[2] - b.lo[2] + 1;
  if (st[0] < b.lo[0] || st[0] + P - 1 > b.hi[0] || st[1] < b.lo[1] || st[1] + P - 1 > b.hi[1]) return false;
  if (!WRAP && (st[2] < b.lo[2] || st[2] + P - 1 > b.hi[2])) return false;
  const long long mvol = (long long)mx * my * mz;
  const int2* M = S.mir + (long long)(st[1] - b.lo[1]) * mx + (st[0] - b.lo[0]);
  long long out[2];
  contract_point_fixed<P>(wx, wy, wz, [&](int f, int a, int bb, int c) {
    const int kz = WRAP ? wrap_index(st[2] + c, S.gd.n[2]) : st[2] + c;
    return M[f * mvol + (long long)(kz - b.lo[2]) * mx * my + bb * mx + a];
  }, out);
  v0 = (double)out[0] * __longlong_as_double((long long)(E[0] - 58) << 52);
  v1 = (double)out[1] * __longlong_as_double((long long)(E[1] - 58) << 52);
  return true;
}

// Local-to-Global from a spherical shell: the global cell centre goes to the
// shell's Cartesian frame (M, shift), then to (r, theta, phi); the azimuthal
// window wraps.  Fixed point, or direct FP64 sums (native FP64, non-finite
// donors).
template <int P, typename ST>
__device__ __forceinline__ void l2g_point_sph(const FillArgs& A, const InterpSeg& S, int i, int j, int k, int& e0,
                                              int& e1) {
  const int* dslot = A.expo + S.dpatch * EXP_SLOTS_PER_PATCH + donor_buf(A, S) * 2;
  const bool fx = sizeof(ST) == 8 && A.fixed && dslot[0] < EXP_NONFINITE && dslot[1] < EXP_NONFINITE;
  double xf[3], q[3];
  affine(S.M, S.shift, S.gt.lo[0] + (i + 0.5) * S.gt.h[0], S.gt.lo[1] + (j + 0.5) * S.gt.h[1],
         S.gt.lo[2] + (k + 0.5) * S.gt.h[2], xf[0], xf[1], xf[2]);
  cart_to_sph(xf, q);
  double v0, v1;
  bool ok;
  if (fx) {
    const double sidx[3] = {(q[0] - S.gd.lo[0]) / S.gd.h[0] - 0.5, (q[1] - S.gd.lo[1]) / S.gd.h[1] - 0.5,
                            (q[2] - S.gd.lo[2]) / S.gd.h[2] - 0.5};
    const int E[2] = {max(dslot[0], 64), max(dslot[1], 64)};
    ok = (S.mir && gather_mirror<P, true>(S, sidx, E, v0, v1)) || gather_fixed<P, true>(S, sidx, E, v0, v1);
  } else {
    ok = interp_point_shell<P>(reinterpret_cast<const ST*>(S.D), S.gd, q[0], q[1], q[2], v0, v1);
  }
  if (!ok) {
    atomicOr(A.err, ERR_UNFILLED);
    return;
  }
  ST* Tt = reinterpret_cast<ST*>(S.T);
  const long long c = S.gt.at(i, j, k);
  Tt[c] = (ST)v0;
  Tt[c + S.gt.vol] = (ST)v1;
  e0 = max(e0, biased_exponent(v0));
  e1 = max(e1, biased_exponent(v1));
}

// The ghost nodes of a spherical shell, one thread per node of its hollow
// padded box.  Azimuthal ghosts (r and theta inside the live ranges) take
// their periodic image, the same physical point, from the shell's own
// interior; the others interpolate the global patch at X_B = M X' + shift
// (Sec. 2.4: the shell's radial and polar ghosts come from the global patch).
template <int P, typename ST>
__device__ __noinline__ void sph_ghost_block(const FillArgs& A, const InterpSeg& S, int r) {
  constexpr bool F32 = sizeof(ST) == 4;
  const int O[3] = {S.gt.n[0] + 2 * NG, S.gt.n[1] + 2 * NG, S.gt.n[2] + 2 * NG};
  const long long count = (long long)O[0] * O[1] * O[2] - (long long)S.gt.n[0] * S.gt.n[1] * S.gt.n[2];
  const long long idx = (long long)r * FILL_THREADS + threadIdx.x;
  int e0 = 0, e1 = 0;
  if (idx < count) {
    int x, y, z;
    if (count < (1ll << 31))
      shell_point_t<unsigned>((unsigned)idx, O, NG, x, y, z);
    else
      shell_point(idx, O, NG, x, y, z);
    const int i = x - NG, j = y - NG, k = z - NG;
    ST* Tt = reinterpret_cast<ST*>(S.T);
    const long long c = S.gt.at(i, j, k);
    if (i >= 0 && i < S.gt.n[0] && j >= 0 && j < S.gt.n[1]) {
      const long long src = S.gt.at(i, j, wrap_index(k, S.gt.n[2]));
      const ST v0 = Tt[src], v1 = Tt[src + S.gt.vol];
      Tt[c] = v0;
      Tt[c + S.gt.vol] = v1;
      e0 = biased_exponent((double)v0);
      e1 = biased_exponent((double)v1);
    } else {
      double xl[3], xb[3];
      sph_to_cart(S.gt.lo[0] + (i + 0.5) * S.gt.h[0], S.gt.lo[1] + (j + 0.5) * S.gt.h[1],
                  S.gt.lo[2] + (k + 0.5) * S.gt.h[2], xl);
      affine(S.M, S.shift, xl[0], xl[1], xl[2], xb[0], xb[1], xb[2]);
      const int* dslot = A.expo + S.dpatch * EXP_SLOTS_PER_PATCH + donor_buf(A, S) * 2;
      const bool fx = !F32 && A.fixed && dslot[0] < EXP_NONFINITE && dslot[1] < EXP_NONFINITE;
      double v0, v1;
      bool ok;
      if (fx) {
        double sidx[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) sidx[a] = (xb[a] - S.gd.lo[a]) / S.gd.h[a] - 0.5;
        const int E[2] = {max(dslot[0], 64), max(dslot[1], 64)};
        ok = (S.mir && gather_mirror<P, false>(S, sidx, E, v0, v1)) || gather_fixed<P, false>(S, sidx, E, v0, v1);
      } else {
        ok = interp_point<P>(reinterpret_cast<const ST*>(S.D), S.gd, xb[0], xb[1], xb[2], v0, v1);
      }
      if (ok) {
        Tt[c] = (ST)v0;
        Tt[c + S.gt.vol] = (ST)v1;
        e0 = biased_exponent(v0);
        e1 = biased_exponent(v1);
      } else {
        atomicOr(A.err, ERR_UNFILLED);
      }
    }
  }
  if (!F32) report_block_max(A.expo + S.tpatch * EXP_SLOTS_PER_PATCH + EXP_GHOST + A.y_buf * 2, e0, e1);
}

// Local-to-Global under a rotating map, from the cover flags: one thread per
// cell of the covered bounding box; the cells whose flag byte is S.want
// (effective ghosts of this patch) are filled.
template <int P, typename ST>
__device__ __noinline__ void masked_block(const FillArgs& A, const InterpSeg& S, int r) {
  constexpr bool F32 = sizeof(ST) == 4;
  const Box& b = S.box;
  const int w0 = b.hi[0] - b.lo[0] + 1, w1 = b.hi[1] - b.lo[1] + 1, w2 = b.hi[2] - b.lo[2] + 1;
  const long long idx = (long long)r * FILL_THREADS + threadIdx.x;
  int e0 = 0, e1 = 0;
  if (idx < (long long)w0 * w1 * w2) {
    const int i = b.lo[0] + (int)(idx % w0), j = b.lo[1] + (int)((idx / w0) % w1),
              k = b.lo[2] + (int)(idx / ((long long)w0 * w1));
    if (S.flags[((long long)k * S.gt.n[1] + j) * S.gt.n[0] + i] == S.want) {
      if (S.sph)
        l2g_point_sph<P, ST>(A, S, i, j, k, e0, e1);
      else
        l2g_point<P, ST>(A, S, i, j, k, e0, e1);
    }
  }
  if (!F32) report_block_max(A.expo + S.tpatch * EXP_SLOTS_PER_PATCH + EXP_GHOST + A.y_buf * 2, e0, e1);
}

// Local-to-Global under a rotating map, from the list of the patch's
// effective ghosts written by the cover-flag kernel (dense warps).
template <int P, typename ST>
__device__ __noinline__ void list_block(const FillArgs& A, const InterpSeg& S, int r) {
  constexpr bool F32 = sizeof(ST) == 4;
  const int count = *S.count;
  int e0 = 0, e1 = 0;
  for (int base = r * FILL_THREADS; base < count; base += S.list_blocks * FILL_THREADS) {
    const int e = base + threadIdx.x;
    if (e < count) {
      const long long idx = S.list[e];
      const int i = (int)(idx % S.gt.n[0]);
      const long long rr = idx / S.gt.n[0];
      if (S.sph)
        l2g_point_sph<P, ST>(A, S, i, (int)(rr % S.gt.n[1]), (int)(rr / S.gt.n[1]), e0, e1);
      else
        l2g_point<P, ST>(A, S, i, (int)(rr % S.gt.n[1]), (int)(rr / S.gt.n[1]), e0, e1);
    }
  }
  if (!F32) report_block_max(A.expo + S.tpatch * EXP_SLOTS_PER_PATCH + EXP_GHOST + A.y_buf * 2, e0, e1);
}

// A tile of a rotated ghost shell in fixed point: the donor box that the
// tile's windows cover (the donor index is affine in the target indices, so
// its range follows from the tile's corners, widened by one cell against
// rounding) is converted once into shared memory; every target then takes
// its own weights and the fixed-point sum from there.  Returns false, with
// nothing written, when the box does not fit or leaves the donor interior.
template <int P>
__device__ __noinline__ bool affine_tile_fixed(const FillArgs& A, const InterpSeg& S, const int org[3], const int T[3], int Es,
                                  int Ep, double* sm, int emax[2]) {
  __shared__ int s_box[7];
  constexpr int CAPB = CAP_R1 + CAP_R2;  // donors per field
  if (threadIdx.x == 0) {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int c = 0; c < 8; ++c) {
      double sidx[3];
      donor_indices(S, org[0] + ((c & 1) ? T[0] - 1 : 0), org[1] + ((c & 2) ? T[1] - 1 : 0),
                    org[2] + ((c & 4) ? T[2] - 1 : 0), sidx);
      for (int a = 0; a < 3; ++a) {
        lo[a] = fmin(lo[a], sidx[a]);
        hi[a] = fmax(hi[a], sidx[a]);
      }
    }
    bool ok = true;
    long long vol = 1;
    for (int a = 0; a < 3; ++a) {
      const int d0 = (int)floor(lo[a]) - 3, d1 = (int)floor(hi[a]) + P - 1;  // window starts floor(s) - 2, +-1
      s_box[a] = max(d0, 0);
      s_box[3 + a] = min(d1, S.gd.n[a] - 1) - s_box[a] + 1;
      ok = ok && s_box[3 + a] > 0;
      vol *= max(s_box[3 + a], 1);
    }
    s_box[6] = ok && vol <= CAPB;
  }
  __syncthreads();
  if (!s_box[6]) return false;
  const int D0[3] = {s_box[0], s_box[1], s_box[2]}, Dn[3] = {s_box[3], s_box[4], s_box[5]};
  const int nb = Dn[0] * Dn[1] * Dn[2], bxy = Dn[0] * Dn[1];
  int2* blk = reinterpret_cast<int2*>(sm);
  const double* D = reinterpret_cast<const double*>(S.D);
  const int E[2] = {max(Es, 64), max(Ep, 64)};
  for (int e = threadIdx.x; e < 2 * nb; e += FILL_THREADS) {
    const int f = e >= nb;
    const int r = e - f * nb;
    const int x = r % Dn[0], y = (r / Dn[0]) % Dn[1], z = r / bxy;
    blk[f * CAPB + r] =
        split31(to_fixed(D[f * S.gd.vol + S.gd.at(D0[0] + x, D0[1] + y, D0[2] + z)], E[f]) * 64);
  }
  __syncthreads();
  double* Tt = reinterpret_cast<double*>(S.T);
  const int ntar = T[0] * T[1] * T[2];
  const double p2[2] = {__longlong_as_double((long long)(E[0] - 58) << 52),
                        __longlong_as_double((long long)(E[1] - 58) << 52)};
  for (int e = threadIdx.x; e < ntar; e += FILL_THREADS) {
    const int i = org[0] + e % T[0], j = org[1] + (e / T[0]) % T[1], k = org[2] + e / (T[0] * T[1]);
    double sidx[3];
    donor_indices(S, i, j, k, sidx);
    int2 wx[P], wy[P], wz[P];
    int st[3];
    fixed_weights<P>(sidx, wx, wy, wz, st);
    const int rx = st[0] - D0[0], ry = st[1] - D0[1], rz = st[2] - D0[2];
    if (rx < 0 || ry < 0 || rz < 0 || rx + P > Dn[0] || ry + P > Dn[1] || rz + P > Dn[2]) {
      // outside the staged box (only possible at the donor's faces): unfilled
      atomicOr(A.err, ERR_UNFILLED);
      continue;
    }
    const int2* b0 = blk + rz * bxy + ry * Dn[0] + rx;
    long long out[2];
    contract_point_fixed<P>(wx, wy, wz, [&](int f, int a, int b, int c) {
      return b0[f * CAPB + c * bxy + b * Dn[0] + a];
    }, out);
    const long long cc = S.gt.at(i, j, k);
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const double v = (double)out[f] * p2[f];
      Tt[cc + f * S.gt.vol] = v;
      emax[f] = max(emax[f], biased_exponent(v));
    }
  }
  return true;
}

// One interpolation tile.  ST is the storage type of the field buffers:
// double (arithmetic FP64 or fixed point, FillArgs::fixed) or float (FP32
// arithmetic, with the weights computed in FP64 and rounded once).
template <int P, typename ST>
__device__ void interp_tile(const FillArgs& A, const InterpSeg& S, const int org[3], const int T[3], int a0,
                            double* sm) {
  constexpr bool F32 = sizeof(ST) == 4;
  double* R1 = sm;                          // [2][CAP_R1]
  double* R2 = R1 + 2 * CAP_R1;             // [2][CAP_R2]
  double* W = R2 + 2 * CAP_R2;              // [3][MAXT][6]
  int2* WQ = reinterpret_cast<int2*>(W + 3 * MAXT * 6);  // [3][MAXT][6] weights on 2^59 split, or binary32
  double* BW = reinterpret_cast<double*>(WQ + 3 * MAXT * 6);  // [MAXT0][MAXD] band matrix of the thin axis
  int2* BQ = reinterpret_cast<int2*>(BW + MAXT0 * MAXD);      // the same on 2^59 split, or binary32
  int* WS = reinterpret_cast<int*>(BQ + MAXT0 * MAXD);   // [3][MAXT] window starts
  float* WF = reinterpret_cast<float*>(WQ);
  float* BF = reinterpret_cast<float*>(BQ);
  ST* Tt = reinterpret_cast<ST*>(S.T);
  const int tid = threadIdx.x;
  if (S.kind == SEG_AFFINE) {
    // rotated target grid: the 1-D weights differ from point to point
    int emax[2] = {0, 0};
    const int* dslot = A.expo + S.dpatch * EXP_SLOTS_PER_PATCH + donor_buf(A, S) * 2;
    const bool fx = !F32 && A.fixed && dslot[0] < EXP_NONFINITE && dslot[1] < EXP_NONFINITE;
    if (!fx || !affine_tile_fixed<P>(A, S, org, T, dslot[0], dslot[1], sm, emax))
      direct_points<P, ST>(A, S, org, T, emax);
    if (!F32) report_block_max(A.expo + S.tpatch * EXP_SLOTS_PER_PATCH + EXP_GHOST + A.y_buf * 2, emax[0], emax[1]);
    return;
  }
  // 1-D weights of every target index of the tile, per axis; the threads of
  // the thin axis also write their row of the band matrix
  for (int e = tid; e < T[0] + T[1] + T[2]; e += FILL_THREADS) {
    const int a = e < T[0] ? 0 : (e < T[0] + T[1] ? 1 : 2);
    const int k = e - (a == 0 ? 0 : (a == 1 ? T[0] : T[0] + T[1]));
    double w[P];
    const int start = lagrange_weights<P>(donor_index(S, a, org[a] + k), w);
    WS[a * MAXT + k] = start;
#pragma unroll
    for (int m = 0; m < P; ++m) {
      W[(a * MAXT + k) * 6 + m] = w[m];
      if (F32)
        WF[(a * MAXT + k) * 6 + m] = (float)w[m];
      else
        WQ[(a * MAXT + k) * 6 + m] = split31(__double2ll_rn(w[m] * 0x1p59));
    }
    if (a == a0 && k < MAXT0) {
      double w0[P];
      const int off = start - lagrange_weights<P>(donor_index(S, a, org[a]), w0);  // window offset in the block
      for (int q = 0; q < MAXD; ++q) {
        const int m = q - off;
        const bool in = m >= 0 && m < P;
        double wm = 0.0;
#pragma unroll
        for (int mm = 0; mm < P; ++mm)
          if (mm == m) wm = w[mm];
        BW[k * MAXD + q] = in ? wm : 0.0;
        if (F32)
          BF[k * MAXD + q] = in ? (float)wm : 0.0f;
        else
          BQ[k * MAXD + q] = in ? split31(__double2ll_rn(wm * 0x1p59)) : make_int2(0, 0);
      }
    }
  }
  __syncthreads();
  int D0[3], Dn[3];
  bool inside = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    D0[a] = WS[a * MAXT];
    Dn[a] = WS[a * MAXT + T[a] - 1] - D0[a] + P;
    inside = inside && D0[a] >= 0 && D0[a] + Dn[a] <= S.gd.n[a];
  }
  // after the thin pass: contract the wide axis whose pass leaves the
  // smaller block first
  const int b1 = a0 == 0 ? 1 : 0, b2 = a0 == 2 ? 1 : 2;
  const long long s1 = (long long)T[a0] * Dn[b1] * Dn[b2];
  const long long s2a = (long long)T[a0] * T[b1] * Dn[b2], s2b = (long long)T[a0] * Dn[b1] * T[b2];
  const int x1 = s2a <= s2b ? b1 : b2, x2 = s2a <= s2b ? b2 : b1;
  const bool fits = inside && T[a0] <= MAXT0 && Dn[a0] <= MAXD && s1 <= CAP_R1 && (s2a <= s2b ? s2a : s2b) <= CAP_R2;
  int emax[2] = {0, 0};
  const int ntar = T[0] * T[1] * T[2];
  if (!fits) {
    direct_points<P, ST>(A, S, org, T, emax);
  } else {
    int d1[3] = {Dn[0], Dn[1], Dn[2]};
    d1[a0] = T[a0];
    int d2[3] = {d1[0], d1[1], d1[2]};
    d2[x1] = T[x1];
    // donor scale: the largest exponent of the donor buffer's live values
    // (complete before this launch; the fill itself only raises the ghost
    // slots), so the scale is known before the donors are read
    const int* dslot = A.expo + S.dpatch * EXP_SLOTS_PER_PATCH + donor_buf(A, S) * 2;
    const int Es = dslot[0], Ep = dslot[1];
    if (F32) {
      thin_pass<P, M_FP32, ST>(S, a0, D0, Dn, T[a0], BF, 0, 0, R1);
      __syncthreads();
      contract<P, M_FP32, false>(R1, CAP_R1, R2, CAP_R2, d1, x1, T[x1], WF + x1 * MAXT * 6, WS + x1 * MAXT, D0[x1]);
      __syncthreads();
      contract<P, M_FP32, false>(R2, CAP_R2, R1, CAP_R1, d2, x2, T[x2], WF + x2 * MAXT * 6, WS + x2 * MAXT, D0[x2]);
      __syncthreads();
      const float* out = reinterpret_cast<const float*>(R1);
      BlockWalk<FILL_THREADS> wk(tid, T[0], T[1], T[2]);
      for (int e = tid; e < 2 * ntar; e += FILL_THREADS, wk.next()) {
        const int f = wk.f;
        const int r = e - f * ntar;
        const int tx = wk.o0, ty = wk.o1, tz = wk.o2;
        Tt[S.gt.at(org[0] + tx, org[1] + ty, org[2] + tz) + f * S.gt.vol] = (ST)out[f * CAP_R1 + r];
      }
    } else if (A.fixed && Es < EXP_NONFINITE && Ep < EXP_NONFINITE) {
      const int Esu = max(Es, 64), Epu = max(Ep, 64);
      thin_pass<P, M_FIXED, ST>(S, a0, D0, Dn, T[a0], BQ, Esu, Epu, R1);
      __syncthreads();
      contract<P, M_FIXED, false>(R1, CAP_R1, R2, CAP_R2, d1, x1, T[x1], WQ + x1 * MAXT * 6, WS + x1 * MAXT, D0[x1]);
      __syncthreads();
      contract<P, M_FIXED, true>(R2, CAP_R2, R1, CAP_R1, d2, x2, T[x2], WQ + x2 * MAXT * 6, WS + x2 * MAXT, D0[x2]);
      __syncthreads();
      // results are on 2^(E - 1075 - 6): exact power-of-two scalings
      const double p2[2] = {__longlong_as_double((long long)(Esu - 58) << 52),
                            __longlong_as_double((long long)(Epu - 58) << 52)};
      const long long* out = reinterpret_cast<const long long*>(R1);
      BlockWalk<FILL_THREADS> wk(tid, T[0], T[1], T[2]);
      for (int e = tid; e < 2 * ntar; e += FILL_THREADS, wk.next()) {
        const int f = wk.f;
        const int r = e - f * ntar;
        const int tx = wk.o0, ty = wk.o1, tz = wk.o2;
        const double v = (double)out[f * CAP_R1 + r] * p2[f];
        Tt[S.gt.at(org[0] + tx, org[1] + ty, org[2] + tz) + f * S.gt.vol] = (ST)v;
        emax[f] = max(emax[f], biased_exponent(v));
      }
    } else {
      thin_pass<P, M_FP64, ST>(S, a0, D0, Dn, T[a0], BW, 0, 0, R1);
      __syncthreads();
      contract<P, M_FP64, false>(R1, CAP_R1, R2, CAP_R2, d1, x1, T[x1], W + x1 * MAXT * 6, WS + x1 * MAXT, D0[x1]);
      __syncthreads();
      contract<P, M_FP64, false>(R2, CAP_R2, R1, CAP_R1, d2, x2, T[x2], W + x2 * MAXT * 6, WS + x2 * MAXT, D0[x2]);
      __syncthreads();
      BlockWalk<FILL_THREADS> wk(tid, T[0], T[1], T[2]);
      for (int e = tid; e < 2 * ntar; e += FILL_THREADS, wk.next()) {
        const int f = wk.f;
        const int r = e - f * ntar;
        const int tx = wk.o0, ty = wk.o1, tz = wk.o2;
        const double v = R1[f * CAP_R1 + r];
        Tt[S.gt.at(org[0] + tx, org[1] + ty, org[2] + tz) + f * S.gt.vol] = (ST)v;
        emax[f] = max(emax[f], biased_exponent(v));
      }
    }
    // each thread's emax[f] covers only entries of field f, the other stays 0
  }
  // exponent slots are kept for binary64 buffers only (the fixed-point scale)
  if (!F32) report_block_max(A.expo + S.tpatch * EXP_SLOTS_PER_PATCH + EXP_GHOST + A.y_buf * 2, emax[0], emax[1]);
}

}  // namespace

// Body of the fill for block b0 of the launch described by A.  The launch
// runs the interpolation tiles first and the outer-shell blocks after them
// (the tiles take longer; measured 5 % faster than the other order); b is
// the block in A's numbering (outer shell first, then the segments).
template <int P, typename ST>
__device__ __forceinline__ void fill_body(const FillArgs& A, const int b0) {
  constexpr bool F32 = sizeof(ST) == 4;
  extern __shared__ double fill_smem[];
  const int ntile = A.total_blocks - A.outer_blocks;
  const int b = b0 < ntile ? b0 + A.outer_blocks : b0 - ntile;
  if (A.reset_buf >= 0 && b0 == 0 && threadIdx.x >= 2 * A.reset_first && threadIdx.x < 2 * A.np)
    A.expo[(threadIdx.x >> 1) * EXP_SLOTS_PER_PATCH + A.reset_buf * 2 + (threadIdx.x & 1)] = 0;
  if (A.reset_buf >= 0 && b0 == 0 && threadIdx.x >= 2 * A.reset_first && threadIdx.x < 2 * A.np)
    A.expo[(threadIdx.x >> 1) * EXP_SLOTS_PER_PATCH + EXP_GHOST + A.reset_buf * 2 + (threadIdx.x & 1)] = 0;
  if (b < A.outer_blocks) {
    // global outer ghost shell, one point per thread
    const long long idx = (long long)b * FILL_THREADS + threadIdx.x;
    int e0 = 0, e1 = 0;
    if (idx < A.outer_count) {
      const int O[3] = {A.gg.n[0] + 2 * NG, A.gg.n[1] + 2 * NG, A.gg.n[2] + 2 * NG};
      int x, y, z;
      if (A.outer_count < (1ll << 31))
        shell_point_t<unsigned>((unsigned)idx, O, NG, x, y, z);
      else
        shell_point(idx, O, NG, x, y, z);
      const int i = x - NG, j = y - NG, k = z - NG;
      const long long c = A.gg.at(i, j, k);
      ST* Yg = reinterpret_cast<ST*>(A.Yg);
      const ST* shell = reinterpret_cast<const ST*>(A.shell_src);
      ST w0, w1;
      if (A.outer_bc == 1) {
        const long long s =
            A.gg.at(wrap_index(i, A.gg.n[0]), wrap_index(j, A.gg.n[1]), wrap_index(k, A.gg.n[2]));
        w0 = Yg[s];
        w1 = Yg[s + A.gg.vol];
      } else if (shell) {
        // the closed form at this very time already sits in another buffer's shell
        w0 = shell[c];
        w1 = shell[c + A.gg.vol];
      } else {
        double v0, v1;
        closed_form(A.akind, A.aparams, A.ascreen, A.apre, A.acount, A.t, A.gg.lo[0] + (i + 0.5) * A.gg.h[0],
                    A.gg.lo[1] + (j + 0.5) * A.gg.h[1], A.gg.lo[2] + (k + 0.5) * A.gg.h[2], v0, v1);
        w0 = (ST)v0;
        w1 = (ST)v1;
      }
      Yg[c] = w0;
      Yg[c + A.gg.vol] = w1;
      e0 = biased_exponent((double)w0);
      e1 = biased_exponent((double)w1);
    }
    if (!F32) report_block_max(A.expo + EXP_GHOST + A.y_buf * 2, e0, e1);
    return;
  }
  // interpolation tile: find its segment, slab and position
  int s = 0;
  while (s + 1 < A.nseg && b >= A.seg[s + 1].block0) ++s;
  const InterpSeg& S = A.seg[s];
  int r = b - S.block0;
  if (S.kind == SEG_MASKED) {
    masked_block<P, ST>(A, S, r);
    return;
  }
  if (S.kind == SEG_LIST) {
    list_block<P, ST>(A, S, r);
    return;
  }
  if (S.kind == SEG_SPH_GHOSTS) {
    sph_ghost_block<P, ST>(A, S, r);
    return;
  }
  int sl = 0;
  while (sl < 5 && r >= S.slab_block0[sl + 1]) ++sl;
  r -= S.slab_block0[sl];
  const int nx = S.tn[sl][0], ny = S.tn[sl][1];
  const int tx = r % nx, ty = (r / nx) % ny, tz = r / (nx * ny);
  int org[3], T[3];
  const int tt[3] = {tx, ty, tz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    org[a] = S.sb[sl][a] + tt[a] * S.td[sl][a];
    T[a] = min(S.td[sl][a], S.sb[sl][a] + S.se[sl][a] - org[a]);
  }
  interp_tile<P, ST>(A, S, org, T, 2 - sl / 2, fill_smem);  // slabs come in z, y, x pairs: the wall axis is thin
}

// Fixed-point mirrors of the donor regions of a fill (binary64 buffers): one
// thread per cell of each region, both fields.
__global__ void __launch_bounds__(256) k_mirror(const __grid_constant__ MirrorArgs A) {
  const long long b = blockIdx.x;
  int q = 0;
  while (q + 1 < A.nr && b >= A.r[q + 1].block0) ++q;
  const MirrorRegion& R = A.r[q];
  const int mx = R.box.hi[0] - R.box.lo[0] + 1, my = R.box.hi[1] - R.box.lo[1] + 1,
            mz = R.box.hi[2] - R.box.lo[2] + 1;
  const long long mvol = (long long)mx * my * mz;
  const long long idx = (b - R.block0) * 256 + threadIdx.x;
  if (idx >= mvol) return;
  const int x = (int)(idx % mx), y = (int)((idx / mx) % my), z = (int)(idx / ((long long)mx * my));
  const long long c = R.g.at(R.box.lo[0] + x, R.box.lo[1] + y, R.box.lo[2] + z);
  const int* slot = A.expo + R.patch * EXP_SLOTS_PER_PATCH + A.y_buf * 2;
#pragma unroll
  for (int f = 0; f < 2; ++f) {
    const int E = max(slot[f], 64);  // a non-finite scale sends the fill to its FP64 path
    R.dst[f * mvol + idx] = split31(to_fixed(R.src[c + f * R.g.vol], E) * 64);
  }
}

void launch_mirror(const MirrorArgs& a, void* stream) {
  if (a.nr > 0 && a.blocks > 0) k_mirror<<<(unsigned)a.blocks, 256, 0, (cudaStream_t)stream>>>(a);
}

template <int P, typename ST>
__global__ void __launch_bounds__(FILL_THREADS, 2) k_fill(const __grid_constant__ FillArgs A) {
  fill_body<P, ST>(A, blockIdx.x);
}

// Batched launch: instance i owns blocks [blk0[i], blk0[i + 1]), arguments
// As[i]; blocks from blk0[ninst] on (a grid padded to a captured capacity)
// have no work.
template <int P, typename ST>
__global__ void __launch_bounds__(FILL_THREADS, 2) k_fill_batch(const FillArgs* __restrict__ As,
                                                             const int* __restrict__ blk0, int ninst) {
  if ((int)blockIdx.x >= blk0[ninst]) return;
  int lo = 0, hi = ninst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((int)blockIdx.x >= blk0[mid]) lo = mid; else hi = mid - 1;
  }
  fill_body<P, ST>(As[lo], blockIdx.x - blk0[lo]);
}

template <int P, typename ST>
static void launch_fill_batch_t(const FillArgs* d_args, const int* d_blk0, int ninst, int blocks, cudaStream_t s) {
  cudaFuncSetAttribute(k_fill_batch<P, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FILL_SMEM);
  k_fill_batch<P, ST><<<blocks, FILL_THREADS, FILL_SMEM, s>>>(d_args, d_blk0, ninst);
}

void launch_fill_batch(const FillArgs* d_args, const int* d_blk0, int ninst, int blocks, int P, bool f32,
                       void* stream) {
  if (blocks <= 0) return;
  const cudaStream_t s = (cudaStream_t)stream;
  if (f32)
    P == 6 ? launch_fill_batch_t<6, float>(d_args, d_blk0, ninst, blocks, s)
           : launch_fill_batch_t<5, float>(d_args, d_blk0, ninst, blocks, s);
  else
    P == 6 ? launch_fill_batch_t<6, double>(d_args, d_blk0, ninst, blocks, s)
           : launch_fill_batch_t<5, double>(d_args, d_blk0, ninst, blocks, s);
}

template <int P, typename ST>
static void launch_fill_t(const FillArgs& a, cudaStream_t s) {
  cudaFuncSetAttribute(k_fill<P, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FILL_SMEM);
  k_fill<P, ST><<<a.total_blocks, FILL_THREADS, FILL_SMEM, s>>>(a);
}

void launch_fill(const FillArgs& a, void* stream) {
  if (a.total_blocks <= 0) return;
  const cudaStream_t s = (cudaStream_t)stream;
  if (a.f32)
    a.P == 6 ? launch_fill_t<6, float>(a, s) : launch_fill_t<5, float>(a, s);
  else
    a.P == 6 ? launch_fill_t<6, double>(a, s) : launch_fill_t<5, double>(a, s);
}

int fill_cap_r1() { return CAP_R1; }
int fill_cap_r2() { return CAP_R2; }
int fill_max_tile() { return MAXT; }
int fill_max_thin_donors() { return MAXD; }
int fill_threads() { return FILL_THREADS; }

}  // namespace mpw
