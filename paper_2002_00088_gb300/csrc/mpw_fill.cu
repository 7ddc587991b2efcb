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

// shared-memory budget of one CTA of the separable path, in doubles (one
// field at a time): donor block, x-contracted block, xy-contracted block
constexpr int CAP_D = 4096;
constexpr int CAP_R1 = 2560;
constexpr int CAP_R2 = 2048;
constexpr int MAXT = 32;  // largest tile extent along an axis
constexpr int FILL_THREADS = 256;
constexpr size_t FILL_SMEM = sizeof(double) * (2 * CAP_D + CAP_R1 + CAP_R2 + 3 * MAXT * 6) + sizeof(int) * 3 * MAXT +
                             sizeof(int2) * 3 * MAXT * 6;

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
__device__ __forceinline__ double donor_index(const InterpSeg& S, int a, int i) {
  return ((S.gt.lo[a] + (i + 0.5) * S.gt.h[a] + S.shift[a]) - S.gd.lo[a]) / S.gd.h[a] - 0.5;
}

// One separable pass: contract axis AX of the block `in` (extents din, x
// fastest) against the 1-D weights of the tile's targets along AX, giving the
// block `out` whose extent along AX is the number of targets T.  ws holds the
// absolute window starts, off the block origin along AX, w the P weights per
// target.
template <int P, int AX>
__device__ __forceinline__ void contract_axis(const double* __restrict__ in, double* __restrict__ out, const int din[3],
                                              int T, const double* __restrict__ w, const int* __restrict__ ws, int off) {
  const int d0 = AX == 0 ? T : din[0], d1 = AX == 1 ? T : din[1], d2 = AX == 2 ? T : din[2];
  const int s1 = din[0], s2 = din[0] * din[1];
  const int st = AX == 0 ? 1 : (AX == 1 ? s1 : s2);
  const int n = d0 * d1 * d2;
  for (int e = threadIdx.x; e < n; e += FILL_THREADS) {
    int o0 = e % d0, o1 = (e / d0) % d1, o2 = e / (d0 * d1);
    const int t = AX == 0 ? o0 : (AX == 1 ? o1 : o2);
    const int c = ws[t] - off;
    if (AX == 0) o0 = c;
    if (AX == 1) o1 = c;
    if (AX == 2) o2 = c;
    const double* src = in + o0 + o1 * s1 + o2 * s2;
    const double* wt = w + t * 6;
    double acc = 0.0;
#pragma unroll
    for (int m = 0; m < P; ++m) acc = fma(wt[m], src[m * st], acc);
    out[e] = acc;
  }
}

// 8-byte asynchronous global -> shared copy (no register round trip) and the
// wait for all of this thread's copies.
__device__ __forceinline__ void cp_async8(double* dst, const double* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;" ::: "memory");
}

// v = hi 2^31 + lo with 0 <= lo < 2^31 (|v| < 2^62).
__device__ __forceinline__ int2 split31(long long v) {
  return make_int2((int)(v & 0x7FFFFFFFll), (int)(v >> 31));
}

// Fixed-point version of contract_axis: inputs and weights split at bit 31
// (x = low 31 bits, y = the rest), output = sum_m a_m w_m / 2^59 from the
// high x high, high x low and low x high partial products, split again for
// the next pass or kept whole after the last one (FINAL).
template <int P, int AX, bool FINAL>
__device__ __forceinline__ void contract_axis_fx(const int2* __restrict__ in, void* __restrict__ out, const int din[3],
                                                 int T, const int2* __restrict__ w, const int* __restrict__ ws,
                                                 int off) {
  const int d0 = AX == 0 ? T : din[0], d1 = AX == 1 ? T : din[1], d2 = AX == 2 ? T : din[2];
  const int s1 = din[0], s2 = din[0] * din[1];
  const int st = AX == 0 ? 1 : (AX == 1 ? s1 : s2);
  const int n = d0 * d1 * d2;
  for (int e = threadIdx.x; e < n; e += FILL_THREADS) {
    int o0 = e % d0, o1 = (e / d0) % d1, o2 = e / (d0 * d1);
    const int t = AX == 0 ? o0 : (AX == 1 ? o1 : o2);
    const int c = ws[t] - off;
    if (AX == 0) o0 = c;
    if (AX == 1) o1 = c;
    if (AX == 2) o2 = c;
    const int2* src = in + o0 + o1 * s1 + o2 * s2;
    const int2* wt = w + t * 6;
    long long hh = 0, hl = 0, lh = 0;
#pragma unroll
    for (int m = 0; m < P; ++m) {
      const int2 a = src[m * st];
      const int2 b = wt[m];
      hh += (long long)a.y * b.y;
      hl += (long long)a.y * b.x;
      lh += (long long)a.x * b.y;
    }
    const long long v = hh * 8 + (hl >> 28) + (lh >> 28);
    if (FINAL)
      static_cast<long long*>(out)[e] = v;
    else
      static_cast<int2*>(out)[e] = split31(v);
  }
}

template <int P, bool FINAL>
__device__ __forceinline__ void contract_fx(const int2* in, void* out, const int din[3], int ax, int T, const int2* w,
                                            const int* ws, int off) {
  if (ax == 0)
    contract_axis_fx<P, 0, FINAL>(in, out, din, T, w, ws, off);
  else if (ax == 1)
    contract_axis_fx<P, 1, FINAL>(in, out, din, T, w, ws, off);
  else
    contract_axis_fx<P, 2, FINAL>(in, out, din, T, w, ws, off);
}

template <int P>
__device__ __forceinline__ void contract(const double* in, double* out, const int din[3], int ax, int T,
                                         const double* w, const int* ws, int off) {
  if (ax == 0)
    contract_axis<P, 0>(in, out, din, T, w, ws, off);
  else if (ax == 1)
    contract_axis<P, 1>(in, out, din, T, w, ws, off);
  else
    contract_axis<P, 2>(in, out, din, T, w, ws, off);
}

template <int P>
__device__ void interp_tile(const FillArgs& A, const InterpSeg& S, const int org[3], const int T[3], double* sm) {
  double* D = sm;                          // [2][CAP_D] donor blocks of psi and Pi
  double* R1 = D + 2 * CAP_D;
  double* R2 = R1 + CAP_R1;
  double* W = R2 + CAP_R2;                 // [3][MAXT][6]
  int* WS = reinterpret_cast<int*>(W + 3 * MAXT * 6);  // [3][MAXT] window starts
  int2* WQ = reinterpret_cast<int2*>(WS + 3 * MAXT);   // [3][MAXT][6] weights on 2^59, split
  __shared__ int s_E[2];                   // largest biased exponent of each field's donor block
  const int tid = threadIdx.x;
  if (tid < 2) s_E[tid] = 0;
  // 1-D weights of every target index of the tile, per axis
  for (int e = tid; e < T[0] + T[1] + T[2]; e += FILL_THREADS) {
    const int a = e < T[0] ? 0 : (e < T[0] + T[1] ? 1 : 2);
    const int k = e - (a == 0 ? 0 : (a == 1 ? T[0] : T[0] + T[1]));
    double w[P];
    WS[a * MAXT + k] = lagrange_weights<P>(donor_index(S, a, org[a] + k), w);
#pragma unroll
    for (int m = 0; m < P; ++m) {
      W[(a * MAXT + k) * 6 + m] = w[m];
      WQ[(a * MAXT + k) * 6 + m] = split31(__double2ll_rn(w[m] * 0x1p59));
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
  // order of the three passes: the one with the fewest multiply-adds whose
  // intermediate blocks fit the shared-memory budget
  int ord[3] = {0, 1, 2};
  bool fits = Dn[0] * Dn[1] * Dn[2] <= CAP_D;
  if (fits) {
    long long best = -1;
    for (int pm = 0; pm < 6; ++pm) {
      const int a0 = pm >> 1, a1 = (a0 + 1 + (pm & 1)) % 3, a2 = 3 - a0 - a1;
      const int Ta0 = a0 == 0 ? T[0] : (a0 == 1 ? T[1] : T[2]);
      const int Ta1 = a1 == 0 ? T[0] : (a1 == 1 ? T[1] : T[2]);
      const int Da1 = a1 == 0 ? Dn[0] : (a1 == 1 ? Dn[1] : Dn[2]);
      const int Da2 = a2 == 0 ? Dn[0] : (a2 == 1 ? Dn[1] : Dn[2]);
      const long long s1 = (long long)Ta0 * Da1 * Da2;
      const long long s2 = (long long)Ta0 * Ta1 * Da2;
      const long long s3 = (long long)T[0] * T[1] * T[2];
      if (s1 > CAP_R1 || s2 > CAP_R2) continue;
      const long long cost = s1 + s2 + s3;
      if (best < 0 || cost < best) {
        best = cost;
        ord[0] = a0, ord[1] = a1, ord[2] = a2;
      }
    }
    fits = best >= 0;
  }
  int emax[2] = {0, 0};
  const int ntar = T[0] * T[1] * T[2];
  if (!(inside && fits)) {
    // direct tensor sum, point by point (reports uninterpolable points)
    for (int e = tid; e < ntar; e += FILL_THREADS) {
      const int x = e % T[0], y = (e / T[0]) % T[1], z = e / (T[0] * T[1]);
      const int i = org[0] + x, j = org[1] + y, k = org[2] + z;
      double v0, v1;
      const double px = S.gt.lo[0] + (i + 0.5) * S.gt.h[0] + S.shift[0];
      const double py = S.gt.lo[1] + (j + 0.5) * S.gt.h[1] + S.shift[1];
      const double pz = S.gt.lo[2] + (k + 0.5) * S.gt.h[2] + S.shift[2];
      if (!interp_point<P>(S.D, S.gd, px, py, pz, v0, v1)) {
        atomicOr(A.err, ERR_UNFILLED);
        continue;
      }
      const long long c = S.gt.at(i, j, k);
      S.T[c] = v0;
      S.T[c + S.gt.vol] = v1;
      emax[0] = max(emax[0], biased_exponent(v0));
      emax[1] = max(emax[1], biased_exponent(v1));
    }
  } else {
    const int nD = Dn[0] * Dn[1] * Dn[2];
    int d1[3] = {Dn[0], Dn[1], Dn[2]};
    d1[ord[0]] = T[ord[0]];
    int d2[3] = {d1[0], d1[1], d1[2]};
    d2[ord[1]] = T[ord[1]];
    // donor blocks of both fields, x fastest, copied asynchronously so that
    // every element of the block is in flight at once
    for (int e = tid; e < nD; e += FILL_THREADS) {
      const int x = e % Dn[0], y = (e / Dn[0]) % Dn[1], z = e / (Dn[0] * Dn[1]);
      const double* src = S.D + S.gd.at(D0[0] + x, D0[1] + y, D0[2] + z);
      cp_async8(D + e, src);
      cp_async8(D + CAP_D + e, src + S.gd.vol);
    }
    cp_async_wait_all();
    if (A.fixed) {
      // largest exponent of each block, on the entries this thread copied
      int e0 = 0, e1 = 0;
      for (int e = tid; e < nD; e += FILL_THREADS) {
        e0 = max(e0, biased_exponent(D[e]));
        e1 = max(e1, biased_exponent(D[CAP_D + e]));
      }
      e0 = __reduce_max_sync(0xffffffffu, e0);
      e1 = __reduce_max_sync(0xffffffffu, e1);
      if ((tid & 31) == 0) {
        atomicMax(&s_E[0], e0);
        atomicMax(&s_E[1], e1);
      }
    }
    __syncthreads();
    for (int f = 0; f < 2; ++f) {
      double* Df = D + f * CAP_D;
      const int E = s_E[f];
      if (A.fixed && E < EXP_NONFINITE) {
        const int Eu = max(E, 64);
        int2* DQ = reinterpret_cast<int2*>(Df);
        // in place: every entry is read and rewritten by the same thread
        for (int e = tid; e < nD; e += FILL_THREADS) DQ[e] = split31(to_fixed(Df[e], Eu) * 64);
        __syncthreads();
        int2* R1Q = reinterpret_cast<int2*>(R1);
        int2* R2Q = reinterpret_cast<int2*>(R2);
        contract_fx<P, false>(DQ, R1Q, Dn, ord[0], T[ord[0]], WQ + ord[0] * MAXT * 6, WS + ord[0] * MAXT, D0[ord[0]]);
        __syncthreads();
        contract_fx<P, false>(R1Q, R2Q, d1, ord[1], T[ord[1]], WQ + ord[1] * MAXT * 6, WS + ord[1] * MAXT,
                              D0[ord[1]]);
        __syncthreads();
        contract_fx<P, true>(R2Q, Df, d2, ord[2], T[ord[2]], WQ + ord[2] * MAXT * 6, WS + ord[2] * MAXT,
                             D0[ord[2]]);
        __syncthreads();
        // results are on 2^(Eu - 1075 - 6): an exact power-of-two scaling
        const double p2 = __longlong_as_double((long long)(Eu - 58) << 52);
        const long long* DR = reinterpret_cast<const long long*>(Df);
        for (int e = tid; e < ntar; e += FILL_THREADS) {
          const int tx = e % T[0], ty = (e / T[0]) % T[1], tz = e / (T[0] * T[1]);
          const double v = (double)DR[e] * p2;
          S.T[S.gt.at(org[0] + tx, org[1] + ty, org[2] + tz) + f * S.gt.vol] = v;
          emax[f] = max(emax[f], biased_exponent(v));
        }
      } else {
        contract<P>(Df, R1, Dn, ord[0], T[ord[0]], W + ord[0] * MAXT * 6, WS + ord[0] * MAXT, D0[ord[0]]);
        __syncthreads();
        contract<P>(R1, R2, d1, ord[1], T[ord[1]], W + ord[1] * MAXT * 6, WS + ord[1] * MAXT, D0[ord[1]]);
        __syncthreads();
        contract<P>(R2, Df, d2, ord[2], T[ord[2]], W + ord[2] * MAXT * 6, WS + ord[2] * MAXT, D0[ord[2]]);
        __syncthreads();
        for (int e = tid; e < ntar; e += FILL_THREADS) {
          const int tx = e % T[0], ty = (e / T[0]) % T[1], tz = e / (T[0] * T[1]);
          const double v = Df[e];
          S.T[S.gt.at(org[0] + tx, org[1] + ty, org[2] + tz) + f * S.gt.vol] = v;
          emax[f] = max(emax[f], biased_exponent(v));
        }
      }
      // R1 and R2 are reused by the next field
      __syncthreads();
    }
  }
  report_block_max(A.expo + S.tpatch * EXP_SLOTS_PER_PATCH + A.y_buf * 2, emax[0], emax[1]);
}

}  // namespace

template <int P>
__global__ void __launch_bounds__(FILL_THREADS) k_fill(const __grid_constant__ FillArgs A) {
  extern __shared__ double fill_smem[];
  if (A.reset_buf >= 0 && blockIdx.x == 0 && threadIdx.x < 2 * A.np)
    A.expo[(threadIdx.x >> 1) * EXP_SLOTS_PER_PATCH + A.reset_buf * 2 + (threadIdx.x & 1)] = 0;
  const int b = blockIdx.x;
  if (b < A.outer_blocks) {
    // global outer ghost shell, one point per thread
    const long long idx = (long long)b * FILL_THREADS + threadIdx.x;
    int e0 = 0, e1 = 0;
    if (idx < A.outer_count) {
      const int O[3] = {A.gg.n[0] + 2 * NG, A.gg.n[1] + 2 * NG, A.gg.n[2] + 2 * NG};
      int x, y, z;
      shell_point(idx, O, NG, x, y, z);
      const int i = x - NG, j = y - NG, k = z - NG;
      const long long c = A.gg.at(i, j, k);
      double w0, w1;
      if (A.outer_bc == 1) {
        const long long s =
            A.gg.at(wrap_index(i, A.gg.n[0]), wrap_index(j, A.gg.n[1]), wrap_index(k, A.gg.n[2]));
        w0 = A.Yg[s];
        w1 = A.Yg[s + A.gg.vol];
      } else if (A.shell_src) {
        // the closed form at this very time already sits in another buffer's shell
        w0 = A.shell_src[c];
        w1 = A.shell_src[c + A.gg.vol];
      } else {
        closed_form(A.akind, A.aparams, A.ascreen, A.apre, A.acount, A.t, A.gg.lo[0] + (i + 0.5) * A.gg.h[0],
                    A.gg.lo[1] + (j + 0.5) * A.gg.h[1], A.gg.lo[2] + (k + 0.5) * A.gg.h[2], w0, w1);
      }
      A.Yg[c] = w0;
      A.Yg[c + A.gg.vol] = w1;
      e0 = biased_exponent(w0);
      e1 = biased_exponent(w1);
    }
    report_block_max(A.expo + A.y_buf * 2, e0, e1);
    return;
  }
  // interpolation tile: find its segment, slab and position
  int s = 0;
  while (s + 1 < A.nseg && b >= A.seg[s + 1].block0) ++s;
  const InterpSeg& S = A.seg[s];
  int r = b - S.block0;
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
  interp_tile<P>(A, S, org, T, fill_smem);
}

void launch_fill(const FillArgs& a, void* stream) {
  if (a.total_blocks <= 0) return;
  if (a.P == 6) {
    cudaFuncSetAttribute(k_fill<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FILL_SMEM);
    k_fill<6><<<a.total_blocks, FILL_THREADS, FILL_SMEM, (cudaStream_t)stream>>>(a);
  } else {
    cudaFuncSetAttribute(k_fill<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FILL_SMEM);
    k_fill<5><<<a.total_blocks, FILL_THREADS, FILL_SMEM, (cudaStream_t)stream>>>(a);
  }
}

int fill_cap_d() { return CAP_D; }
int fill_cap_r1() { return CAP_R1; }
int fill_cap_r2() { return CAP_R2; }
int fill_max_tile() { return MAXT; }
int fill_threads() { return FILL_THREADS; }

}  // namespace mpw
