// mpw_kernels.cu -- CUDA kernels of libmpw (sm_103a): ghost-zone fill
// (analytic / periodic outer BC, Local-to-Global, Global-to-Local), cover
// flags with buffer, the native-FP64 fused RHS + RK4 stage kernel, and the
// pack / unpack / closed-form helpers behind the C ABI.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "mpw_fixed.cuh"
#include "mpw_internal.cuh"

namespace mpw {

// ---------------------------------------------------------------------------
// Closed forms (Sec. 3): spherical Gaussian pulse pairs, plane-wave sums and
// the static harmonic basis.  psi = [g(t+r) - g(t-r)] / (2r) with
// g(s) = A s exp(-s^2/w^2) solves the wave equation with psi(0) = A
// exp(-r^2/w^2), Pi(0) = 0; Pi is its time derivative.  Near r = 0 the
// quotient is replaced by its Taylor expansion g'(t) + r^2 g'''(t)/6.
__device__ __forceinline__ void gauss_pulse(double A, double w, double r, double t, double& ps, double& pv) {
  const double a = 1.0 / (w * w);
  if (r < 1e-5) {
    const double e = A * exp(-a * t * t), t2 = t * t;
    const double g1 = e * (1.0 - 2.0 * a * t2);
    const double g2 = e * (4.0 * a * a * t2 * t - 6.0 * a * t);
    const double g3 = e * (-6.0 * a + 24.0 * a * a * t2 - 8.0 * a * a * a * t2 * t2);
    const double g4 = e * (60.0 * a * a * t - 80.0 * a * a * a * t2 * t + 16.0 * a * a * a * a * t2 * t2 * t);
    ps += g1 + r * r * g3 / 6.0;
    pv += g2 + r * r * g4 / 6.0;
  } else {
    const double sp = t + r, sm = t - r;
    const double ep = A * exp(-a * sp * sp), em = A * exp(-a * sm * sm);
    const double inv = 1.0 / (2.0 * r);
    ps += (ep * sp - em * sm) * inv;
    pv += (ep * (1.0 - 2.0 * a * sp * sp) - em * (1.0 - 2.0 * a * sm * sm)) * inv;
  }
}

__device__ void closed_form(int kind, const double* __restrict__ P, int count, double t, double x, double y,
                            double z, double& ps, double& pv) {
  ps = 0.0;
  pv = 0.0;
  if (kind == 0) {
    for (int q = 0; q < count; ++q) {
      const double* g = P + 5 * q;
      const double dx = x - g[2], dy = y - g[3], dz = z - g[4];
      gauss_pulse(g[0], g[1], sqrt(dx * dx + dy * dy + dz * dz), t, ps, pv);
    }
  } else if (kind == 1) {
    ps = P[0];
    for (int q = 0; q < count; ++q) {
      const double* wv = P + 1 + 5 * q;
      const double kk = sqrt(wv[1] * wv[1] + wv[2] * wv[2] + wv[3] * wv[3]);
      double sn, cs;
      sincos(wv[1] * x + wv[2] * y + wv[3] * z - kk * t + wv[4], &sn, &cs);
      ps += wv[0] * sn;
      pv -= wv[0] * kk * cs;
    }
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
template <int P>
__device__ bool interp_point(const double* __restrict__ src, const Geom& g, double x, double y, double z,
                             double& o0, double& o1) {
  double wx[P], wy[P], wz[P];
  const int sx = lagrange_weights<P>((x - g.lo[0]) / g.h[0] - 0.5, wx);
  const int sy = lagrange_weights<P>((y - g.lo[1]) / g.h[1] - 0.5, wy);
  const int sz = lagrange_weights<P>((z - g.lo[2]) / g.h[2] - 0.5, wz);
  if (sx < 0 || sy < 0 || sz < 0 || sx + P > g.n[0] || sy + P > g.n[1] || sz + P > g.n[2]) return false;
  const double* s0 = src;
  const double* s1 = src + g.vol;
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
        r0 = fma(wx[a], s0[row + a], r0);
        r1 = fma(wx[a], s1[row + a], r1);
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

template <int P>
__device__ __forceinline__ bool interp(const double* src, const Geom& g, double x, double y, double z, double& o0,
                                       double& o1) {
  return interp_point<P>(src, g, x, y, z, o0, o1);
}

// Maps idx in [0, Ox*Oy*Oz - Ix*Iy*Iz) onto the points of the hollow box of
// outer extent O whose walls are th thick (I = max(O - 2 th, 0)).
__device__ __forceinline__ void shell_point(long long idx, const int O[3], int th, int& x, int& y, int& z) {
  const int Ix = max(O[0] - 2 * th, 0), Iy = max(O[1] - 2 * th, 0), Iz = max(O[2] - 2 * th, 0);
  const long long pxy = (long long)O[0] * O[1];
  const long long nz = pxy * (O[2] - Iz);
  if (idx < nz) {
    const int zs = (int)(idx / pxy);
    const long long r = idx - (long long)zs * pxy;
    z = zs < th ? zs : zs + Iz;
    y = (int)(r / O[0]);
    x = (int)(r - (long long)y * O[0]);
    return;
  }
  idx -= nz;
  const long long rowsy = (long long)O[0] * (O[1] - Iy);
  const long long ny = rowsy * Iz;
  if (idx < ny) {
    const int zz = (int)(idx / rowsy);
    const long long r = idx - (long long)zz * rowsy;
    z = th + zz;
    const int ys = (int)(r / O[0]);
    x = (int)(r - (long long)ys * O[0]);
    y = ys < th ? ys : ys + Iy;
    return;
  }
  idx -= ny;
  const int wx = O[0] - Ix;
  const long long per_z = (long long)wx * Iy;
  const int zz = (int)(idx / per_z);
  const long long r = idx - (long long)zz * per_z;
  z = th + zz;
  const int yy = (int)(r / wx);
  const int xs = (int)(r - (long long)yy * wx);
  y = th + yy;
  x = xs < th ? xs : xs + Ix;
}

__device__ __forceinline__ int wrap_index(int i, int n) { return ((i % n) + n) % n; }

// ---------------------------------------------------------------------------
// Ghost-zone fill of one substage (Sec. 2.4): global outer shell (analytic or
// periodic), Local-to-Global into the global effective ghost cells,
// Global-to-Local into every local ghost shell.  The three target sets are
// disjoint and each reads only data the others do not write (the buffer makes
// every interpolation donor a live cell), so they run as one launch.
// Warp-aggregated atomicMax of the exponents written by each lane into the
// exponent slots of the patch it wrote (patch < 0: nothing written).
__device__ __forceinline__ void report_exponents(int* expo, int buf, int patch, double v0, double v1) {
  const unsigned mask = __activemask();
  const unsigned peers = __match_any_sync(mask, patch);
  const int e0 = __reduce_max_sync(peers, patch >= 0 ? biased_exponent(v0) : 0);
  const int e1 = __reduce_max_sync(peers, patch >= 0 ? biased_exponent(v1) : 0);
  if (patch >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) {
    atomicMax(&expo[patch * EXP_SLOTS_PER_PATCH + buf * 2], e0);
    atomicMax(&expo[patch * EXP_SLOTS_PER_PATCH + buf * 2 + 1], e1);
  }
}

// Global outer ghost shell point idx: analytic closed form or periodic wrap.
__device__ __forceinline__ void fill_outer(const FillArgs& A, long long idx, double& w0, double& w1) {
  const int O[3] = {A.gg.n[0] + 2 * NG, A.gg.n[1] + 2 * NG, A.gg.n[2] + 2 * NG};
  int x, y, z;
  shell_point(idx, O, NG, x, y, z);
  const int i = x - NG, j = y - NG, k = z - NG;
  const long long c = A.gg.at(i, j, k);
  if (A.outer_bc == 1) {
    const long long s = A.gg.at(wrap_index(i, A.gg.n[0]), wrap_index(j, A.gg.n[1]), wrap_index(k, A.gg.n[2]));
    w0 = A.Yg[s];
    w1 = A.Yg[s + A.gg.vol];
  } else {
    closed_form(A.akind, A.aparams, A.acount, A.t, A.gg.lo[0] + (i + 0.5) * A.gg.h[0],
                A.gg.lo[1] + (j + 0.5) * A.gg.h[1], A.gg.lo[2] + (k + 0.5) * A.gg.h[2], w0, w1);
  }
  A.Yg[c] = w0;
  A.Yg[c + A.gg.vol] = w1;
}

// Local-to-Global (Sec. 2.4.2): effective ghost cell number r of the shell
// under local patch q, interpolated from q at the substage time.
template <int P>
__device__ __forceinline__ bool fill_l2g(const FillArgs& A, int q, long long r, double& w0, double& w1) {
  const FillLocal& L = A.loc[q];
  int x, y, z;
  shell_point(r, L.shell_dim, NG, x, y, z);
  const int i = L.shell_lo[0] + x, j = L.shell_lo[1] + y, k = L.shell_lo[2] + z;
  const uint8_t f = A.flags[((long long)k * A.gg.n[1] + j) * A.gg.n[0] + i];
  if ((f & 3) != FLAG_GHOST || (f >> 2) != q + 1) {
    atomicOr(A.err, ERR_BOUNDS);
    return false;
  }
  if (!interp<P>(L.Y, L.g, A.gg.lo[0] + (i + 0.5) * A.gg.h[0] - L.X0[0],
                 A.gg.lo[1] + (j + 0.5) * A.gg.h[1] - L.X0[1], A.gg.lo[2] + (k + 0.5) * A.gg.h[2] - L.X0[2], w0,
                 w1)) {
    atomicOr(A.err, ERR_UNFILLED);
    return false;
  }
  const long long c = A.gg.at(i, j, k);
  A.Yg[c] = w0;
  A.Yg[c + A.gg.vol] = w1;
  return true;
}

// Global-to-Local (Sec. 2.4.1): ghost point number r of local patch q,
// interpolated from the global patch at the substage time.
template <int P>
__device__ __forceinline__ bool fill_g2l(const FillArgs& A, int q, long long r, double& w0, double& w1) {
  const FillLocal& L = A.loc[q];
  const int O[3] = {L.g.n[0] + 2 * NG, L.g.n[1] + 2 * NG, L.g.n[2] + 2 * NG};
  int x, y, z;
  shell_point(r, O, NG, x, y, z);
  const int i = x - NG, j = y - NG, k = z - NG;
  if (!interp<P>(A.Yg, A.gg, L.g.lo[0] + (i + 0.5) * L.g.h[0] + L.X0[0], L.g.lo[1] + (j + 0.5) * L.g.h[1] + L.X0[1],
                 L.g.lo[2] + (k + 0.5) * L.g.h[2] + L.X0[2], w0, w1)) {
    atomicOr(A.err, ERR_UNFILLED);
    return false;
  }
  const long long c = L.g.at(i, j, k);
  L.Y[c] = w0;
  L.Y[c + L.g.vol] = w1;
  return true;
}

// Ghost-zone fill of one substage (Sec. 2.4): global outer shell, then the
// Local-to-Global segments, then the Global-to-Local segments, as consecutive
// ranges of one index space.  The target sets are disjoint and each reads only
// data the others do not write (the buffer makes every interpolation donor a
// live cell), so one launch serves them all.  Block 0 also clears the
// exponent slots of the buffer the next RHS launch will write.
template <int P>
__global__ void __launch_bounds__(256) k_fill(const __grid_constant__ FillArgs A) {
  if (A.reset_buf >= 0 && blockIdx.x == 0 && threadIdx.x < 2 * A.np)
    A.expo[(threadIdx.x >> 1) * EXP_SLOTS_PER_PATCH + A.reset_buf * 2 + (threadIdx.x & 1)] = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < A.total; idx += stride) {
    int wrote = -1;
    double w0 = 0.0, w1 = 0.0;
    if (idx < A.outer_count) {
      fill_outer(A, idx, w0, w1);
      wrote = 0;
    } else {
      for (int q = 0; q < A.nloc; ++q) {
        const FillLocal& L = A.loc[q];
        if (idx >= L.l2g_begin && idx < L.l2g_begin + L.l2g_count) {
          if (fill_l2g<P>(A, q, idx - L.l2g_begin, w0, w1)) wrote = 0;
          break;
        }
        if (idx >= L.g2l_begin && idx < L.g2l_begin + L.g2l_count) {
          if (fill_g2l<P>(A, q, idx - L.g2l_begin, w0, w1)) wrote = q + 1;
          break;
        }
      }
    }
    report_exponents(A.expo, A.y_buf, wrote, w0, w1);
  }
}

void launch_fill(const FillArgs& a, void* stream) {
  if (a.total <= 0) return;
  long long blocks = (a.total + 255) / 256;
  if (blocks > 152LL * 16) blocks = 152LL * 16;
  if (a.P == 6)
    k_fill<6><<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(a);
  else
    k_fill<5><<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(a);
}

// ---------------------------------------------------------------------------
// Cover flags with buffer (Sec. 2.4.2), from the covered box of every local
// patch at t_n.  A covered cell's L-infinity distance to the nearest
// uncovered cell is min over axes of its distance to the box faces; LIVE if
// d <= buffer, GHOST if d <= buffer + NG, DEAD beyond.  DEAD cells of u are
// poisoned with NaN; cells that turn LIVE after having been GHOST or DEAD are
// REVIVED: u_n there is interpolated from the owning local patch at t_n.
template <int P>
__global__ void __launch_bounds__(256) k_flags(const __grid_constant__ FlagArgs A) {
  const long long N = (long long)A.n[0] * A.n[1] * A.n[2];
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= N) return;
  const int i = (int)(idx % A.n[0]);
  const long long r = idx / A.n[0];
  const int j = (int)(r % A.n[1]);
  const int k = (int)(r / A.n[1]);
  int owner = 0, d = 0;
  for (int q = 0; q < A.nloc; ++q) {
    const Box& b = A.box[q];
    if (i >= b.lo[0] && i <= b.hi[0] && j >= b.lo[1] && j <= b.hi[1] && k >= b.lo[2] && k <= b.hi[2]) {
      owner = q + 1;
      d = min(min(min(i - b.lo[0], b.hi[0] - i), min(j - b.lo[1], b.hi[1] - j)), min(k - b.lo[2], b.hi[2] - k)) + 1;
      break;
    }
  }
  int st = (owner == 0 || d <= A.buffer) ? FLAG_LIVE : (d <= A.buffer + NG ? FLAG_GHOST : FLAG_DEAD);
  if (A.old_valid && st == FLAG_LIVE) {
    const int os = A.flags[idx] & 3;
    if (os == FLAG_GHOST || os == FLAG_DEAD) st = FLAG_REVIVED;
  }
  A.flags[idx] = (uint8_t)(st | (owner << 2));
  const long long c = A.gg.at(i, j, k);
  if (st == FLAG_DEAD) {
    A.Ug[c] = __longlong_as_double(0x7ff8000000000000LL);
    A.Ug[c + A.gg.vol] = __longlong_as_double(0x7ff8000000000000LL);
  } else if (st == FLAG_REVIVED) {
    const int q = owner - 1;
    double v0, v1;
    const bool ok = interp<P>(A.Uloc[q], A.gl[q], A.gg.lo[0] + (i + 0.5) * A.gg.h[0] - A.X0[q][0],
                              A.gg.lo[1] + (j + 0.5) * A.gg.h[1] - A.X0[q][1],
                              A.gg.lo[2] + (k + 0.5) * A.gg.h[2] - A.X0[q][2], v0, v1);
    if (!ok) {
      atomicOr(A.err, ERR_UNFILLED);
      return;
    }
    A.Ug[c] = v0;
    A.Ug[c + A.gg.vol] = v1;
    atomicMax(&A.expo[BUF_U * 2], biased_exponent(v0));
    atomicMax(&A.expo[BUF_U * 2 + 1], biased_exponent(v1));
  }
}

void launch_flags(const FlagArgs& a, void* stream) {
  const long long N = (long long)a.n[0] * a.n[1] * a.n[2];
  const unsigned blocks = (unsigned)((N + 255) / 256);
  if (a.P == 6)
    k_flags<6><<<blocks, 256, 0, (cudaStream_t)stream>>>(a);
  else
    k_flags<5><<<blocks, 256, 0, (cudaStream_t)stream>>>(a);
}

// ---------------------------------------------------------------------------
// Interior <- closed form at time t (positions X_B = numeric + X0).
__global__ void k_analytic(double* buf, const Geom g, double X0x, double X0y, double X0z, int akind, int acount,
                           const double* __restrict__ P, double t) {
  const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= N) return;
  const int i = (int)(idx % g.n[0]);
  const long long r = idx / g.n[0];
  const int j = (int)(r % g.n[1]);
  const int k = (int)(r / g.n[1]);
  double ps, pv;
  closed_form(akind, P, acount, t, g.lo[0] + (i + 0.5) * g.h[0] + X0x, g.lo[1] + (j + 0.5) * g.h[1] + X0y,
              g.lo[2] + (k + 0.5) * g.h[2] + X0z, ps, pv);
  const long long c = g.at(i, j, k);
  buf[c] = ps;
  buf[c + g.vol] = pv;
}

void launch_analytic(double* buf, const Geom& g, double X0x, double X0y, double X0z, int akind, int acount,
                     const double* aparams, double t, void* stream) {
  const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
  k_analytic<<<(unsigned)((N + 255) / 256), 256, 0, (cudaStream_t)stream>>>(buf, g, X0x, X0y, X0z, akind, acount,
                                                                            aparams, t);
}

// Padded buffer -> dense array (interior, or the whole padded box).  With
// flags, global cells that are not live read as NaN.
__global__ void k_pack(const double* __restrict__ buf, const Geom g, double* __restrict__ d0,
                       double* __restrict__ d1, int padded, const uint8_t* __restrict__ flags) {
  const int e = padded ? 2 * NG : 0, o = padded ? NG : 0;
  const int m0 = g.n[0] + e, m1 = g.n[1] + e, m2 = g.n[2] + e;
  const long long N = (long long)m0 * m1 * m2;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= N) return;
  const int i = (int)(idx % m0) - o;
  const long long r = idx / m0;
  const int j = (int)(r % m1) - o;
  const int k = (int)(r / m1) - o;
  const long long c = g.at(i, j, k);
  double v0 = buf[c], v1 = buf[c + g.vol];
  if (flags) {
    const int f = flags[((long long)k * g.n[1] + j) * g.n[0] + i] & 3;
    if (f == FLAG_GHOST || f == FLAG_DEAD) v0 = v1 = __longlong_as_double(0x7ff8000000000000LL);
  }
  d0[idx] = v0;
  d1[idx] = v1;
}

void launch_pack(const double* buf, const Geom& g, double* d0, double* d1, int padded, const uint8_t* flags,
                 void* stream) {
  const int e = padded ? 2 * NG : 0;
  const long long N = (long long)(g.n[0] + e) * (g.n[1] + e) * (g.n[2] + e);
  k_pack<<<(unsigned)((N + 255) / 256), 256, 0, (cudaStream_t)stream>>>(buf, g, d0, d1, padded,
                                                                        padded ? nullptr : flags);
}

__global__ void k_unpack(double* buf, const Geom g, const double* __restrict__ d0, const double* __restrict__ d1) {
  const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= N) return;
  const int i = (int)(idx % g.n[0]);
  const long long r = idx / g.n[0];
  const int j = (int)(r % g.n[1]);
  const int k = (int)(r / g.n[1]);
  const long long c = g.at(i, j, k);
  buf[c] = d0[idx];
  buf[c + g.vol] = d1[idx];
}

void launch_unpack(double* buf, const Geom& g, const double* d0, const double* d1, void* stream) {
  const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
  k_unpack<<<(unsigned)((N + 255) / 256), 256, 0, (cudaStream_t)stream>>>(buf, g, d0, d1);
}

}  // namespace mpw

namespace mpw {

// Largest biased exponent of the live interior values of a buffer (both
// fields), for buffers written from outside the step (set_fields,
// fill_analytic).  slot2 points at the two slots of the buffer.
__global__ void k_expo_scan(const double* __restrict__ buf, const Geom g, const uint8_t* __restrict__ flags,
                            int* slot2) {
  const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
  int e0 = 0, e1 = 0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < N;
       idx += (long long)gridDim.x * blockDim.x) {
    if (flags) {
      const int f = flags[idx] & 3;
      if (f == FLAG_GHOST || f == FLAG_DEAD) continue;
    }
    const int i = (int)(idx % g.n[0]);
    const long long r = idx / g.n[0];
    const int j = (int)(r % g.n[1]);
    const int k = (int)(r / g.n[1]);
    const long long c = g.at(i, j, k);
    e0 = max(e0, biased_exponent(buf[c]));
    e1 = max(e1, biased_exponent(buf[c + g.vol]));
  }
  e0 = __reduce_max_sync(0xffffffffu, e0);
  e1 = __reduce_max_sync(0xffffffffu, e1);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&slot2[0], e0);
    atomicMax(&slot2[1], e1);
  }
}

void launch_expo_scan(const double* buf, const Geom& g, const uint8_t* flags, int* slot2, void* stream) {
  const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
  long long blocks = (N + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_expo_scan<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(buf, g, flags, slot2);
}

}  // namespace mpw
