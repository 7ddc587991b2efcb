// mpw_kernels.cu -- CUDA kernels of libmpw (sm_103a): ghost-zone fill
// (analytic / periodic outer BC, Local-to-Global, Global-to-Local), cover
// flags with buffer, the native-FP64 fused RHS + RK4 stage kernel, and the
// pack / unpack / closed-form helpers behind the C ABI.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

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
template <int P>
__global__ void __launch_bounds__(256) k_fill(const __grid_constant__ FillArgs A) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < A.total; idx += stride) {
    if (idx < A.outer_count) {
      const int O[3] = {A.gg.n[0] + 2 * NG, A.gg.n[1] + 2 * NG, A.gg.n[2] + 2 * NG};
      int x, y, z;
      shell_point(idx, O, NG, x, y, z);
      const int i = x - NG, j = y - NG, k = z - NG;
      const long long c = A.gg.at(i, j, k);
      if (A.outer_bc == 1) {
        const long long s =
            A.gg.at(wrap_index(i, A.gg.n[0]), wrap_index(j, A.gg.n[1]), wrap_index(k, A.gg.n[2]));
        A.Yg[c] = A.Yg[s];
        A.Yg[c + A.gg.vol] = A.Yg[s + A.gg.vol];
      } else {
        double ps, pv;
        closed_form(A.akind, A.aparams, A.acount, A.t, A.gg.lo[0] + (i + 0.5) * A.gg.h[0],
                    A.gg.lo[1] + (j + 0.5) * A.gg.h[1], A.gg.lo[2] + (k + 0.5) * A.gg.h[2], ps, pv);
        A.Yg[c] = ps;
        A.Yg[c + A.gg.vol] = pv;
      }
      continue;
    }
    for (int q = 0; q < A.nloc; ++q) {
      const FillLocal& L = A.loc[q];
      if (idx >= L.l2g_begin && idx < L.l2g_begin + L.l2g_count) {
        int x, y, z;
        shell_point(idx - L.l2g_begin, L.shell_dim, NG, x, y, z);
        const int i = L.shell_lo[0] + x, j = L.shell_lo[1] + y, k = L.shell_lo[2] + z;
        const uint8_t f = A.flags[((long long)k * A.gg.n[1] + j) * A.gg.n[0] + i];
        if ((f & 3) != FLAG_GHOST || (f >> 2) != q + 1) {
          atomicOr(A.err, ERR_BOUNDS);
          break;
        }
        double v0, v1;
        const bool ok = interp<P>(L.Y, L.g, A.gg.lo[0] + (i + 0.5) * A.gg.h[0] - L.X0[0],
                                  A.gg.lo[1] + (j + 0.5) * A.gg.h[1] - L.X0[1],
                                  A.gg.lo[2] + (k + 0.5) * A.gg.h[2] - L.X0[2], v0, v1);
        if (!ok) {
          atomicOr(A.err, ERR_UNFILLED);
          break;
        }
        const long long c = A.gg.at(i, j, k);
        A.Yg[c] = v0;
        A.Yg[c + A.gg.vol] = v1;
        break;
      }
      if (idx >= L.g2l_begin && idx < L.g2l_begin + L.g2l_count) {
        const int O[3] = {L.g.n[0] + 2 * NG, L.g.n[1] + 2 * NG, L.g.n[2] + 2 * NG};
        int x, y, z;
        shell_point(idx - L.g2l_begin, O, NG, x, y, z);
        const int i = x - NG, j = y - NG, k = z - NG;
        double v0, v1;
        const bool ok = interp<P>(A.Yg, A.gg, L.g.lo[0] + (i + 0.5) * L.g.h[0] + L.X0[0],
                                  L.g.lo[1] + (j + 0.5) * L.g.h[1] + L.X0[1],
                                  L.g.lo[2] + (k + 0.5) * L.g.h[2] + L.X0[2], v0, v1);
        if (!ok) {
          atomicOr(A.err, ERR_UNFILLED);
          break;
        }
        const long long c = L.g.at(i, j, k);
        L.Y[c] = v0;
        L.Y[c + L.g.vol] = v1;
        break;
      }
    }
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
// Native FP64 fused RHS + RK4 stage (reference GPU path; Sec. 2.2-2.3).
// One CTA owns a TX x TY column tile and marches a chunk of zc planes: the z
// neighbours of its own column sit in a 7-deep register queue, the x/y
// neighbours of the current plane in shared memory (halo 3, star stencil).
template <int TX, int TY>
__global__ void __launch_bounds__(TX* TY) k_rhs_fp64(const __grid_constant__ RhsArgs A) {
  __shared__ double sm[2][TY + 6][TX + 6];
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
  const double* Ys = Pt.Y;
  const double* Yp = Pt.Y + g.vol;
  double qs[7], qp[7];
#pragma unroll
  for (int o = 0; o < 6; ++o) {
    qs[o] = 0.0;
    qp[o] = 0.0;
    if (in_box) {
      const long long c = g.at(i, j, z0 - NG + o);
      qs[o] = Ys[c];
      qp[o] = Yp[c];
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
  const double c2x = Pt.c2[0], c2y = Pt.c2[1], c2z = Pt.c2[2];
  const double kx = Pt.cko[0], ky = Pt.cko[1], kz = Pt.cko[2];
  const double c1x = Pt.c1[0], c1y = Pt.c1[1], c1z = Pt.c1[2];
  constexpr int SY = TX + 6;
  for (int z = z0; z < z1; ++z) {
    if (in_box) {
      const long long c = g.at(i, j, z + NG);
      qs[6] = Ys[c];
      qp[6] = Yp[c];
    }
    __syncthreads();
    sm[0][lj + 3][li + 3] = qs[3];
    sm[1][lj + 3][li + 3] = qp[3];
    if (h_ok) {
      const long long c = g.at(hi_, hj, z);
      sm[0][hsj][hsi] = Ys[c];
      sm[1][hsj][hsi] = Yp[c];
    }
    __syncthreads();
    bool live = in_xy;
    if (live && check_flags) {
      const int f = A.flags[((long long)z * g.n[1] + j) * g.n[0] + i] & 3;
      live = (f == FLAG_LIVE) || (f == FLAG_REVIVED);
    }
    if (live) {
      const double* rs = &sm[0][lj + 3][li + 3];
      const double* rp = &sm[1][lj + 3][li + 3];
      const double u0 = qs[3], v0 = qp[3];
      const double xs1 = rs[-1] + rs[1], xs2 = rs[-2] + rs[2], xs3 = rs[-3] + rs[3];
      const double ys1 = rs[-SY] + rs[SY], ys2 = rs[-2 * SY] + rs[2 * SY], ys3 = rs[-3 * SY] + rs[3 * SY];
      const double zs1 = qs[2] + qs[4], zs2 = qs[1] + qs[5], zs3 = qs[0] + qs[6];
      const double xp1 = rp[-1] + rp[1], xp2 = rp[-2] + rp[2], xp3 = rp[-3] + rp[3];
      const double yp1 = rp[-SY] + rp[SY], yp2 = rp[-2 * SY] + rp[2 * SY], yp3 = rp[-3 * SY] + rp[3 * SY];
      const double zp1 = qp[2] + qp[4], zp2 = qp[1] + qp[5], zp3 = qp[0] + qp[6];
      const double d2 = c2x * (16.0 * xs1 - xs2 - 30.0 * u0) + c2y * (16.0 * ys1 - ys2 - 30.0 * u0) +
                        c2z * (16.0 * zs1 - zs2 - 30.0 * u0);
      const double kos = kx * (xs3 - 6.0 * xs2 + 15.0 * xs1 - 20.0 * u0) +
                         ky * (ys3 - 6.0 * ys2 + 15.0 * ys1 - 20.0 * u0) +
                         kz * (zs3 - 6.0 * zs2 + 15.0 * zs1 - 20.0 * u0);
      const double kop = kx * (xp3 - 6.0 * xp2 + 15.0 * xp1 - 20.0 * v0) +
                         ky * (yp3 - 6.0 * yp2 + 15.0 * yp1 - 20.0 * v0) +
                         kz * (zp3 - 6.0 * zp2 + 15.0 * zp1 - 20.0 * v0);
      double Ks = v0 + kos, Kp = d2 + kop;
      if (Pt.moving) {
        Ks += c1x * (8.0 * (rs[1] - rs[-1]) - (rs[2] - rs[-2])) +
              c1y * (8.0 * (rs[SY] - rs[-SY]) - (rs[2 * SY] - rs[-2 * SY])) +
              c1z * (8.0 * (qs[4] - qs[2]) - (qs[5] - qs[1]));
        Kp += c1x * (8.0 * (rp[1] - rp[-1]) - (rp[2] - rp[-2])) +
              c1y * (8.0 * (rp[SY] - rp[-SY]) - (rp[2 * SY] - rp[-2 * SY])) +
              c1z * (8.0 * (qp[4] - qp[2]) - (qp[5] - qp[1]));
      }
      const long long c = g.at(i, j, z);
      if (A.stage == 3) {
        Pt.OUT[c] = fma(A.alpha, Ks, Pt.ACC[c]);
        Pt.OUT[c + g.vol] = fma(A.alpha, Kp, Pt.ACC[c + g.vol]);
      } else {
        const double us = A.stage == 0 ? u0 : Pt.U[c];
        const double up = A.stage == 0 ? v0 : Pt.U[c + g.vol];
        const double as = A.stage == 0 ? u0 : Pt.ACC[c];
        const double ap = A.stage == 0 ? v0 : Pt.ACC[c + g.vol];
        Pt.OUT[c] = fma(A.alpha, Ks, us);
        Pt.OUT[c + g.vol] = fma(A.alpha, Kp, up);
        Pt.ACC[c] = fma(A.beta, Ks, as);
        Pt.ACC[c + g.vol] = fma(A.beta, Kp, ap);
      }
    }
#pragma unroll
    for (int o = 0; o < 6; ++o) {
      qs[o] = qs[o + 1];
      qp[o] = qp[o + 1];
    }
  }
}

void launch_rhs_fp64(const RhsArgs& a, int blocks, void* stream) {
  k_rhs_fp64<RHS_TX, RHS_TY><<<blocks, RHS_TX * RHS_TY, 0, (cudaStream_t)stream>>>(a);
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
