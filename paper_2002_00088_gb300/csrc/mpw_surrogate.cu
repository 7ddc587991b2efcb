// mpw_surrogate.cu -- the learned surrogate of include/mpw_surrogate.h: the
// four-layer network's trainer (forward, squared-error loss, backward, Adam)
// and inference, and the kernels that turn FP64 wave fields into the
// network's features, its training targets and, from its output, the state
// four RK4 steps later.
//
// The FP64 arithmetic of the feature, target and update kernels uses
// explicitly rounded operations (no contraction into fused multiply-adds), in
// the order the header states, so that every value is defined to the bit.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/mpw_surrogate.h"
#include "mpw_fixed.cuh"
#include "mpw_internal.cuh"

namespace {

using mpw::set_last_error;

// layer table: padded channel counts, activation, parameter offsets
struct Layer {
  int cin, cout, relu;
  long long w, b;
};
constexpr int NLAYER = 4;
constexpr int CIN[NLAYER] = {8, 32, 32, 32};
constexpr int COUT[NLAYER] = {32, 32, 32, 8};

long long layer_table(Layer L[NLAYER]) {
  long long off = 0;
  for (int l = 0; l < NLAYER; ++l) {
    L[l].cin = CIN[l];
    L[l].cout = COUT[l];
    L[l].relu = l < NLAYER - 1;
    L[l].w = off;
    off += (long long)COUT[l] * 27 * CIN[l];
    L[l].b = off;
    off += COUT[l];
  }
  return off;
}

mpw_status fail(mpw_status st, const char* msg) {
  set_last_error(msg);
  return st;
}

mpw_status cuda_fail(cudaError_t e) {
  static thread_local char buf[160];
  std::snprintf(buf, sizeof(buf), "CUDA error: %s", cudaGetErrorString(e));
  set_last_error(buf);
  return MPW_ERR_CUDA;
}

#define SUR_TRY(x)                                    \
  do {                                                \
    cudaError_t e_ = (x);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_);      \
  } while (0)

#define MPW_TRY(x)                                    \
  do {                                                \
    mpw_status s_ = (x);                              \
    if (s_ != MPW_OK) return s_;                      \
  } while (0)

struct Dims {
  int n0, n1, n2, batch;
  __host__ __device__ long long points() const { return (long long)n0 * n1 * n2; }
};

// ---------------------------------------------------------------- kernels

// 16 x, exactly as __dmul_rn(16.0, x): where x is normal and 16 x stays
// finite, the biased exponent is raised by 4 (an integer add, not an FP64
// operation); zeros, subnormals, infinities and NaNs take the multiply.
__device__ __forceinline__ double times16(double x) {
  const int hi = __double2hiint(x);
  const unsigned e = ((unsigned)hi >> 20) & 0x7ffu;
  return e - 1u < 2042u ? __hiloint2double(hi + (4 << 20), __double2loint(x)) : __dmul_rn(16.0, x);
}

// 12 h^2 L u along one axis: (16 (u[-1] + u[1]) - (u[-2] + u[2])) - 30 u,
// with t30 = 30 u (the same for the three axes)
__device__ __forceinline__ double axis_sum(double um2, double um1, double t30, double up1, double up2) {
  return __dsub_rn(__dsub_rn(times16(__dadd_rn(um1, up1)), __dadd_rn(um2, up2)), t30);
}

// L u at (i, j, k) of sample volume u (periodic): ((Sx + Sy) + Sz) / (12 h^2).
// Offsets within a sample fit in 32 bits (n0 n1 n2 < 2^31).
__device__ __forceinline__ double lap4(const double* __restrict__ u, const Dims& d, int i, int j, int k,
                                       double inv12h2) {
  const int n0 = d.n0, pl = d.n0 * d.n1;
  const int c0 = (k * d.n1 + j) * n0 + i;
  const double t30 = __dmul_rn(30.0, __ldg(u + c0));
  const int xm1 = i >= 1 ? -1 : n0 - 1, xm2 = i >= 2 ? -2 : n0 - 2;
  const int xp1 = i + 1 < n0 ? 1 : 1 - n0, xp2 = i + 2 < n0 ? 2 : 2 - n0;
  const int ym1 = (j >= 1 ? -1 : d.n1 - 1) * n0, ym2 = (j >= 2 ? -2 : d.n1 - 2) * n0;
  const int yp1 = (j + 1 < d.n1 ? 1 : 1 - d.n1) * n0, yp2 = (j + 2 < d.n1 ? 2 : 2 - d.n1) * n0;
  const int zm1 = (k >= 1 ? -1 : d.n2 - 1) * pl, zm2 = (k >= 2 ? -2 : d.n2 - 2) * pl;
  const int zp1 = (k + 1 < d.n2 ? 1 : 1 - d.n2) * pl, zp2 = (k + 2 < d.n2 ? 2 : 2 - d.n2) * pl;
  const double* q = u + c0;
  const double sx = axis_sum(__ldg(q + xm2), __ldg(q + xm1), t30, __ldg(q + xp1), __ldg(q + xp2));
  const double sy = axis_sum(__ldg(q + ym2), __ldg(q + ym1), t30, __ldg(q + yp1), __ldg(q + yp2));
  const double sz = axis_sum(__ldg(q + zm2), __ldg(q + zm1), t30, __ldg(q + zp1), __ldg(q + zp2));
  return __dmul_rn(__dadd_rn(__dadd_rn(sx, sy), sz), inv12h2);
}

// Per-sample maxima of binary32 bit patterns (non-negative values, so the
// integer order is the float order) over a 256-thread block: each warp keeps
// the maximum of its current sample (a warp's 32 indices lie in one sample,
// P being a multiple of 128) and flushes it when the sample changes; at the
// end the block merges its warps and issues one atomic per sample it saw,
// instead of one per warp and iteration on the same few addresses.
struct BlockMax {
  long long cur = -1;
  unsigned m[2] = {0u, 0u};
  __device__ void flush(unsigned* out, int nv) {
    if (cur < 0) return;
    for (int v = 0; v < nv; ++v) {
      const unsigned r = __reduce_max_sync(0xffffffffu, m[v]);
      if ((threadIdx.x & 31) == 0 && r) atomicMax(&out[nv * cur + v], r);
    }
  }
  // warp-uniform: the sample of this warp's indices
  __device__ void enter(long long b, unsigned* out, int nv) {
    if (b == cur) return;
    flush(out, nv);
    cur = b;
    m[0] = m[1] = 0u;
  }
  __device__ void finish(unsigned* out, int nv) {
    __shared__ long long wb[8];
    __shared__ unsigned wm[8][2];
    const int warp = threadIdx.x >> 5;
    unsigned r[2] = {0u, 0u};
    for (int v = 0; v < nv; ++v) r[v] = __reduce_max_sync(0xffffffffu, m[v]);
    if ((threadIdx.x & 31) == 0) {
      wb[warp] = cur;
      wm[warp][0] = r[0];
      wm[warp][1] = r[1];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      long long b = -1;
      unsigned acc[2] = {0u, 0u};
      for (int w = 0; w <= (int)(blockDim.x >> 5); ++w) {
        const long long bw = w < (int)(blockDim.x >> 5) ? wb[w] : -2;
        if (bw != b) {
          if (b >= 0)
            for (int v = 0; v < nv; ++v)
              if (acc[v]) atomicMax(&out[nv * b + v], acc[v]);
          b = bw;
          acc[0] = acc[1] = 0u;
        }
        if (w < (int)(blockDim.x >> 5) && bw >= 0) {
          acc[0] = max(acc[0], wm[w][0]);
          acc[1] = max(acc[1], wm[w][1]);
        }
      }
    }
  }
};

__global__ void __launch_bounds__(256) k_absmax(const double* psi, const double* pi, Dims d, double delta,
                                                unsigned* maxbits) {
  const long long P = d.points(), N = P * d.batch;
  BlockMax bm;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < N; base += (long long)gridDim.x * blockDim.x) {
    const long long wfirst = base + (threadIdx.x & ~31);
    if (wfirst >= N) break;  // warp-uniform
    bm.enter(wfirst / P, maxbits, 1);
    const long long i = base + threadIdx.x;
    if (i < N) bm.m[0] = max(bm.m[0], __float_as_uint(__double2float_rn(fmax(fabs(psi[i]), __dmul_rn(delta, fabs(pi[i]))))));
  }
  bm.finish(maxbits, 1);
}

// Per-sample products that the feature and update kernels would otherwise
// form at every point (the same roundings, so the same values): s, s Delta,
// s Delta^2 .. s Delta^6 (features), a = sigma / s and a / Delta (update),
// with s = scale[b].  sc: [batch][9].
__global__ void k_sample_coef(const float* scale, int batch, double delta, double d2, double d3, double d4, double d5,
                              double d6, double sigma, double* sc) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  const double sv = (double)scale[b];
  const double a = __ddiv_rn(sigma, sv);
  const double v[9] = {sv, __dmul_rn(sv, delta), __dmul_rn(sv, d2), __dmul_rn(sv, d3), __dmul_rn(sv, d4),
                       __dmul_rn(sv, d5), __dmul_rn(sv, d6), a, __ddiv_rn(a, delta)};
  for (int q = 0; q < 9; ++q) sc[b * 9 + q] = v[q];
}

__global__ void k_scale(const unsigned* maxbits, int batch, float* scale) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  const float m = __uint_as_float(maxbits[b]);
  scale[b] = m > 0.0f ? __double2float_rn(__ddiv_rn(1.0, (double)m)) : 1.0f;
}

struct Coef {
  // Delta, Delta^2 .. Delta^6, Delta^2/2, Delta^3/6, Delta^4/24, 1/(12 h^2), sigma
  double delta, d2, d3, d4, d5, d6, hd2, d36, d424, inv12h2, sigma;
};


// lap: the chain L psi, L Pi, L^2 psi, L^2 Pi, L^3 psi, L^3 Pi ([6][batch * points])
__global__ void k_features(const double* psi, const double* pi, Dims d, const double* sc, const double* lap,
                           uint4* x) {
  const long long N = d.points() * d.batch;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N; g += (long long)gridDim.x * blockDim.x) {
    const double* cs = sc + 9 * (g / d.points());
    const double f[7] = {__dmul_rn(cs[0], psi[g]),        __dmul_rn(cs[1], pi[g]),         __dmul_rn(cs[2], lap[g]),
                         __dmul_rn(cs[3], lap[N + g]),    __dmul_rn(cs[4], lap[2 * N + g]), __dmul_rn(cs[5], lap[3 * N + g]),
                         __dmul_rn(cs[6], lap[4 * N + g])};
    __nv_bfloat162 h[4];
    for (int q = 0; q < 3; ++q) h[q] = __floats2bfloat162_rn(__double2float_rn(f[2 * q]), __double2float_rn(f[2 * q + 1]));
    h[3] = __floats2bfloat162_rn(__double2float_rn(f[6]), 0.0f);
    x[g] = make_uint4(*reinterpret_cast<unsigned*>(&h[0]), *reinterpret_cast<unsigned*>(&h[1]),
                      *reinterpret_cast<unsigned*>(&h[2]), *reinterpret_cast<unsigned*>(&h[3]));
  }
}

// L of F fields of every sample (F = 1: a; F = 2: a and b) into out, field f
// at out + f * batch * points.  Grid (n1, n2, batch); the threads of a block
// walk the row.
template <int F>
__global__ void k_lap(const double* a, const double* b, Dims d, double inv12h2, double* out) {
  const int j = blockIdx.x, k = blockIdx.y, s = blockIdx.z;
  const long long P = d.points(), N = P * d.batch, o = (long long)s * P;
  const long long row = o + ((long long)k * d.n1 + j) * d.n0;
  for (int i = threadIdx.x; i < d.n0; i += blockDim.x) {
    out[row + i] = lap4(a + o, d, i, j, k, inv12h2);
    if (F == 2) out[N + row + i] = lap4(b + o, d, i, j, k, inv12h2);
  }
}

template <int F>
void launch_lap(const double* a, const double* b, const Dims& d, double inv12h2, double* out, cudaStream_t st) {
  k_lap<F><<<dim3((unsigned)d.n1, (unsigned)d.n2, (unsigned)d.batch), 128, 0, st>>>(a, b, d, inv12h2, out);
}

__global__ void k_targets(const double* psi0, const double* pi0, const double* psi1, const double* pi1, Dims d,
                          Coef c, const float* scale, const double* lap, float2* t) {
  const long long P = d.points(), N = P * d.batch;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N; g += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(g / P);
    const double lp = lap[g], lq = lap[N + g], llp = lap[2 * N + g], llq = lap[3 * N + g];
    double r0 = __dsub_rn(__dsub_rn(psi1[g], psi0[g]), __dmul_rn(c.delta, pi0[g]));
    r0 = __dsub_rn(__dsub_rn(__dsub_rn(r0, __dmul_rn(c.hd2, lp)), __dmul_rn(c.d36, lq)), __dmul_rn(c.d424, llp));
    double r1 = __dsub_rn(__dsub_rn(pi1[g], pi0[g]), __dmul_rn(c.delta, lp));
    r1 = __dsub_rn(__dsub_rn(__dsub_rn(r1, __dmul_rn(c.hd2, lq)), __dmul_rn(c.d36, llp)), __dmul_rn(c.d424, llq));
    const double cs = __ddiv_rn((double)scale[b], c.sigma);
    t[g] = make_float2(__double2float_rn(__dmul_rn(cs, r0)), __double2float_rn(__dmul_rn(__dmul_rn(cs, c.delta), r1)));
  }
}

// (psi1, Pi1) from (psi0, Pi0), their Laplacians and the network output y
// ([..][8], channels 0, 1)
__global__ void k_apply(const double* psi0, const double* pi0, Dims d, Coef c, const double* sc, const double* lap,
                        const float* y, double* psi1, double* pi1) {
  const long long P = d.points(), N = P * d.batch;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N; g += (long long)gridDim.x * blockDim.x) {
    const double* cs = sc + 9 * (g / P);
    const double lp = lap[g], lq = lap[N + g], llp = lap[2 * N + g], llq = lap[3 * N + g];
    const double a = cs[7], ad = cs[8];   // sigma / s and its quotient by Delta
    const float2 yv = *reinterpret_cast<const float2*>(y + g * 8);
    const double n0 = (double)yv.x, n1 = (double)yv.y;
    double u = __dadd_rn(psi0[g], __dmul_rn(c.delta, pi0[g]));
    u = __dadd_rn(__dadd_rn(__dadd_rn(u, __dmul_rn(c.hd2, lp)), __dmul_rn(c.d36, lq)), __dmul_rn(c.d424, llp));
    psi1[g] = __dadd_rn(u, __dmul_rn(a, n0));
    double v = __dadd_rn(pi0[g], __dmul_rn(c.delta, lp));
    v = __dadd_rn(__dadd_rn(__dadd_rn(v, __dmul_rn(c.hd2, lq)), __dmul_rn(c.d36, llp)), __dmul_rn(c.d424, llq));
    pi1[g] = __dadd_rn(v, __dmul_rn(ad, n1));
  }
}

}  // namespace

namespace {

__global__ void k_to_bf16(const float* w, __nv_bfloat16* w16, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    w16[i] = __float2bfloat16_rn(w[i]);
}

unsigned grid_for(long long n, int threads = 256) {
  long long b = (n + threads - 1) / threads;
  return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}


// Residual of a call against the method's RHS: with f = Pi, f' = L psi for
// psi and f = L psi, f' = L Pi for Pi, the two-point quadrature with end
// corrections, int_0^Delta f = Delta/2 (f0 + f1) + Delta^2/12 (f0' - f1'),
// leaves O(Delta^5) for the exact evolution.  lap: L psi0, L Pi0, L psi1,
// L Pi1.  Writes, per sample, max(|R_psi|, Delta |R_Pi|) and max(|psi0|,
// Delta |Pi0|) as binary32 bit patterns (atomic maximum).
__global__ void __launch_bounds__(256) k_check(const double* psi0, const double* pi0, const double* psi1,
                                               const double* pi1, Dims d, Coef c, const double* lap, unsigned* out) {
  const long long P = d.points(), N = P * d.batch;
  const double hd = 0.5 * c.delta, d12 = c.d2 / 12.0;
  BlockMax bm;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < N; base += (long long)gridDim.x * blockDim.x) {
    const long long wfirst = base + (threadIdx.x & ~31);
    if (wfirst >= N) break;  // warp-uniform
    bm.enter(wfirst / P, out, 2);
    const long long g = base + threadIdx.x;
    if (g < N) {
      const double lp0 = lap[g], lq0 = lap[N + g], lp1 = lap[2 * N + g], lq1 = lap[3 * N + g];
      const double rp = (psi1[g] - psi0[g]) - hd * (pi0[g] + pi1[g]) + d12 * (lp1 - lp0);
      const double rq = (pi1[g] - pi0[g]) - hd * (lp0 + lp1) + d12 * (lq1 - lq0);
      bm.m[0] = max(bm.m[0], __float_as_uint(__double2float_ru(fmax(fabs(rp), c.delta * fabs(rq)))));
      bm.m[1] = max(bm.m[1], __float_as_uint(__double2float_rn(fmax(fabs(psi0[g]), c.delta * fabs(pi0[g])))));
    }
  }
  bm.finish(out, 2);
}

struct HermiteBoxes {
  int nb;
  mpw::Box b[mpw::MAX_PATCHES];
};

// Quintic Hermite interpolant in time of the state between two calls: the
// four RK4 stage states of one step, written into the cells of the given
// boxes of four padded patch buffers in one pass.  Stage k is
// y = c0 y0 + c1 y0' + c2 y0'' + c3 y1 + c4 y1' + c5 y1'' (cf[6 k ..]: the
// basis and its derivatives at the step's start, times Delta^k, combined as
// the RK4 stage input of a linear system), with y = psi, y' = Pi, y'' = L psi
// for psi and y = Pi, y' = L psi, y'' = L Pi for Pi.  slot[k] receives the
// largest biased exponent of each field of buffer k (one atomic per block).
struct HermiteOut {
  double* buf[4];
  int* slot[4];
};

__global__ void __launch_bounds__(256) k_hermite(HermiteOut out, mpw::Geom g, const double* u, long long P,
                                                 const double* cf, HermiteBoxes hb) {
  const double *psi0 = u, *pi0 = u + P, *psi1 = u + 2 * P, *pi1 = u + 3 * P;
  const double *lp0 = u + 4 * P, *lq0 = u + 5 * P, *lp1 = u + 6 * P, *lq1 = u + 7 * P;
  const mpw::Box& bx = hb.b[blockIdx.y];
  const int w0 = bx.hi[0] - bx.lo[0] + 1, w1 = bx.hi[1] - bx.lo[1] + 1, w2 = bx.hi[2] - bx.lo[2] + 1;
  const long long V = (long long)w0 * w1 * w2;
  int em[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < V; e += (long long)gridDim.x * blockDim.x) {
    const int i = bx.lo[0] + (int)(e % w0), j = bx.lo[1] + (int)((e / w0) % w1), k = bx.lo[2] + (int)(e / ((long long)w0 * w1));
    const long long q = ((long long)k * g.n[1] + j) * g.n[0] + i;
    const double a0 = psi0[q], a1 = pi0[q], a2 = lp0[q], a3 = psi1[q], a4 = pi1[q], a5 = lp1[q];
    const double b2 = lq0[q], b5 = lq1[q];
    const long long at = g.at(i, j, k);
#pragma unroll
    for (int st = 0; st < 4; ++st) {
      const double* c = cf + 6 * st;
      const double ys = c[0] * a0 + c[1] * a1 + c[2] * a2 + c[3] * a3 + c[4] * a4 + c[5] * a5;
      const double yp = c[0] * a1 + c[1] * a2 + c[2] * b2 + c[3] * a4 + c[4] * a5 + c[5] * b5;
      out.buf[st][at] = ys;
      out.buf[st][g.vol + at] = yp;
      em[2 * st] = max(em[2 * st], mpw::biased_exponent(ys));
      em[2 * st + 1] = max(em[2 * st + 1], mpw::biased_exponent(yp));
    }
  }
  __shared__ int bm[8][8];
  const int warp = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    const int r = __reduce_max_sync(0xffffffffu, em[v]);
    if ((threadIdx.x & 31) == 0) bm[warp][v] = r;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    int r = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = max(r, bm[w][threadIdx.x]);
    if (r) atomicMax(out.slot[threadIdx.x >> 1] + (threadIdx.x & 1), r);
  }
}

}  // namespace

struct mpw_sur {
  int device = 0;
  cudaStream_t stream = nullptr;
  double dt = 0.0, h = 0.0, sigma = 1.0;
  Coef coef{};
  Layer L[NLAYER];
  long long nparam = 0;
  float* w = nullptr;  // master parameters, their gradient, Adam moments
  float* g = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  __nv_bfloat16* w16 = nullptr;  // BF16 copy the layers read
  int t = 0;                     // Adam steps taken
  long long cap = 0;             // points the activation buffers hold
  __nv_bfloat16* act[NLAYER - 1] = {};
  __nv_bfloat16* grad[2] = {};
  __nv_bfloat16* gy = nullptr;
  float* y = nullptr;
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  double* loss = nullptr;
  // inference workspace
  long long xcap = 0;
  uint16_t* x = nullptr;
  double* lap = nullptr;  // the Laplacian chain of the last input (6 * xcap)
  int bcap = 0;
  float* scale = nullptr;
  unsigned* maxbits = nullptr;
  double* sc = nullptr;   // per-sample products of the last features ([bcap][9])
};

namespace {

mpw_status use(mpw_sur* s) {
  if (!s) return fail(MPW_ERR_ARG, "null surrogate handle");
  SUR_TRY(cudaSetDevice(s->device));
  return MPW_OK;
}

mpw_status dims_of(int batch, const int n[3], Dims& d) {
  if (!n || batch < 1 || n[0] < 16 || n[1] < 8 || n[2] < 5 || n[0] % 16 || n[1] % 8)
    return fail(MPW_ERR_ARG, "surrogate: volume must have n0 % 16 == 0, n1 % 8 == 0, n2 >= 5, batch >= 1");
  d = Dims{n[0], n[1], n[2], batch};
  return MPW_OK;
}

void free_buffers(mpw_sur* s) {
  for (auto*& p : s->act) cudaFree(p), p = nullptr;
  for (auto*& p : s->grad) cudaFree(p), p = nullptr;
  cudaFree(s->gy);
  cudaFree(s->y);
  s->gy = nullptr;
  s->y = nullptr;
  s->cap = 0;
}

mpw_status ensure_train(mpw_sur* s, long long P) {
  if (P <= s->cap) return MPW_OK;
  free_buffers(s);
  for (auto*& p : s->act) SUR_TRY(cudaMalloc(&p, (size_t)P * 32 * 2));
  for (auto*& p : s->grad) SUR_TRY(cudaMalloc(&p, (size_t)P * 32 * 2));
  SUR_TRY(cudaMalloc(&s->gy, (size_t)P * 8 * 2));
  SUR_TRY(cudaMalloc(&s->y, (size_t)P * 8 * 4));
  s->cap = P;
  return MPW_OK;
}

mpw_status ensure_infer(mpw_sur* s, long long P, int batch) {
  if (P > s->xcap) {
    cudaFree(s->x);
    cudaFree(s->lap);
    s->x = nullptr;
    s->lap = nullptr;
    s->xcap = 0;
    SUR_TRY(cudaMalloc(&s->x, (size_t)P * 8 * 2));
    SUR_TRY(cudaMalloc(&s->lap, (size_t)P * 6 * sizeof(double)));
    s->xcap = P;
  }
  if (batch > s->bcap) {
    cudaFree(s->scale);
    cudaFree(s->maxbits);
    cudaFree(s->sc);
    s->scale = nullptr;
    s->maxbits = nullptr;
    s->sc = nullptr;
    s->bcap = 0;
    SUR_TRY(cudaMalloc(&s->scale, (size_t)batch * 4));
    SUR_TRY(cudaMalloc(&s->maxbits, (size_t)batch * 4));
    SUR_TRY(cudaMalloc(&s->sc, (size_t)batch * 9 * sizeof(double)));
    s->bcap = batch;
  }
  return MPW_OK;
}

// The Laplacian chain of (psi, Pi) into s->lap: L psi, L Pi, L^2 psi, L^2 Pi,
// L^3 psi (the features read no L^3 Pi).
mpw_status lap_chain(mpw_sur* s, const double* psi, const double* pi, const Dims& d) {
  const long long N = d.points() * d.batch;
  launch_lap<2>(psi, pi, d, s->coef.inv12h2, s->lap, s->stream);
  launch_lap<2>(s->lap, s->lap + N, d, s->coef.inv12h2, s->lap + 2 * N, s->stream);
  launch_lap<1>(s->lap + 2 * N, nullptr, d, s->coef.inv12h2, s->lap + 4 * N, s->stream);
  SUR_TRY(cudaGetLastError());
  return MPW_OK;
}

const uint16_t* W16(const mpw_sur* s, int l) { return reinterpret_cast<const uint16_t*>(s->w16 + s->L[l].w); }

// layers 1-3 into s->act, layer 4 into y (FP32)
mpw_status forward_chain(mpw_sur* s, const uint16_t* x, const Dims& d, float* y) {
  const int n[3] = {d.n0, d.n1, d.n2};
  const uint16_t* in = x;
  for (int l = 0; l < NLAYER - 1; ++l) {
    uint16_t* out = reinterpret_cast<uint16_t*>(s->act[l]);
    MPW_TRY(mpw_conv3_forward(in, s->L[l].cin, W16(s, l), s->w + s->L[l].b, s->L[l].cout, d.batch, n, 1, nullptr,
                              out, nullptr, s->stream));
    in = out;
  }
  const Layer& L = s->L[NLAYER - 1];
  return mpw_conv3_forward(in, L.cin, W16(s, NLAYER - 1), s->w + L.b, L.cout, d.batch, n, 0, nullptr, nullptr, y,
                           s->stream);
}

}  // namespace

extern "C" {

long long mpw_sur_param_count(void) {
  Layer L[NLAYER];
  return layer_table(L);
}

mpw_status mpw_sur_create(int device, void* stream, double dt, double h, double sigma, mpw_sur** out) {
  if (!out) return fail(MPW_ERR_ARG, "null output handle");
  *out = nullptr;
  if (!(dt > 0.0) || !(h > 0.0) || !(sigma > 0.0)) return fail(MPW_ERR_ARG, "surrogate: dt, h and sigma must be > 0");
  mpw_sur* s = new mpw_sur;
  s->device = device;
  s->stream = (cudaStream_t)stream;
  s->dt = dt;
  s->h = h;
  s->sigma = sigma;
  const double D = 4.0 * dt;
  s->coef = Coef{D,          D * D,          D * D * D,          D * D * D * D,        D * D * D * D * D,
                  D * D * D * D * D * D, D * D / 2.0, D * D * D / 6.0, D * D * D * D / 24.0, 1.0 / (12.0 * h * h),
                  sigma};
  s->nparam = layer_table(s->L);
  auto bail = [&](cudaError_t e) {
    mpw_sur_destroy(s);
    return cuda_fail(e);
  };
  cudaError_t e;
  if ((e = cudaSetDevice(device))) return bail(e);
  const size_t pb = (size_t)s->nparam * 4;
  for (float** p : {&s->w, &s->g, &s->m, &s->v}) {
    if ((e = cudaMalloc(p, pb))) return bail(e);
    if ((e = cudaMemsetAsync(*p, 0, pb, s->stream))) return bail(e);
  }
  if ((e = cudaMalloc(&s->w16, (size_t)s->nparam * 2))) return bail(e);
  if ((e = cudaMemsetAsync(s->w16, 0, (size_t)s->nparam * 2, s->stream))) return bail(e);
  for (int l = 0; l < NLAYER; ++l) {
    const size_t b = mpw_conv3_wgrad_scratch_bytes(s->L[l].cin, s->L[l].cout);
    if (b > s->scratch_bytes) s->scratch_bytes = b;
  }
  if ((e = cudaMalloc(&s->scratch, s->scratch_bytes))) return bail(e);
  if ((e = cudaMalloc(&s->loss, sizeof(double)))) return bail(e);
  if ((e = cudaStreamSynchronize(s->stream))) return bail(e);
  *out = s;
  return MPW_OK;
}

void mpw_sur_destroy(mpw_sur* s) {
  if (!s) return;
  cudaSetDevice(s->device);
  cudaStreamSynchronize(s->stream);
  free_buffers(s);
  for (void* p : {(void*)s->w, (void*)s->g, (void*)s->m, (void*)s->v, (void*)s->w16, s->scratch, (void*)s->loss,
                  (void*)s->x, (void*)s->lap, (void*)s->scale, (void*)s->maxbits, (void*)s->sc})
    cudaFree(p);
  delete s;
}

mpw_status mpw_sur_set_params(mpw_sur* s, const float* params, long long count) {
  MPW_TRY(use(s));
  if (!params || count != s->nparam) return fail(MPW_ERR_ARG, "surrogate: params must hold mpw_sur_param_count() values");
  const size_t pb = (size_t)count * 4;
  SUR_TRY(cudaMemcpyAsync(s->w, params, pb, cudaMemcpyHostToDevice, s->stream));
  SUR_TRY(cudaMemsetAsync(s->m, 0, pb, s->stream));
  SUR_TRY(cudaMemsetAsync(s->v, 0, pb, s->stream));
  SUR_TRY(cudaMemsetAsync(s->g, 0, pb, s->stream));
  k_to_bf16<<<grid_for(count), 256, 0, s->stream>>>(s->w, s->w16, count);
  SUR_TRY(cudaGetLastError());
  SUR_TRY(cudaStreamSynchronize(s->stream));
  s->t = 0;
  return MPW_OK;
}

static mpw_status copy_out(mpw_sur* s, const float* src, float* dst, long long count) {
  MPW_TRY(use(s));
  if (!dst || count != s->nparam) return fail(MPW_ERR_ARG, "surrogate: buffer must hold mpw_sur_param_count() values");
  SUR_TRY(cudaMemcpyAsync(dst, src, (size_t)count * 4, cudaMemcpyDeviceToHost, s->stream));
  SUR_TRY(cudaStreamSynchronize(s->stream));
  return MPW_OK;
}

mpw_status mpw_sur_get_params(mpw_sur* s, float* params, long long count) {
  return s ? copy_out(s, s->w, params, count) : fail(MPW_ERR_ARG, "null surrogate handle");
}

mpw_status mpw_sur_get_grads(mpw_sur* s, float* grads, long long count) {
  return s ? copy_out(s, s->g, grads, count) : fail(MPW_ERR_ARG, "null surrogate handle");
}

mpw_status mpw_sur_features(mpw_sur* s, const double* psi0, const double* pi0, int batch, const int n[3],
                            uint16_t* x, float* scale) {
  MPW_TRY(use(s));
  Dims d;
  MPW_TRY(dims_of(batch, n, d));
  if (!psi0 || !pi0 || !x || !scale) return fail(MPW_ERR_ARG, "surrogate: null tensor");
  const long long N = d.points() * batch;
  MPW_TRY(ensure_infer(s, N, batch));
  SUR_TRY(cudaMemsetAsync(s->maxbits, 0, (size_t)batch * 4, s->stream));
  k_absmax<<<grid_for(N), 256, 0, s->stream>>>(psi0, pi0, d, s->coef.delta, s->maxbits);
  k_scale<<<(batch + 127) / 128, 128, 0, s->stream>>>(s->maxbits, batch, scale);
  MPW_TRY(lap_chain(s, psi0, pi0, d));
  const Coef& c = s->coef;
  k_sample_coef<<<(batch + 127) / 128, 128, 0, s->stream>>>(scale, batch, c.delta, c.d2, c.d3, c.d4, c.d5, c.d6, c.sigma,
                                                          s->sc);
  k_features<<<grid_for(N), 256, 0, s->stream>>>(psi0, pi0, d, s->sc, s->lap, reinterpret_cast<uint4*>(x));
  SUR_TRY(cudaGetLastError());
  return MPW_OK;
}

mpw_status mpw_sur_targets(mpw_sur* s, const double* psi0, const double* pi0, const double* psi1, const double* pi1,
                           int batch, const int n[3], const float* scale, float* t) {
  MPW_TRY(use(s));
  Dims d;
  MPW_TRY(dims_of(batch, n, d));
  if (!psi0 || !pi0 || !psi1 || !pi1 || !scale || !t) return fail(MPW_ERR_ARG, "surrogate: null tensor");
  const long long P = d.points() * batch;
  MPW_TRY(ensure_infer(s, P, batch));
  MPW_TRY(lap_chain(s, psi0, pi0, d));
  k_targets<<<grid_for(P), 256, 0, s->stream>>>(psi0, pi0, psi1, pi1, d, s->coef, scale, s->lap,
                                               reinterpret_cast<float2*>(t));
  SUR_TRY(cudaGetLastError());
  return MPW_OK;
}

mpw_status mpw_sur_forward(mpw_sur* s, const uint16_t* x, int batch, const int n[3], float* y) {
  MPW_TRY(use(s));
  Dims d;
  MPW_TRY(dims_of(batch, n, d));
  if (!x || !y) return fail(MPW_ERR_ARG, "surrogate: null tensor");
  MPW_TRY(ensure_train(s, d.points() * batch));
  return forward_chain(s, x, d, y);
}

mpw_status mpw_sur_train_step(mpw_sur* s, const uint16_t* x, const float* t, int batch, const int n[3], float lr,
                              double* loss) {
  MPW_TRY(use(s));
  Dims d;
  MPW_TRY(dims_of(batch, n, d));
  if (!x || !t || !(lr > 0.0f)) return fail(MPW_ERR_ARG, "surrogate: null tensor or lr <= 0");
  const long long P = d.points() * batch;
  MPW_TRY(ensure_train(s, P));
  MPW_TRY(forward_chain(s, x, d, s->y));
  uint16_t* gy = reinterpret_cast<uint16_t*>(s->gy);
  MPW_TRY(mpw_mse_grad(s->y, 8, t, 2, P, gy, s->loss, s->stream));
  // backward, layer 4 down to layer 1; gradients at activations are masked by
  // the ReLU of the layer that produced them
  const uint16_t* gout = gy;
  for (int l = NLAYER - 1; l >= 0; --l) {
    const Layer& L = s->L[l];
    const uint16_t* in = l == 0 ? x : reinterpret_cast<const uint16_t*>(s->act[l - 1]);
    MPW_TRY(mpw_conv3_backward_weights(in, L.cin, gout, L.cout, batch, n, s->g + L.w, s->g + L.b, s->scratch,
                                       s->scratch_bytes, s->stream));
    if (l == 0) break;
    uint16_t* gin = reinterpret_cast<uint16_t*>(s->grad[l & 1]);
    MPW_TRY(mpw_conv3_backward_data(gout, L.cout, W16(s, l), L.cin, batch, n, in, gin, nullptr, s->stream));
    gout = gin;
  }
  double host_loss = 0.0;
  if (loss) SUR_TRY(cudaMemcpyAsync(&host_loss, s->loss, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  s->t += 1;
  MPW_TRY(mpw_adam_step(s->w, reinterpret_cast<uint16_t*>(s->w16), s->g, s->m, s->v, s->nparam, lr, 0.9f, 0.999f,
                        1e-8f, s->t, s->stream));
  if (loss) {
    SUR_TRY(cudaStreamSynchronize(s->stream));
    *loss = host_loss;
  }
  return MPW_OK;
}

mpw_status mpw_sur_predict(mpw_sur* s, const double* psi0, const double* pi0, int batch, const int n[3], double* psi1,
                           double* pi1) {
  MPW_TRY(use(s));
  Dims d;
  MPW_TRY(dims_of(batch, n, d));
  if (!psi0 || !pi0 || !psi1 || !pi1) return fail(MPW_ERR_ARG, "surrogate: null tensor");
  if (psi1 == psi0 || psi1 == pi0 || pi1 == psi0 || pi1 == pi0) return fail(MPW_ERR_ARG, "surrogate: outputs alias inputs");
  const long long P = d.points() * batch;
  MPW_TRY(ensure_infer(s, P, batch));
  MPW_TRY(ensure_train(s, P));
  MPW_TRY(mpw_sur_features(s, psi0, pi0, batch, n, s->x, s->scale));
  MPW_TRY(forward_chain(s, s->x, d, s->y));
  // s->lap holds the chain of (psi0, Pi0) and s->sc its per-sample products,
  // both from the features
  k_apply<<<grid_for(P), 256, 0, s->stream>>>(psi0, pi0, d, s->coef, s->sc, s->lap, s->y, psi1, pi1);
  SUR_TRY(cudaGetLastError());
  return MPW_OK;
}

mpw_status mpw_sur_check(mpw_sur* s, const double* psi0, const double* pi0, const double* psi1, const double* pi1,
                         int batch, const int n[3], double* lap, float* out) {
  MPW_TRY(use(s));
  Dims d;
  MPW_TRY(dims_of(batch, n, d));
  if (!psi0 || !pi0 || !psi1 || !pi1 || !out) return fail(MPW_ERR_ARG, "surrogate: null tensor");
  const long long N = d.points() * batch;
  if (!lap) {
    MPW_TRY(ensure_infer(s, N, batch));
    lap = s->lap;
  }
  SUR_TRY(cudaMemsetAsync(out, 0, (size_t)batch * 2 * sizeof(float), s->stream));
  launch_lap<2>(psi0, pi0, d, s->coef.inv12h2, lap, s->stream);
  launch_lap<2>(psi1, pi1, d, s->coef.inv12h2, lap + 2 * N, s->stream);
  k_check<<<grid_for(N), 256, 0, s->stream>>>(psi0, pi0, psi1, pi1, d, s->coef, lap, reinterpret_cast<unsigned*>(out));
  SUR_TRY(cudaGetLastError());
  return MPW_OK;
}

}  // extern "C"

namespace mpw {

mpw_status sur_check_after_predict(mpw_sur* s, const double* psi0, const double* pi0, const double* psi1,
                                   const double* pi1, const int n[3], double* lap, float* out) {
  MPW_TRY(use(s));
  Dims d;
  MPW_TRY(dims_of(1, n, d));
  const long long N = d.points();
  if (!lap || !out || N > s->xcap) return fail(MPW_ERR_ARG, "surrogate: check without a prediction");
  SUR_TRY(cudaMemsetAsync(out, 0, 2 * sizeof(float), s->stream));
  SUR_TRY(cudaMemcpyAsync(lap, s->lap, (size_t)2 * N * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
  launch_lap<2>(psi1, pi1, d, s->coef.inv12h2, lap + 2 * N, s->stream);
  k_check<<<grid_for(N), 256, 0, s->stream>>>(psi0, pi0, psi1, pi1, d, s->coef, lap, reinterpret_cast<unsigned*>(out));
  SUR_TRY(cudaGetLastError());
  return MPW_OK;
}

void launch_hermite(double* const buf[4], int* const slot2[4], const Geom& g, const double* u, const double* coef_dev,
                    const Box* boxes, int nbox, void* stream) {
  if (nbox <= 0) return;
  HermiteBoxes hb{};
  hb.nb = nbox;
  long long vmax = 0;
  for (int q = 0; q < nbox; ++q) {
    hb.b[q] = boxes[q];
    long long v = 1;
    for (int a = 0; a < 3; ++a) v *= std::max(boxes[q].hi[a] - boxes[q].lo[a] + 1, 0);
    vmax = std::max(vmax, v);
  }
  if (vmax == 0) return;
  HermiteOut out{};
  for (int k = 0; k < 4; ++k) {
    out.buf[k] = buf[k];
    out.slot[k] = slot2[k];
  }
  const long long P = (long long)g.n[0] * g.n[1] * g.n[2];
  const dim3 grid(grid_for(vmax), (unsigned)nbox);
  k_hermite<<<grid, 256, 0, (cudaStream_t)stream>>>(out, g, u, P, coef_dev, hb);
}

bool sur_geometry(const mpw_sur* s, double* dt, double* h, void** stream) {
  if (!s) return false;
  *dt = s->dt;
  *h = s->h;
  *stream = s->stream;
  return true;
}

}  // namespace mpw
