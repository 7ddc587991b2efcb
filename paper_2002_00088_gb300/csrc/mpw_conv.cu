// mpw_conv.cu -- tensor-core layers of the learned surrogate (the C ABI of
// include/mpw_surrogate.h): periodic 3x3x3 convolution, its input and weight
// gradients, Adam and the squared-error gradient.
//
// Forward and input gradient of volumes 128 points wide run on the
// 5th-generation tensor cores (k_conv3_tc, tcgen05.mma with TMEM
// accumulators; described below).  Every other volume, and the weight
// gradient, use an implicit GEMM on mma.sync m16n8k16 (BF16 operands, FP32
// accumulation):
//  - k_conv3_t<CIN, COUT>: M = points (a warp owns 16 x-points on two
//    planes), N = output channels, K = 27 taps x CIN.  A persistent CTA
//    stages the layer's weights once and the periodic 18 x 10 x 4 halo of
//    each 16 x 8 x 2 block; both operands come from shared memory through
//    ldmatrix and the K loop is unrolled.
//  - The input gradient is the forward kernel reading the weights mirrored
//    and transposed.
//  - k_conv3_wgrad: M = output channels, N = input channels, K = points; each
//    CTA keeps its partial sums in registers over its blocks and k_sum_parts
//    adds the partials in a fixed order (deterministic).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>

#include "../../include/mpw_surrogate.h"
#include "mpw_internal.cuh"
#include "mpw_tma.cuh"

namespace mpw {
namespace {

constexpr int BX = 16, BY = 8;                   // output block: BY warp rows of BX x-points
constexpr int HX = BX + 2, HY = BY + 2, HZ = 3;  // its periodic halo
constexpr int HPTS = HX * HY * HZ;
constexpr int FWD_THREADS = 32 * BY;
constexpr int WG_WARPS = 16;
constexpr int WG_THREADS = 32 * WG_WARPS;

// BF16 elements per halo point in shared memory: 32 channels padded to 40 make
// the eight rows of an A fragment fall in distinct banks (20-word stride).
template <int C>
__host__ __device__ constexpr int xstride() { return C == 32 ? 40 : C; }
// K = 27 taps x CIN rounded up to the MMA depth, and the padded weight row
template <int CIN>
__host__ __device__ constexpr int kdim() { return (27 * CIN + 15) / 16 * 16; }
template <int CIN>
__host__ __device__ constexpr int wstride() { return kdim<CIN>() + 8; }

struct Vol {
  int n0, n1, n2, batch;
};

__device__ __forceinline__ int wrap1(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// D = A B + D, A 16x16 row-major, B 16x8 column-major, BF16 in, FP32 out
__device__ __forceinline__ void mma_bf16(float c[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// block index -> sample b, plane z, first row y0, first column x0
__device__ __forceinline__ void block_origin(long long blk, const Vol& v, int& b, int& z, int& y0, int& x0) {
  const int bx = v.n0 / BX, by = v.n1 / BY;
  x0 = (int)(blk % bx) * BX;
  blk /= bx;
  y0 = (int)(blk % by) * BY;
  blk /= by;
  z = (int)(blk % v.n2);
  b = (int)(blk / v.n2);
}

__device__ __forceinline__ long long point_index(const Vol& v, int b, int z, int y, int x) {
  return (((long long)b * v.n2 + z) * v.n1 + y) * v.n0 + x;
}

// the HX x HY x 3 periodic halo of a block, C channels, 16-byte copies
template <int C>
__device__ void stage_halo(__nv_bfloat16* Xs, const __nv_bfloat16* x, const Vol& v, int b, int z, int y0, int x0) {
  constexpr int CH = C / 8;
  for (int i = threadIdx.x; i < HPTS * CH; i += blockDim.x) {
    const int hp = i / CH, ch = i - hp * CH;
    const int hx = hp % HX, hy = (hp / HX) % HY, hz = hp / (HX * HY);
    const long long p = point_index(v, b, wrap1(z + hz - 1, v.n2), wrap1(y0 + hy - 1, v.n1), wrap1(x0 + hx - 1, v.n0));
    *reinterpret_cast<int4*>(Xs + hp * xstride<C>() + ch * 8) = *reinterpret_cast<const int4*>(x + p * C + ch * 8);
  }
}

struct FwdArgs {
  const __nv_bfloat16* x;
  const __nv_bfloat16* w;
  const float* bias;
  const __nv_bfloat16* mask;
  __nv_bfloat16* y;
  float* y32;
  Vol v;
  long long nblocks;
  int relu;
  int flip;  // 1: w is the layer W[CIN][27][COUT] and this launch is its input gradient
};

// ---------------------------------------------------------------------------
// Two output planes per warp (M = 2 x 16 points), operands loaded with
// ldmatrix, the K loop unrolled with compile-time offsets.  A block is
// 16 x 8 x 2 points; its periodic halo is 18 x 10 x 4.  With 32 input
// channels a 16-deep K step is half of one tap; with 8, it is two taps, and
// the lanes that address the upper half of the A fragment read the second
// tap (the padding tap past the 27th reads tap 27's neighbour, whose weights
// are zero).

constexpr int HZ2 = 4;
constexpr int HPTS2 = HX * HY * HZ2;

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t& r0, uint32_t& r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(addr));
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(FWD_THREADS, 2) k_conv3_t(const FwdArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int XS = xstride<CIN>(), KP = kdim<CIN>(), WS = wstride<CIN>(), NT = COUT / 8, KSTEPS = KP / 16;
  __nv_bfloat16* Ws = reinterpret_cast<__nv_bfloat16*>(smem);
  __nv_bfloat16* Xs = Ws + COUT * WS;
  for (int i = threadIdx.x; i < COUT * KP; i += blockDim.x) {
    const int n = i / KP, k = i - n * KP;
    __nv_bfloat16 val = __float2bfloat16(0.0f);
    if (k < 27 * CIN) {
      const int tap = k / CIN, c = k - tap * CIN;
      val = A.flip ? A.w[((long long)c * 27 + 26 - tap) * COUT + n] : A.w[((long long)n * 27 + tap) * CIN + c];
    }
    Ws[n * WS + k] = val;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  // ldmatrix rows: A matrices (points 0-7 | 8-15) x (k 0-7 | 8-15); B matrices
  // (n-tile, k 0-7 | 8-15)
  const int arow = (lane & 7) + ((lane >> 3) & 1) * 8, khi = lane >> 4;
  const int akof = CIN == 32 ? khi * 8 : 0;
  const int bq = lane >> 3, br = lane & 7;
  const uint32_t xs0 = smem_u32(Xs), ws0 = smem_u32(Ws);
  uint32_t a_addr[2], b_addr[NT > 1 ? 2 : 1];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) a_addr[mt] = xs0 + (((mt * HY + warp) * HX + arow) * XS + akof) * 2;
  if constexpr (NT > 1) {
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) b_addr[jj] = ws0 + ((8 * (2 * jj + (bq >> 1)) + br) * WS + 8 * (bq & 1)) * 2;
  } else {
    b_addr[0] = ws0 + (br * WS + 8 * (bq & 1)) * 2;
  }
  const int bx = A.v.n0 / BX, by = A.v.n1 / BY, bz = (A.v.n2 + 1) / 2;
  for (long long blk = blockIdx.x; blk < A.nblocks; blk += gridDim.x) {
    long long r = blk;
    const int x0 = (int)(r % bx) * BX;
    r /= bx;
    const int y0 = (int)(r % by) * BY;
    r /= by;
    const int z = (int)(r % bz) * 2;
    const int b = (int)(r / bz);
    __syncthreads();
    constexpr int CH = CIN / 8;
    for (int i = threadIdx.x; i < HPTS2 * CH; i += blockDim.x) {
      const int hp = i / CH, ch = i - hp * CH;
      const int hx = hp % HX, hy = (hp / HX) % HY, hz = hp / (HX * HY);
      const long long p = point_index(A.v, b, wrap1(z + hz - 1, A.v.n2), wrap1(y0 + hy - 1, A.v.n1),
                                      wrap1(x0 + hx - 1, A.v.n0));
      *reinterpret_cast<int4*>(Xs + hp * XS + ch * 8) = *reinterpret_cast<const int4*>(A.x + p * CIN + ch * 8);
    }
    __syncthreads();
    float acc[2][NT][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int j = 0; j < NT; ++j) acc[mt][j][0] = acc[mt][j][1] = acc[mt][j][2] = acc[mt][j][3] = 0.0f;
#pragma unroll
    for (int s = 0; s < KSTEPS; ++s) {
      // byte offset of this lane's A row for K step s
      uint32_t aoff;
      if constexpr (CIN == 32) {
        const int tap = s / 2, dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
        aoff = (uint32_t)((((dz * HY + dy) * HX + dx) * XS + (s % 2) * 16) * 2);
      } else {
        const int t0 = 2 * s, t1 = 2 * s + 1 < 27 ? 2 * s + 1 : 26;
        const uint32_t o0 = (uint32_t)((((t0 / 9) * HY + (t0 / 3) % 3) * HX + t0 % 3) * XS * 2);
        const uint32_t o1 = (uint32_t)((((t1 / 9) * HY + (t1 / 3) % 3) * HX + t1 % 3) * XS * 2);
        aoff = khi ? o1 : o0;
      }
      uint32_t a[2][4], bb[NT][2];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) ldsm_x4(a_addr[mt] + aoff, a[mt][0], a[mt][1], a[mt][2], a[mt][3]);
      const uint32_t koff = (uint32_t)(s * 16 * 2);
      if constexpr (NT > 1) {
#pragma unroll
        for (int jj = 0; jj < NT / 2; ++jj)
          ldsm_x4(b_addr[jj] + koff, bb[2 * jj][0], bb[2 * jj][1], bb[2 * jj + 1][0], bb[2 * jj + 1][1]);
      } else {
        ldsm_x2(b_addr[0] + koff, bb[0][0], bb[0][1]);
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int j = 0; j < NT; ++j) mma_bf16(acc[mt][j], a[mt][0], a[mt][1], a[mt][2], a[mt][3], bb[j][0], bb[j][1]);
    }
    const int y = y0 + warp;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int zz = z + mt;
      if (zz >= A.v.n2) break;
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const int co = 8 * j + 2 * t;
        const float bias0 = A.bias ? A.bias[co] : 0.0f, bias1 = A.bias ? A.bias[co + 1] : 0.0f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const long long p = point_index(A.v, b, zz, y, x0 + g + 8 * h);
          float v0 = acc[mt][j][2 * h] + bias0, v1 = acc[mt][j][2 * h + 1] + bias1;
          if (A.relu) {
            v0 = fmaxf(v0, 0.0f);
            v1 = fmaxf(v1, 0.0f);
          }
          if (A.mask) {
            const __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162*>(A.mask + p * COUT + co);
            if (!(__bfloat162float(m.x) > 0.0f)) v0 = 0.0f;
            if (!(__bfloat162float(m.y) > 0.0f)) v1 = 0.0f;
          }
          if (A.y32) *reinterpret_cast<float2*>(A.y32 + p * COUT + co) = make_float2(v0, v1);
          if (A.y) *reinterpret_cast<__nv_bfloat162*>(A.y + p * COUT + co) = __floats2bfloat162_rn(v0, v1);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// tcgen05 path (volumes 128 points wide, n0 = 128): forward and input
// gradient as an implicit GEMM on the 5th-generation tensor cores.
//  - One MMA (tcgen05.mma.cta_group::1.kind::f16, BF16 operands, FP32
//    accumulation in TMEM) multiplies an input x-row, unshifted (A: M = 128
//    points x K = 16 channels), by the weights of the three x-taps of one
//    (dz, dy) stacked along N (B: N = 3 x COUT, the last layer's 24 padded
//    to 32).  Accumulated over the (dz, dy) rows and the channels, column
//    dx * COUT + c of accumulator lane p holds sum W[c][tap(dz, dy, dx)] .
//    x[p]; the epilogue forms the output as D_0[p - 1] + D_1[p] + D_2[p + 1]
//    (periodic in p), by one-lane warp shuffles and, across the four warps,
//    through shared memory.  18 MMAs per row with 32 input channels (two
//    K = 16 steps per (dz, dy) row), 6 with 8 (the K halves are two z-rows
//    of one dy: (dz 0, 1) and (dz 1 with zero weights, dz 2)).  A K = 16
//    MMA costs about the same time for N = 32 as for N = 96 on GB300, so
//    stacking the taps along N cuts the MMA time of a row threefold.
//  - Operands in shared memory, K-major without swizzle.  An input row is
//    stored channel-group-major, [channel / 8][128 points][8 channels]:
//    the 8 x 8 core matrices are 8 consecutive 16-byte point rows (128 B),
//    so the stride along M is 128 B (SBO) and the next channel group, along
//    K, is 2048 B away (LBO).  Weights: [mma][K half][N][8 channels].
//  - Input rows arrive by TMA (one box per input x-row, landing
//    channel-group-major) into a ring of y-slots x 3 z-rows indexed by a running
//    count of loaded rows, so that consecutive chunks flow through the ring
//    without draining it.
//  - Warp roles: warp 8 (one thread) issues the TMA loads, warp 9 (one
//    thread) the MMAs,
//    warps 0-7 read the accumulator (thread = point of TMEM lane quadrant
//    w % 4), combine the taps, add the bias, apply ReLU / mask and store;
//    warps 0-3 take the even rows and warps 4-7 the odd ones, so that each
//    group has two rows' time per row.  Four accumulators rotate;
//    mbarriers hand rows between the roles (an input row landed, an input
//    row's last MMAs done, a row's MMAs done, an accumulator read).  Every wait is bounded; a wait that runs out makes
//    the CTA stop issuing work and report through the error word.
namespace tc {
constexpr int M = 128;
constexpr int GROUPS = 4;      // epilogue groups of four warps (one per TMEM lane quadrant)
constexpr int EPI = GROUPS * 128;        // epilogue threads: warps 0 .. 4 GROUPS - 1
constexpr int W_LOAD = EPI / 32, W_MMA = W_LOAD + 1, W_WAIT = W_LOAD + 2;   // one-thread roles
constexpr int THREADS = EPI + 96;
constexpr int ALIGN = 1024;    // of the smem carve-up (the 64-byte swizzle repeats every 512 B)
template <int COUT>
__host__ __device__ constexpr int nt() { return COUT == 32 ? 96 : 32; }
constexpr int NBUF = 4;        // TMEM accumulators
template <int COUT>
__host__ __device__ constexpr int tmem_cols() { return COUT == 32 ? 512 : 128; }
template <int CIN>
__host__ __device__ constexpr int nmma() { return CIN == 32 ? 18 : 6; }
template <int CIN>
__host__ __device__ constexpr int row_bytes() { return M * CIN * 2; }
// y-slots of the input ring (three z-rows each): 3 in use, the rest in flight
template <int CIN>
__host__ __device__ constexpr int slots() { return CIN == 32 ? 6 : 8; }
template <int CIN, int COUT>
__host__ __device__ constexpr int w_bytes() { return nmma<CIN>() * 2 * nt<COUT>() * 16; }
// weights | ring | boundary exchange (GROUPS x 2 parities x 2 sides x 4
// quadrants x COUT floats) | barriers (full, done, freed)
template <int CIN, int COUT>
__host__ __device__ constexpr int smem_bytes() {
  return ALIGN + w_bytes<CIN, COUT>() + slots<CIN>() * 3 * row_bytes<CIN>() + GROUPS * 2 * 2 * 4 * COUT * 4 +
         8 * (2 * slots<CIN>() + 2 * NBUF) + 16;
}

// Instruction descriptor of kind::f16: D F32, A and B BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
// Shared-memory matrix descriptor (64 bits, K-major): start address >> 4 in
// bits 0-13, leading-dimension byte offset (between core matrices along K)
// >> 4 in bits 16-29, stride-dimension byte offset (between groups of eight
// rows along M or N) >> 4 in bits 32-45, the descriptor version 1 in bit 46,
// the swizzle mode in bits 61-63.
//  - sdesc: no swizzle, rows of 16 bytes 128 bytes apart per eight rows;
__host__ __device__ constexpr uint32_t sdesc_hi() { return (128u >> 4) | (1u << 14); }
//  - sdesc_sw64: 64-byte swizzle (mode 4), rows of 64 bytes (32 channels), the
//    eight-row groups 512 bytes apart; the leading offset is unused because a
//    K step of 16 channels stays inside one 64-byte row.  The K half of a
//    row is selected by adding 32 bytes to the start address: the swizzle is
//    applied to the final address bits, so the offset composes with it.
__host__ __device__ constexpr uint32_t sdesc_hi_sw64() { return (512u >> 4) | (1u << 14) | (4u << 29); }

// One MMA; the descriptors come as (low, high) 32-bit words.
__device__ __forceinline__ void mma(uint32_t d, uint32_t a_lo, uint32_t a_hi, uint32_t b_lo, uint32_t b_hi, uint32_t id,
                                    int acc) {
  asm volatile(
      "{\n .reg .pred p;\n .reg .b64 da, db;\n setp.ne.b32 p, %6, 0;\n mov.b64 da, {%1, %2};\n mov.b64 db, {%3, %4};\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %5, p;\n}\n" ::"r"(d),
      "r"(a_lo), "r"(a_hi), "r"(b_lo), "r"(b_hi), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// The output rows of a CTA: an even share of the batch x n2 x n1 rows, in
// (b, z, y) order, cut into chunks at the plane boundaries (a chunk is one
// (b, z) and consecutive y).  Every role of the CTA walks the same sequence.
struct Chunks {
  long long cur, end;
  int n1, n2;
  __device__ Chunks(long long total, int n1_, int n2_)
      : cur(total * blockIdx.x / gridDim.x), end(total * (blockIdx.x + 1) / gridDim.x), n1(n1_), n2(n2_) {}
  __device__ bool next(int& b, int& z, int& yb, int& R) {
    if (cur >= end) return false;
    const long long plane = cur / n1;
    yb = (int)(cur - plane * n1);
    R = (int)min(end - cur, (long long)(n1 - yb));
    z = (int)(plane % n2);
    b = (int)(plane / n2);
    cur += R;
    return true;
  }
};

typedef unsigned long long f2;   // two binary32 values, low word first
__device__ __forceinline__ f2 pk2(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float lo2(f2 v) { return __uint_as_float((unsigned)(v & 0xFFFFFFFFull)); }
__device__ __forceinline__ float hi2(f2 v) { return __uint_as_float((unsigned)(v >> 32)); }
// Packed addition (add.rn.f32x2): each lane rounded as the scalar addition.
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int r, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(dst), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(r), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void bar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
}  // namespace tc

template <int CIN, int COUT>
__global__ void __launch_bounds__(tc::THREADS, 1)
    k_conv3_tc(const FwdArgs A, const __grid_constant__ CUtensorMap xmap, int* err) {
  using namespace tc;
  constexpr int NT = nt<COUT>(), NM = nmma<CIN>(), RB = row_bytes<CIN>(), NG8 = COUT / 8;
  constexpr int SLOTS = slots<CIN>();
  constexpr uint32_t ID = idesc(M, NT);
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned long long sbase =
      (reinterpret_cast<unsigned long long>(smem) + (ALIGN - 1)) & ~(unsigned long long)(ALIGN - 1);
  unsigned char* Ws = reinterpret_cast<unsigned char*>(sbase);
  unsigned char* Xs = Ws + w_bytes<CIN, COUT>();
  float* bnd = reinterpret_cast<float*>(Xs + SLOTS * 3 * RB);  // [group][parity][side][quadrant][COUT]
  unsigned long long* full = reinterpret_cast<unsigned long long*>(bnd + GROUPS * 2 * 2 * 4 * COUT);
  unsigned long long* empty = full + SLOTS;    // an input row's last MMAs done
  unsigned long long* done = empty + SLOTS;    // MMAs of an accumulator committed
  unsigned long long* freed = done + NBUF;     // accumulator read by the epilogue
  uint32_t* tslot = reinterpret_cast<uint32_t*>(freed + NBUF);
  uint32_t* ready = tslot + 1;   // rows the MMA thread may start
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t ws_a = smem_u32(Ws), xs_a = smem_u32(Xs);
  // ---- weights: [mma][K half][n = dx * COUT + c][8 channels], zero outside.
  // The raw tensor is first copied with 16-byte loads into the input ring
  // (not in use yet), then packed from there one 16-byte unit per step.
  {
    constexpr int RAW = 27 * CIN * COUT;
    static_assert(RAW * 2 <= SLOTS * 3 * RB, "raw weights must fit in the ring");
    __nv_bfloat16* raw = reinterpret_cast<__nv_bfloat16*>(Xs);
    if ((reinterpret_cast<unsigned long long>(A.w) & 15ull) == 0) {
      const int4* src = reinterpret_cast<const int4*>(A.w);
      int4* dst = reinterpret_cast<int4*>(raw);
      for (int i = tid; i < RAW / 8; i += THREADS) dst[i] = __ldg(src + i);
    } else {
      for (int i = tid; i < RAW; i += THREADS) raw[i] = A.w[i];
    }
    __syncthreads();
    int4* W = reinterpret_cast<int4*>(Ws);
    for (int u = tid; u < NM * 2 * NT; u += THREADS) {
      const int n = u % NT, kh = (u / NT) % 2, j = u / (2 * NT);
      const int dx = n / COUT, co = n % COUT;
      int dz, dy, c0;
      if (CIN == 32) {
        dz = (j / 2) / 3;
        dy = (j / 2) % 3;
        c0 = 16 * (j % 2) + 8 * kh;
      } else {
        dy = j / 2;
        const int pair = j % 2;
        dz = (pair == 1 && kh == 0) ? -1 : pair + kh;
        c0 = 0;
      }
      __align__(16) __nv_bfloat16 v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = __float2bfloat16(0.0f);
      if (dx < 3 && dz >= 0) {
        const int tap = (dz * 3 + dy) * 3 + dx;
#pragma unroll
        for (int e = 0; e < 8; ++e)
          v[e] = A.flip ? raw[((c0 + e) * 27 + 26 - tap) * COUT + co] : raw[(co * 27 + tap) * CIN + c0 + e];
      }
      W[u] = *reinterpret_cast<const int4*>(v);
    }
  }
  __shared__ __align__(16) float sbias[COUT];
  if (tid < COUT) sbias[tid] = A.bias ? A.bias[tid] : 0.0f;
  if (tid == 0) {
    for (int q = 0; q < SLOTS; ++q) {
      bar_init(smem_u32(&full[q]), 1);
      bar_init(smem_u32(&empty[q]), 1);
    }
    for (int q = 0; q < NBUF; ++q) {
      bar_init(smem_u32(&done[q]), 1);
      bar_init(smem_u32(&freed[q]), 4);   // one arrival per warp of a group
    }
    *ready = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(tmem_cols<COUT>()));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // weights -> tensor core
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const int n1 = A.v.n1, n2 = A.v.n2;
  const long long nrows = (long long)A.v.batch * n2 * n1;
  if (warp == W_LOAD) {
    // ================= TMA loads (one thread): every input row of every
    // chunk, in order; load L goes into slot L mod SLOTS once the MMAs that
    // read the slot's previous row are done
    if (lane == 0) {
      int q = 0, L = 0;
      unsigned ph = 0;   // parity of the slot's previous load, wrapped once the ring has filled
      bool stop = false;
      Chunks ch(nrows, n1, n2);
      int b, z, yb, R;
      while (!stop && ch.next(b, z, yb, R)) {
        for (int u = 0; u < R + 2; ++u, ++L) {
          if (L >= SLOTS && !bar_wait(smem_u32(&empty[q]), ph)) {
            stop = true;
            break;
          }
          const uint32_t bar = smem_u32(&full[q]);
          bar_expect_tx(bar, 3 * RB);
          const int yy = wrap1(yb - 1 + u, n1);
#pragma unroll
          for (int dz = 0; dz < 3; ++dz) {
            const int row = ((b * n2) + wrap1(z + dz - 1, n2)) * n1 + yy;
            tma_load_3d(xs_a + (uint32_t)((q * 3 + dz) * RB), &xmap, 0, 0, row, bar);
          }
          if (++q == SLOTS) {
            q = 0;
            if (L >= SLOTS) ph ^= 1u;
          }
        }
      }
      if (stop) {
        if (err) atomicOr(err, ERR_TIMEOUT);
        // the copies still in flight land (bounded) before the CTA exits
        for (int l = L - SLOTS; l < L; ++l)
          if (l >= 0) bar_wait(smem_u32(&full[l % SLOTS]), (unsigned)((l / SLOTS) & 1));
      }
    }
  } else if (warp == W_WAIT) {
    // ================= waits on behalf of the MMA thread (one thread): a
    // row may start once its last input row has landed and its accumulator
    // has been read; the count of such rows goes to `ready`.  The MMA
    // thread then polls one shared word instead of two mbarriers, which
    // keeps the tensor core's short queue fed.
    if (lane == 0) {
      int qf = 0, bf = 0;
      unsigned pf = 0, pb = 0;
      unsigned grow = 0;
      bool stop = false;
      Chunks ch(nrows, n1, n2);
      int b, z, yb, R;
      while (!stop && ch.next(b, z, yb, R)) {
        for (int r = 0; r < R && !stop; ++r, ++grow) {
          // input rows r, r + 1, r + 2 of the chunk: all three for the
          // chunk's first row, then the one new row (R + 2 loads a chunk)
          for (int k = (r == 0 ? 3 : 1); k > 0; --k) {
            if (!bar_wait(smem_u32(&full[qf]), pf)) {
              stop = true;
              break;
            }
            if (++qf == SLOTS) qf = 0, pf ^= 1u;
          }
          if (!stop && grow >= (unsigned)NBUF && !bar_wait(smem_u32(&freed[bf]), pb)) stop = true;
          if (++bf == NBUF) {
            bf = 0;
            if (grow >= (unsigned)NBUF) pb ^= 1u;
          }
          if (!stop)
            asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(smem_u32(ready)), "r"(grow + 1) : "memory");
        }
      }
      if (stop) {
        asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(smem_u32(ready)), "r"(0xffffffffu) : "memory");
        if (err) atomicOr(err, ERR_TIMEOUT);
      }
    }
  } else if (warp == W_MMA) {
    // ================= MMAs (one thread)
    if (lane == 0) {
      // descriptor words: the high halves are constant, the low halves are
      // the start address >> 4 plus the leading offset, so an operand at a
      // byte offset is the base word plus offset >> 4
      constexpr uint32_t A_HI = CIN == 32 ? sdesc_hi_sw64() : sdesc_hi();
      constexpr uint32_t A_LBO = CIN == 32 ? (1u << 16) : ((uint32_t)(RB >> 4) << 16);
      constexpr uint32_t B_HI = sdesc_hi();
      const uint32_t b_lo0 = (ws_a >> 4) | ((uint32_t)((NT * 16) >> 4) << 16);
      int q0 = 0;   // slot of the chunk's current first input row
      unsigned grow = 0;
      bool stop = false;
      Chunks ch(nrows, n1, n2);
      int b, z, yb, R;
      while (!stop && ch.next(b, z, yb, R)) {
        for (int r = 0; r < R; ++r, ++grow) {
          bool ok = false;
          for (unsigned it = 0; it < WAIT_LIMIT; ++it) {
            unsigned v;
            asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_u32(ready)) : "memory");
            if (v == 0xffffffffu) break;
            if (v > grow) {
              ok = true;
              break;
            }
          }
          if (!ok) {
            stop = true;
            break;
          }
          const int q1 = q0 + 1 == SLOTS ? 0 : q0 + 1, q2 = q1 + 1 == SLOTS ? 0 : q1 + 1;
          const uint32_t a_lo[3] = {((xs_a + (uint32_t)(q0 * 3 * RB)) >> 4) | A_LBO,
                                    ((xs_a + (uint32_t)(q1 * 3 * RB)) >> 4) | A_LBO,
                                    ((xs_a + (uint32_t)(q2 * 3 * RB)) >> 4) | A_LBO};
          const int buf = (int)(grow & (NBUF - 1));
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t d = tmem + (uint32_t)(buf * NT);
#pragma unroll
          for (int j = 0; j < NM; ++j) {
            const int dy = CIN == 32 ? (j / 2) % 3 : j / 2;
            const int dz = CIN == 32 ? (j / 2) / 3 : j % 2;       // dz of the first K half
            const uint32_t off = (uint32_t)(dz * RB + (CIN == 32 ? 32 * (j % 2) : 0));
            mma(d, a_lo[dy] + (off >> 4), A_HI, b_lo0 + (uint32_t)((j * 2 * NT * 16) >> 4), B_HI, ID, j > 0);
          }
          commit(smem_u32(&done[buf]));
          // input row r is read by no later row of the chunk; the chunk's
          // last row also retires rows R and R + 1
          commit(smem_u32(&empty[q0]));
          if (r == R - 1) {
            commit(smem_u32(&empty[q1]));
            commit(smem_u32(&empty[q2]));
          }
          q0 = q1;
        }
        // past the chunk's last two input rows
        q0 = q0 + 2 >= SLOTS ? q0 + 2 - SLOTS : q0 + 2;
      }
      if (stop && err) atomicOr(err, ERR_TIMEOUT);
    }
  } else {
    // ================= epilogue: thread = point p of the row; group
    // `grp` takes the rows g with g mod GROUPS = grp, always in accumulator
    // grp.  Registers: D_0 and D_2 first (their sum needs the exchange across
    // the quadrants), D_1 after, so that at most two of the three are live.
    const int quad = warp & 3, grp = warp >> 2;
    const int p = 32 * quad + lane;
    const int src_l = (lane + 31) & 31, src_r = (lane + 1) & 31;
    long long grow = 0;
    bool stop = false;
    Chunks ch(nrows, n1, n2);
    int b, z, yb, R;
    while (!stop && ch.next(b, z, yb, R)) {
      for (int r = 0; r < R; ++r, ++grow) {
        if ((int)(grow % GROUPS) != grp) continue;
        const int buf = (int)(grow & (NBUF - 1));
        // the group's threads stop together if any wait ran out, so that
        // none is left at a named barrier
        const unsigned ok = bar_wait(smem_u32(&done[buf]), (unsigned)((grow / NBUF) & 1)) ? 1u : 0u;
        int any_fail;
        asm volatile("{\n .reg .pred p, q;\n setp.eq.u32 q, %1, 0;\n bar.red.or.pred p, %2, 128, q;\n selp.s32 %0, 1, 0, p;\n}\n"
                     : "=r"(any_fail) : "r"(ok), "r"(1 + grp) : "memory");
        if (any_fail) {
          stop = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        float d0[COUT], d2[COUT];
        const uint32_t t0 = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(buf * NT);
        if constexpr (COUT == 32) {
          ld32(t0, d0);
          ld32(t0 + 64u, d2);
        } else {
          ld8(t0, d0);
          ld8(t0 + 16u, d2);
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        // D_0 of the quadrant's last point and D_2 of its first, for the
        // neighbouring quadrants (periodic in p); two buffers alternate
        // between the group's rows
        float* bq = bnd + ((grp * 2 + (int)((grow / GROUPS) & 1)) * 2) * 4 * COUT;
        if (lane == 31)
#pragma unroll
          for (int n = 0; n < COUT; n += 4)
            *reinterpret_cast<float4*>(bq + quad * COUT + n) = make_float4(d0[n], d0[n + 1], d0[n + 2], d0[n + 3]);
        if (lane == 0)
#pragma unroll
          for (int n = 0; n < COUT; n += 4)
            *reinterpret_cast<float4*>(bq + 4 * COUT + quad * COUT + n) = make_float4(d2[n], d2[n + 1], d2[n + 2], d2[n + 3]);
        asm volatile("bar.sync %0, 128;" ::"r"(1 + GROUPS + grp) : "memory");
        // Lane 31's D_0 and lane 0's D_2 feed only the neighbouring
        // quadrants' outputs, so those registers now take the values coming
        // in: lane 31 the D_0 of point 32 quad - 1, lane 0 the D_2 of point
        // 32 quad + 32.  A rotation by one lane then hands every lane its
        // D_0[p - 1] and D_2[p + 1] with no per-lane selection.
        if (lane == 31) {
          const float* e = bq + ((quad + 3) & 3) * COUT;
#pragma unroll
          for (int n = 0; n < COUT; n += 4) {
            const float4 t = *reinterpret_cast<const float4*>(e + n);
            d0[n] = t.x, d0[n + 1] = t.y, d0[n + 2] = t.z, d0[n + 3] = t.w;
          }
        }
        if (lane == 0) {
          const float* e = bq + 4 * COUT + ((quad + 1) & 3) * COUT;
#pragma unroll
          for (int n = 0; n < COUT; n += 4) {
            const float4 t = *reinterpret_cast<const float4*>(e + n);
            d2[n] = t.x, d2[n + 1] = t.y, d2[n + 2] = t.z, d2[n + 3] = t.w;
          }
        }
        // s = D_0[p - 1] + D_2[p + 1], two channels at once (into d0)
#pragma unroll
        for (int n = 0; n < COUT; n += 2) {
          const float l0 = __shfl_sync(0xffffffffu, d0[n], src_l), l1 = __shfl_sync(0xffffffffu, d0[n + 1], src_l);
          const float r0 = __shfl_sync(0xffffffffu, d2[n], src_r), r1 = __shfl_sync(0xffffffffu, d2[n + 1], src_r);
          const f2 t = add2(pk2(l0, l1), pk2(r0, r1));
          d0[n] = lo2(t);
          d0[n + 1] = hi2(t);
        }
        // D_1, then the accumulator is free
        float d1[COUT];
        if constexpr (COUT == 32)
          ld32(t0 + 32u, d1);
        else
          ld8(t0 + 8u, d1);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) bar_arrive(smem_u32(&freed[buf]));
        const long long pi = point_index(A.v, b, z, yb + r, p);
#pragma unroll
        for (int g = 0; g < NG8; ++g) {
          const float4 b0 = *reinterpret_cast<const float4*>(sbias + 8 * g);
          const float4 b1 = *reinterpret_cast<const float4*>(sbias + 8 * g + 4);
          const float bs[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
          float v[8];
#pragma unroll
          for (int e = 0; e < 8; e += 2) {
            const int n = 8 * g + e;
            // (D_0[p - 1] + D_2[p + 1]) + (D_1[p] + bias)
            const f2 t = add2(pk2(d0[n], d0[n + 1]), add2(pk2(d1[n], d1[n + 1]), pk2(bs[e], bs[e + 1])));
            v[e] = lo2(t);
            v[e + 1] = hi2(t);
          }
          if (A.relu)
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = fmaxf(v[e], 0.0f);
          if (A.mask) {
            const int4 mk = *reinterpret_cast<const int4*>(A.mask + pi * COUT + 8 * g);
            const __nv_bfloat16* mb = reinterpret_cast<const __nv_bfloat16*>(&mk);
#pragma unroll
            for (int e = 0; e < 8; ++e)
              if (!(__bfloat162float(mb[e]) > 0.0f)) v[e] = 0.0f;
          }
          if (A.y32) {
            *reinterpret_cast<float4*>(A.y32 + pi * COUT + 8 * g) = make_float4(v[0], v[1], v[2], v[3]);
            *reinterpret_cast<float4*>(A.y32 + pi * COUT + 8 * g + 4) = make_float4(v[4], v[5], v[6], v[7]);
          }
          if (A.y) {
            int4 o;
            __nv_bfloat162* ob = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
            for (int e = 0; e < 4; ++e) ob[e] = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
            *reinterpret_cast<int4*>(A.y + pi * COUT + 8 * g) = o;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols<COUT>()));
}

// ---------------------------------------------------------------------------
// tcgen05 path for 32 input and 8 output channels: the y- and x-taps of one
// dz stacked along N (9 x 8 = 72 columns, padded to 80), so that an input
// row takes 6 MMAs (3 dz x 2 K halves) instead of the 18 N = 32 MMAs per
// output row of k_conv3_tc, whose N is a third used.  The accumulator of an
// input row yy holds, in column block dy, its contributions to output row
// yy - dy + 1: output row y sums block 0 of the accumulator of row y - 1,
// block 1 of row y and block 2 of row y + 1, then the x-taps as in
// k_conv3_tc.  Accumulators rotate over NA TMEM slots; a slot is freed once
// the three output rows that read it have (the first reader of a chunk's
// edge row arrives for the readers it lacks).  Every input row now feeds
// one MMA group, so its ring slot is released as soon as that group is done.
namespace tcy {
constexpr int CIN = 32, COUT = 8, NT = 80, NM = 6, NA = 6, SLOTS = 8;
constexpr int RB = tc::M * CIN * 2;
constexpr int W_BYTES = NM * 2 * NT * 16;
constexpr int SMEM = tc::ALIGN + W_BYTES + SLOTS * 3 * RB + tc::GROUPS * 2 * 2 * 4 * COUT * 4 + 8 * (2 * SLOTS + 2 * NA) +
                     16;
}  // namespace tcy

__global__ void __launch_bounds__(tc::THREADS, 1)
    k_conv3_tc_yx(const FwdArgs A, const __grid_constant__ CUtensorMap xmap, int* err) {
  using namespace tc;
  using tcy::CIN;
  using tcy::COUT;
  using tcy::NA;
  using tcy::NM;
  using tcy::NT;
  using tcy::RB;
  using tcy::SLOTS;
  constexpr uint32_t ID = idesc(M, NT);
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned long long sbase =
      (reinterpret_cast<unsigned long long>(smem) + (ALIGN - 1)) & ~(unsigned long long)(ALIGN - 1);
  unsigned char* Ws = reinterpret_cast<unsigned char*>(sbase);
  unsigned char* Xs = Ws + tcy::W_BYTES;
  float* bnd = reinterpret_cast<float*>(Xs + SLOTS * 3 * RB);  // [group][parity][side][quadrant][COUT]
  unsigned long long* full = reinterpret_cast<unsigned long long*>(bnd + GROUPS * 2 * 2 * 4 * COUT);
  unsigned long long* empty = full + SLOTS;  // an input row's MMAs done
  unsigned long long* done = empty + SLOTS;  // an accumulator's MMAs committed
  unsigned long long* freed = done + NA;     // an accumulator read by its three output rows
  uint32_t* tslot = reinterpret_cast<uint32_t*>(freed + NA);
  uint32_t* ready = tslot + 1;  // input rows the MMA thread may start
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t ws_a = smem_u32(Ws), xs_a = smem_u32(Xs);
  // ---- weights: [mma j = 2 dz + K half][8-channel group][n = 24 dy + 8 dx + c][8 channels]
  {
    constexpr int RAW = 27 * CIN * COUT;
    static_assert(RAW * 2 <= SLOTS * 3 * RB, "raw weights must fit in the ring");
    __nv_bfloat16* raw = reinterpret_cast<__nv_bfloat16*>(Xs);
    if ((reinterpret_cast<unsigned long long>(A.w) & 15ull) == 0) {
      const int4* src = reinterpret_cast<const int4*>(A.w);
      int4* dst = reinterpret_cast<int4*>(raw);
      for (int i = tid; i < RAW / 8; i += THREADS) dst[i] = __ldg(src + i);
    } else {
      for (int i = tid; i < RAW; i += THREADS) raw[i] = A.w[i];
    }
    __syncthreads();
    int4* W = reinterpret_cast<int4*>(Ws);
    for (int u = tid; u < NM * 2 * NT; u += THREADS) {
      const int n = u % NT, kh = (u / NT) % 2, j = u / (2 * NT);
      const int dz = j / 2, c0 = 16 * (j % 2) + 8 * kh;
      __align__(16) __nv_bfloat16 v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = __float2bfloat16(0.0f);
      if (n < 9 * COUT) {
        const int dy = n / (3 * COUT), dx = (n / COUT) % 3, co = n % COUT;
        const int tap = (dz * 3 + dy) * 3 + dx;
#pragma unroll
        for (int e = 0; e < 8; ++e)
          v[e] = A.flip ? raw[((c0 + e) * 27 + 26 - tap) * COUT + co] : raw[(co * 27 + tap) * CIN + c0 + e];
      }
      W[u] = *reinterpret_cast<const int4*>(v);
    }
  }
  __shared__ __align__(16) float sbias[COUT];
  if (tid < COUT) sbias[tid] = A.bias ? A.bias[tid] : 0.0f;
  if (tid == 0) {
    for (int q = 0; q < SLOTS; ++q) {
      bar_init(smem_u32(&full[q]), 1);
      bar_init(smem_u32(&empty[q]), 1);
    }
    for (int q = 0; q < NA; ++q) {
      bar_init(smem_u32(&done[q]), 1);
      bar_init(smem_u32(&freed[q]), 3 * 4);   // three output rows, one arrival per warp of a group
    }
    *ready = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const int n1 = A.v.n1, n2 = A.v.n2;
  const long long nrows = (long long)A.v.batch * n2 * n1;
  if (warp == W_LOAD) {
    // ================= TMA loads: every input row of every chunk, in order
    if (lane == 0) {
      int q = 0, L = 0;
      unsigned ph = 0;
      bool stop = false;
      Chunks ch(nrows, n1, n2);
      int b, z, yb, R;
      while (!stop && ch.next(b, z, yb, R)) {
        for (int u = 0; u < R + 2; ++u, ++L) {
          if (L >= SLOTS && !bar_wait(smem_u32(&empty[q]), ph)) {
            stop = true;
            break;
          }
          const uint32_t bar = smem_u32(&full[q]);
          bar_expect_tx(bar, 3 * RB);
          const int yy = wrap1(yb - 1 + u, n1);
#pragma unroll
          for (int dz = 0; dz < 3; ++dz) {
            const int row = ((b * n2) + wrap1(z + dz - 1, n2)) * n1 + yy;
            tma_load_3d(xs_a + (uint32_t)((q * 3 + dz) * RB), &xmap, 0, 0, row, bar);
          }
          if (++q == SLOTS) {
            q = 0;
            if (L >= SLOTS) ph ^= 1u;
          }
        }
      }
      if (stop) {
        if (err) atomicOr(err, ERR_TIMEOUT);
        for (int l = L - SLOTS; l < L; ++l)
          if (l >= 0) bar_wait(smem_u32(&full[l % SLOTS]), (unsigned)((l / SLOTS) & 1));
      }
    }
  } else if (warp == W_WAIT) {
    // ================= waits for the MMA thread: input row L may start once
    // it has landed and its accumulator slot's previous row has been read
    if (lane == 0) {
      int qf = 0, af = 0;
      unsigned pf = 0, pa = 0, L = 0;
      bool stop = false;
      Chunks ch(nrows, n1, n2);
      int b, z, yb, R;
      while (!stop && ch.next(b, z, yb, R)) {
        for (int u = 0; u < R + 2 && !stop; ++u, ++L) {
          if (!bar_wait(smem_u32(&full[qf]), pf)) stop = true;
          if (++qf == SLOTS) qf = 0, pf ^= 1u;
          if (!stop && L >= (unsigned)NA && !bar_wait(smem_u32(&freed[af]), pa)) stop = true;
          if (++af == NA) {
            af = 0;
            if (L >= (unsigned)NA) pa ^= 1u;
          }
          if (!stop)
            asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(smem_u32(ready)), "r"(L + 1) : "memory");
        }
      }
      if (stop) {
        asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(smem_u32(ready)), "r"(0xffffffffu) : "memory");
        if (err) atomicOr(err, ERR_TIMEOUT);
      }
    }
  } else if (warp == W_MMA) {
    // ================= MMAs (one thread): 6 per input row
    if (lane == 0) {
      constexpr uint32_t A_HI = sdesc_hi_sw64(), B_HI = sdesc_hi();
      const uint32_t b_lo0 = (ws_a >> 4) | ((uint32_t)((NT * 16) >> 4) << 16);
      int q = 0, a = 0;
      unsigned L = 0;
      bool stop = false;
      Chunks ch(nrows, n1, n2);
      int b, z, yb, R;
      while (!stop && ch.next(b, z, yb, R)) {
        for (int u = 0; u < R + 2; ++u, ++L) {
          bool ok = false;
          for (unsigned it = 0; it < WAIT_LIMIT; ++it) {
            unsigned v;
            asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_u32(ready)) : "memory");
            if (v == 0xffffffffu) break;
            if (v > L) {
              ok = true;
              break;
            }
          }
          if (!ok) {
            stop = true;
            break;
          }
          const uint32_t a_lo = ((xs_a + (uint32_t)(q * 3 * RB)) >> 4) | (1u << 16);
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t d = tmem + (uint32_t)(a * NT);
#pragma unroll
          for (int j = 0; j < NM; ++j) {
            const uint32_t off = (uint32_t)((j / 2) * RB + 32 * (j % 2));
            mma(d, a_lo + (off >> 4), A_HI, b_lo0 + (uint32_t)((j * 2 * NT * 16) >> 4), B_HI, ID, j > 0);
          }
          commit(smem_u32(&done[a]));
          commit(smem_u32(&empty[q]));
          if (++q == SLOTS) q = 0;
          if (++a == NA) a = 0;
        }
      }
      if (stop && err) atomicOr(err, ERR_TIMEOUT);
    }
  } else {
    // ================= epilogue: group `grp` takes the output rows g with
    // g mod GROUPS = grp; thread = point p of the row
    const int quad = warp & 3, grp = warp >> 2;
    const int p = 32 * quad + lane;
    const int src_l = (lane + 31) & 31, src_r = (lane + 1) & 31;
    long long grow = 0;
    unsigned L0 = 0;   // the chunk's first input row (load index)
    bool stop = false;
    Chunks ch(nrows, n1, n2);
    int b, z, yb, R;
    while (!stop && ch.next(b, z, yb, R)) {
      for (int r = 0; r < R; ++r, ++grow) {
        if ((int)(grow % GROUPS) != grp) continue;
        const unsigned u2 = L0 + (unsigned)r + 2;   // the last of the three accumulators
        const unsigned ok = bar_wait(smem_u32(&done[u2 % NA]), (u2 / NA) & 1u) ? 1u : 0u;
        int any_fail;
        asm volatile("{\n .reg .pred p, q;\n setp.eq.u32 q, %1, 0;\n bar.red.or.pred p, %2, 128, q;\n selp.s32 %0, 1, 0, p;\n}\n"
                     : "=r"(any_fail) : "r"(ok), "r"(1 + grp) : "memory");
        if (any_fail) {
          stop = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // E[dx][c] = block 0 of row r, block 1 of row r + 1, block 2 of row r + 2
        float e[3][COUT];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const uint32_t t0 = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(((L0 + r + k) % NA) * NT + k * 3 * COUT);
          float v0[COUT], v1[COUT], v2[COUT];
          ld8(t0, v0);
          ld8(t0 + 8u, v1);
          ld8(t0 + 16u, v2);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int c = 0; c < COUT; ++c) {
            e[0][c] = k == 0 ? v0[c] : e[0][c] + v0[c];
            e[1][c] = k == 0 ? v1[c] : e[1][c] + v1[c];
            e[2][c] = k == 0 ? v2[c] : e[2][c] + v2[c];
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            // readers of chunk row uc: the output rows max(0, uc - 2) .. min(R - 1, uc);
            // the first of them arrives for the ones the chunk lacks
            const int uc = r + k, first = uc - 2 > 0 ? uc - 2 : 0, last = uc < R - 1 ? uc : R - 1;
            const unsigned cnt = r == first ? (unsigned)(1 + 3 - (last - first + 1)) : 1u;
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&freed[(L0 + r + k) % NA])),
                         "r"(cnt) : "memory");
          }
        }
        float* bq = bnd + ((grp * 2 + (int)((grow / GROUPS) & 1)) * 2) * 4 * COUT;
        if (lane == 31)
#pragma unroll
          for (int c = 0; c < COUT; c += 4)
            *reinterpret_cast<float4*>(bq + quad * COUT + c) = make_float4(e[0][c], e[0][c + 1], e[0][c + 2], e[0][c + 3]);
        if (lane == 0)
#pragma unroll
          for (int c = 0; c < COUT; c += 4)
            *reinterpret_cast<float4*>(bq + 4 * COUT + quad * COUT + c) =
                make_float4(e[2][c], e[2][c + 1], e[2][c + 2], e[2][c + 3]);
        asm volatile("bar.sync %0, 128;" ::"r"(1 + GROUPS + grp) : "memory");
        // as in k_conv3_tc: the edge lanes take the neighbouring quadrants'
        // values, then one-lane rotations combine the x-taps
        if (lane == 31) {
          const float* ep = bq + ((quad + 3) & 3) * COUT;
#pragma unroll
          for (int c = 0; c < COUT; c += 4) {
            const float4 t = *reinterpret_cast<const float4*>(ep + c);
            e[0][c] = t.x, e[0][c + 1] = t.y, e[0][c + 2] = t.z, e[0][c + 3] = t.w;
          }
        }
        if (lane == 0) {
          const float* ep = bq + 4 * COUT + ((quad + 1) & 3) * COUT;
#pragma unroll
          for (int c = 0; c < COUT; c += 4) {
            const float4 t = *reinterpret_cast<const float4*>(ep + c);
            e[2][c] = t.x, e[2][c + 1] = t.y, e[2][c + 2] = t.z, e[2][c + 3] = t.w;
          }
        }
        const long long pi = point_index(A.v, b, z, yb + r, p);
        float v[COUT];
#pragma unroll
        for (int c = 0; c < COUT; c += 2) {
          const float l0 = __shfl_sync(0xffffffffu, e[0][c], src_l), l1 = __shfl_sync(0xffffffffu, e[0][c + 1], src_l);
          const float r0 = __shfl_sync(0xffffffffu, e[2][c], src_r), r1 = __shfl_sync(0xffffffffu, e[2][c + 1], src_r);
          // (E_0[p - 1] + E_2[p + 1]) + (E_1[p] + bias)
          const f2 t = add2(add2(pk2(l0, l1), pk2(r0, r1)), add2(pk2(e[1][c], e[1][c + 1]), pk2(sbias[c], sbias[c + 1])));
          v[c] = lo2(t);
          v[c + 1] = hi2(t);
        }
        if (A.relu)
#pragma unroll
          for (int c = 0; c < COUT; ++c) v[c] = fmaxf(v[c], 0.0f);
        if (A.mask) {
          const int4 mk = *reinterpret_cast<const int4*>(A.mask + pi * COUT);
          const __nv_bfloat16* mb = reinterpret_cast<const __nv_bfloat16*>(&mk);
#pragma unroll
          for (int c = 0; c < COUT; ++c)
            if (!(__bfloat162float(mb[c]) > 0.0f)) v[c] = 0.0f;
        }
        if (A.y32) {
          *reinterpret_cast<float4*>(A.y32 + pi * COUT) = make_float4(v[0], v[1], v[2], v[3]);
          *reinterpret_cast<float4*>(A.y32 + pi * COUT + 4) = make_float4(v[4], v[5], v[6], v[7]);
        }
        if (A.y) {
          int4 o;
          __nv_bfloat162* ob = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
          for (int c = 0; c < 4; ++c) ob[c] = __floats2bfloat162_rn(v[2 * c], v[2 * c + 1]);
          *reinterpret_cast<int4*>(A.y + pi * COUT) = o;
        }
      }
      L0 += (unsigned)R + 2;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

struct WgArgs {
  const __nv_bfloat16* x;  // layer input [..][CIN]
  const __nv_bfloat16* g;  // gradient at the layer output [..][COUT]
  float* part;             // [gridDim.x][COUT * 27 * CIN + COUT]
  Vol v;
  long long nblocks;
};

// Weight and bias gradient partials of one CTA.  Jobs (tap, 16 output
// channels) are spread over the warps; a job keeps CIN / 8 accumulator tiles.
template <int CIN, int COUT>
__global__ void __launch_bounds__(WG_THREADS) k_conv3_wgrad(const WgArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int XS = xstride<CIN>(), GS = COUT + 8;
  constexpr int MT = (COUT + 15) / 16, NT = CIN / 8, JOBS = 27 * MT, JPW = (JOBS + WG_WARPS - 1) / WG_WARPS;
  __nv_bfloat16* Xs = reinterpret_cast<__nv_bfloat16*>(smem);
  __nv_bfloat16* Gs = Xs + HPTS * XS;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gq = lane >> 2, t = lane & 3;
  float acc[JPW][NT][4];
#pragma unroll
  for (int i = 0; i < JPW; ++i)
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[i][j][0] = acc[i][j][1] = acc[i][j][2] = acc[i][j][3] = 0.0f;
  float bsum = 0.0f;
  for (long long blk = blockIdx.x; blk < A.nblocks; blk += gridDim.x) {
    int b, z, y0, x0;
    block_origin(blk, A.v, b, z, y0, x0);
    __syncthreads();
    stage_halo<CIN>(Xs, A.x, A.v, b, z, y0, x0);
    constexpr int GCH = COUT / 8;
    for (int i = threadIdx.x; i < BX * BY * GCH; i += blockDim.x) {
      const int q = i / GCH, ch = i - q * GCH, r = q / BX, m = q - r * BX;
      const long long p = point_index(A.v, b, z, y0 + r, x0 + m);
      *reinterpret_cast<int4*>(Gs + q * GS + ch * 8) = *reinterpret_cast<const int4*>(A.g + p * COUT + ch * 8);
    }
    __syncthreads();
    if (threadIdx.x < COUT)
      for (int q = 0; q < BX * BY; ++q) bsum += __bfloat162float(Gs[q * GS + threadIdx.x]);
#pragma unroll
    for (int i = 0; i < JPW; ++i) {
      const int job = warp + WG_WARPS * i;
      if (job >= JOBS) break;  // warp-uniform
      const int tap = job / MT, mt = job - tap * MT;
      const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
      const int co = 16 * mt + gq;
      for (int s = 0; s < BY; ++s) {
        // A[m = channel][k = point of row s]: rows co, co + 8; points 2t, 2t+1 (+8)
        uint32_t a[4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int q = s * BX + 2 * t + 8 * h;
          a[2 * h] = pack2(Gs[q * GS + co], Gs[(q + 1) * GS + co]);
          a[2 * h + 1] = co + 8 < COUT ? pack2(Gs[q * GS + co + 8], Gs[(q + 1) * GS + co + 8]) : 0u;
        }
        // B[k = point][n = input channel 8 nt + gq], the point shifted by the tap
        const int hp = (dz * HY + s + dy) * HX + 2 * t + dx;
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          const int ci = 8 * nt + gq;
          const uint32_t b0 = pack2(Xs[hp * XS + ci], Xs[(hp + 1) * XS + ci]);
          const uint32_t b1 = pack2(Xs[(hp + 8) * XS + ci], Xs[(hp + 9) * XS + ci]);
          mma_bf16(acc[i][nt], a[0], a[1], a[2], a[3], b0, b1);
        }
      }
    }
  }
  float* P = A.part + (long long)blockIdx.x * (COUT * 27 * CIN + COUT);
#pragma unroll
  for (int i = 0; i < JPW; ++i) {
    const int job = warp + WG_WARPS * i;
    if (job >= JOBS) break;
    const int tap = job / MT, mt = job - tap * MT, co = 16 * mt + gq;
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      const int ci = 8 * nt + 2 * t;
      P[((long long)co * 27 + tap) * CIN + ci] = acc[i][nt][0];
      P[((long long)co * 27 + tap) * CIN + ci + 1] = acc[i][nt][1];
      if (co + 8 < COUT) {
        P[((long long)(co + 8) * 27 + tap) * CIN + ci] = acc[i][nt][2];
        P[((long long)(co + 8) * 27 + tap) * CIN + ci + 1] = acc[i][nt][3];
      }
    }
  }
  if (threadIdx.x < COUT) P[COUT * 27 * CIN + threadIdx.x] = bsum;
}

// out[i] = sum over the partials in index order (gw for i < nw, then gb)
__global__ void k_sum_parts(const float* part, int nparts, int len, int nw, float* gw, float* gb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  float s = 0.0f;
  for (int c = 0; c < nparts; ++c) s += part[(long long)c * len + i];
  if (i < nw)
    gw[i] = s;
  else
    gb[i - nw] = s;
}

__global__ void k_adam(float* w, __nv_bfloat16* w16, const float* g, float* m, float* v, long long n, float lr_c1,
                       float c2, float b1, float b2, float eps) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr_c1 * mi / (sqrtf(vi * c2) + eps);
    w[i] = wi;
    if (w16) w16[i] = __float2bfloat16_rn(wi);
  }
}

__global__ void k_mse(const float* y, int cy, const float* t, int used, long long points, __nv_bfloat16* gy,
                      double* loss, float gscale, double inv) {
  double local = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < points;
       p += (long long)gridDim.x * blockDim.x) {
    for (int c = 0; c < cy; ++c) {
      const float d = c < used ? y[p * cy + c] - t[p * used + c] : 0.0f;
      gy[p * cy + c] = __float2bfloat16_rn(gscale * d);
      local += (double)d * d;
    }
  }
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if (loss && (threadIdx.x & 31) == 0) atomicAdd(loss, local * inv);
}

}  // namespace
}  // namespace mpw

// ============================================================================ host side

namespace {
using namespace mpw;

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

int sm_count() {
  int d = 0, n = 0;
  if (cudaGetDevice(&d) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// shapes the kernels are instantiated for: (8, 32), (32, 32), (32, 8)
bool supported(int cin, int cout) {
  return (cin == 8 || cin == 32) && (cout == 8 || cout == 32) && !(cin == 8 && cout == 8);
}

mpw_status check_volume(int batch, const int n[3], Vol& v, long long& nblocks) {
  if (!n || batch < 1 || n[0] < 16 || n[1] < 8 || n[2] < 3 || n[0] % BX || n[1] % BY)
    return fail(MPW_ERR_ARG, "conv3: volume must have n0 % 16 == 0, n1 % 8 == 0, n2 >= 3 and batch >= 1");
  v = Vol{n[0], n[1], n[2], batch};
  nblocks = (long long)batch * n[2] * (n[1] / BY) * (n[0] / BX);
  return MPW_OK;
}

template <int CIN, int COUT>
cudaError_t launch_conv(FwdArgs a, cudaStream_t s) {
  const int smem = (COUT * wstride<CIN>() + HPTS2 * xstride<CIN>()) * 2;
  cudaError_t e = cudaFuncSetAttribute(k_conv3_t<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  a.nblocks = (long long)a.v.batch * ((a.v.n2 + 1) / 2) * (a.v.n1 / BY) * (a.v.n0 / BX);
  const long long grid = a.nblocks < 2LL * sm_count() ? a.nblocks : 2LL * sm_count();
  k_conv3_t<CIN, COUT><<<(unsigned)grid, FWD_THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

// Which forward kernel serves a launch: 0 = tcgen05 wherever the volume is
// 128 points wide, mma.sync otherwise; 1 = mma.sync always (mpw_conv3_select).
int g_conv_kernel = 0;

// TMA map of a channels-last BF16 volume of CIN channels and 128-point rows,
// with the dimensions ordered (8 channels, 128 points, CIN / 8 groups, rows)
// so that one box, a whole x-row, lands channel-group-major in shared memory
// ([group][point][8 channels]).
bool encode_act_map(CUtensorMap* map, const void* x, int cin, const Vol& v) {
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  if (!encode) return false;
  // One box is one x-row of 128 points.  With 32 channels a point is one
  // 64-byte line, swizzled on the way in; with 8 channels the row is a
  // contiguous 2 KB, fetched as 16 lines of 128 bytes (eight points each).
  const cuuint64_t rows = (cuuint64_t)v.n1 * v.n2 * v.batch;
  const bool wide = cin == 32;
  const cuuint64_t dims[3] = {wide ? 32u : 64u, wide ? (cuuint64_t)v.n0 : (cuuint64_t)v.n0 / 8, rows};
  const cuuint64_t strides[2] = {wide ? 64u : 128u, (cuuint64_t)v.n0 * cin * 2};
  const cuuint32_t box[3] = {wide ? 32u : 64u, wide ? (cuuint32_t)tc::M : (cuuint32_t)tc::M / 8, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(x), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, wide ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int CIN, int COUT>
cudaError_t launch_conv_tc(const FwdArgs& a, cudaStream_t s) {
  constexpr int smem = tc::smem_bytes<CIN, COUT>();
  CUtensorMap map;
  if (!encode_act_map(&map, a.x, CIN, a.v)) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_conv3_tc<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const long long rows = (long long)a.v.batch * a.v.n2 * a.v.n1;
  const long long grid = rows < sm_count() ? rows : sm_count();
  k_conv3_tc<CIN, COUT><<<(unsigned)grid, tc::THREADS, smem, s>>>(a, map, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_conv_tc_yx(const FwdArgs& a, cudaStream_t s) {
  CUtensorMap map;
  if (!encode_act_map(&map, a.x, tcy::CIN, a.v)) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_conv3_tc_yx, cudaFuncAttributeMaxDynamicSharedMemorySize, tcy::SMEM);
  if (e != cudaSuccess) return e;
  const long long rows = (long long)a.v.batch * a.v.n2 * a.v.n1;
  const long long grid = rows < sm_count() ? rows : sm_count();
  k_conv3_tc_yx<<<(unsigned)grid, tc::THREADS, tcy::SMEM, s>>>(a, map, nullptr);
  return cudaGetLastError();
}

cudaError_t dispatch_conv(int cin, int cout, const FwdArgs& a, cudaStream_t s) {
  if (g_conv_kernel == 0 && a.v.n0 == tc::M) {
    if (cin == 8) return launch_conv_tc<8, 32>(a, s);
    if (cout == 8) return launch_conv_tc_yx(a, s);
    return launch_conv_tc<32, 32>(a, s);
  }
  if (cin == 8) return launch_conv<8, 32>(a, s);
  if (cout == 8) return launch_conv<32, 8>(a, s);
  return launch_conv<32, 32>(a, s);
}

long long wgrad_grid(long long nblocks) { return nblocks < 2LL * sm_count() ? nblocks : 2LL * sm_count(); }

template <int CIN, int COUT>
cudaError_t launch_wgrad(const WgArgs& a, long long grid, cudaStream_t s) {
  const int smem = (HPTS * xstride<CIN>() + BX * BY * (COUT + 8)) * 2;
  cudaError_t e = cudaFuncSetAttribute(k_conv3_wgrad<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k_conv3_wgrad<CIN, COUT><<<(unsigned)grid, WG_THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

mpw_status mpw_conv3_forward(const uint16_t* x, int cin, const uint16_t* w, const float* bias, int cout, int batch,
                             const int n[3], int relu, const uint16_t* mask, uint16_t* y, float* y32, void* stream) {
  if (!supported(cin, cout)) return fail(MPW_ERR_ARG, "conv3: (cin, cout) must be (8, 32), (32, 32) or (32, 8)");
  if (!x || !w || (!y && !y32)) return fail(MPW_ERR_ARG, "conv3: null input, weights or output");
  if (!aligned16(x) || !aligned16(y) || !aligned16(y32) || !aligned16(mask))
    return fail(MPW_ERR_ARG, "conv3: tensors must be 16-byte aligned");
  FwdArgs a{};
  if (mpw_status st = check_volume(batch, n, a.v, a.nblocks)) return st;
  a.x = reinterpret_cast<const __nv_bfloat16*>(x);
  a.w = reinterpret_cast<const __nv_bfloat16*>(w);
  a.bias = bias;
  a.mask = reinterpret_cast<const __nv_bfloat16*>(mask);
  a.y = reinterpret_cast<__nv_bfloat16*>(y);
  a.y32 = y32;
  a.relu = relu ? 1 : 0;
  a.flip = 0;
  if (cudaError_t e = dispatch_conv(cin, cout, a, (cudaStream_t)stream)) return cuda_fail(e);
  return MPW_OK;
}

mpw_status mpw_conv3_backward_data(const uint16_t* gy, int cout, const uint16_t* w, int cin, int batch,
                                   const int n[3], const uint16_t* mask, uint16_t* gx, float* gx32, void* stream) {
  if (!supported(cin, cout)) return fail(MPW_ERR_ARG, "conv3: (cin, cout) must be (8, 32), (32, 32) or (32, 8)");
  if (!gy || !w || (!gx && !gx32)) return fail(MPW_ERR_ARG, "conv3: null gradient, weights or output");
  if (!aligned16(gy) || !aligned16(gx) || !aligned16(gx32) || !aligned16(mask))
    return fail(MPW_ERR_ARG, "conv3: tensors must be 16-byte aligned");
  FwdArgs a{};
  if (mpw_status st = check_volume(batch, n, a.v, a.nblocks)) return st;
  a.x = reinterpret_cast<const __nv_bfloat16*>(gy);
  a.w = reinterpret_cast<const __nv_bfloat16*>(w);
  a.mask = reinterpret_cast<const __nv_bfloat16*>(mask);
  a.y = reinterpret_cast<__nv_bfloat16*>(gx);
  a.y32 = gx32;
  a.flip = 1;
  // the transposed layer: its input channels are the layer's outputs
  if (cudaError_t e = dispatch_conv(cout, cin, a, (cudaStream_t)stream)) return cuda_fail(e);
  return MPW_OK;
}

mpw_status mpw_conv3_select(int kernel) {
  if (kernel != 0 && kernel != 1) return fail(MPW_ERR_ARG, "conv3: kernel must be 0 (tcgen05 where possible) or 1");
  g_conv_kernel = kernel;
  return MPW_OK;
}

size_t mpw_conv3_wgrad_scratch_bytes(int cin, int cout) {
  if (!supported(cin, cout)) return 0;
  return (size_t)2 * sm_count() * (size_t)(cout * 27 * cin + cout) * sizeof(float);
}

mpw_status mpw_conv3_backward_weights(const uint16_t* x, int cin, const uint16_t* gy, int cout, int batch,
                                      const int n[3], float* gw, float* gb, void* scratch, size_t scratch_bytes,
                                      void* stream) {
  if (!supported(cin, cout)) return fail(MPW_ERR_ARG, "conv3: (cin, cout) must be (8, 32), (32, 32) or (32, 8)");
  if (!x || !gy || !gw || !gb || !scratch) return fail(MPW_ERR_ARG, "conv3: null tensor or scratch");
  if (!aligned16(x) || !aligned16(gy)) return fail(MPW_ERR_ARG, "conv3: tensors must be 16-byte aligned");
  WgArgs a{};
  if (mpw_status st = check_volume(batch, n, a.v, a.nblocks)) return st;
  const long long grid = wgrad_grid(a.nblocks);
  const int len = cout * 27 * cin + cout;
  if (scratch_bytes < (size_t)grid * len * sizeof(float)) return fail(MPW_ERR_ARG, "conv3: scratch too small");
  a.x = reinterpret_cast<const __nv_bfloat16*>(x);
  a.g = reinterpret_cast<const __nv_bfloat16*>(gy);
  a.part = static_cast<float*>(scratch);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (cin == 8)
    e = launch_wgrad<8, 32>(a, grid, s);
  else if (cout == 8)
    e = launch_wgrad<32, 8>(a, grid, s);
  else
    e = launch_wgrad<32, 32>(a, grid, s);
  if (e != cudaSuccess) return cuda_fail(e);
  k_sum_parts<<<(len + 255) / 256, 256, 0, s>>>(a.part, (int)grid, len, cout * 27 * cin, gw, gb);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e);
  return MPW_OK;
}

mpw_status mpw_adam_step(float* w, uint16_t* w16, const float* g, float* m, float* v, long long count, float lr,
                         float b1, float b2, float eps, int t, void* stream) {
  if (!w || !g || !m || !v || count < 0 || t < 1) return fail(MPW_ERR_ARG, "adam: null tensor, count < 0 or t < 1");
  if (count == 0) return MPW_OK;
  const double lr_c1 = (double)lr / (1.0 - std::pow((double)b1, t));
  const double c2 = 1.0 / (1.0 - std::pow((double)b2, t));
  long long blocks = (count + 255) / 256;
  if (blocks > 8LL * sm_count()) blocks = 8LL * sm_count();
  k_adam<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(w, reinterpret_cast<__nv_bfloat16*>(w16), g, m, v, count,
                                                             (float)lr_c1, (float)c2, b1, b2, eps);
  if (cudaError_t e = cudaGetLastError()) return cuda_fail(e);
  return MPW_OK;
}

mpw_status mpw_mse_grad(const float* y, int cy, const float* t, int used, long long points, uint16_t* gy,
                        double* loss, void* stream) {
  if (!y || !t || !gy || cy < 1 || used < 1 || used > cy || points < 1)
    return fail(MPW_ERR_ARG, "mse: null tensor or bad channel counts");
  cudaStream_t s = (cudaStream_t)stream;
  if (loss)
    if (cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(double), s)) return cuda_fail(e);
  long long blocks = (points + 255) / 256;
  if (blocks > 8LL * sm_count()) blocks = 8LL * sm_count();
  const double inv = 1.0 / ((double)points * used);
  k_mse<<<(unsigned)blocks, 256, 0, s>>>(y, cy, t, used, points, reinterpret_cast<__nv_bfloat16*>(gy), loss,
                                         (float)(2.0 * inv), inv);
  if (cudaError_t e = cudaGetLastError()) return cuda_fail(e);
  return MPW_OK;
}

}  // extern "C"
