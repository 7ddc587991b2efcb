// mpw_rhs_args.cuh -- the part of libmpw's device interface that the fused
// RHS + stage kernels (k_rhs, k_rhs32) depend on: the padded field layout,
// the covered boxes and the RHS argument tables.
//
// Layout in HBM.  Every patch owns one allocation of 8 field arrays
// (state u, accumulator, two stage buffers; x 2 fields psi, Pi).  A field
// array is a padded box of (n+6) planes x (n+6) rows with a row pitch px that
// is a multiple of 128 B; the interior cell i = 0 sits at column xoff, 32 B
// into the row (xoff = 4 binary64 or 8 binary32 elements), so that the 32
// points of a warp write whole 32-byte sectors; the ghost cells
// i = -3..-1 sit just left of it.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace mpw {

constexpr int NG = 3;
constexpr int XOFF_BYTES = 32;  // byte offset of interior column 0 in a row
constexpr int MAX_PATCHES = 16;
constexpr int MAX_APARAMS = 1024;

enum { BUF_U = 0, BUF_ACC = 1, BUF_YA = 2, BUF_YB = 3 };
enum { FLAG_LIVE = 0, FLAG_GHOST = 1, FLAG_DEAD = 2, FLAG_REVIVED = 3 };
// Bits of the device error word: a ghost point that could not be
// interpolated (Sec. 2.4.1 "skip"), a bounded mbarrier wait that ran out.
enum { ERR_UNFILLED = 1, ERR_TIMEOUT = 8 };

// Try-waits a TMA pipeline wait gets by default (about a second and more on
// GB300); a wait that runs out reports ERR_TIMEOUT instead of hanging.
constexpr unsigned WAIT_LIMIT = 1u << 20;

struct Geom {
  int n[3];
  int px, py;
  int xoff;           // column of interior cell i = 0 (XOFF_BYTES / element size)
  long long plane, vol;
  double lo[3], h[3];
  __host__ __device__ __forceinline__ long long at(int i, int j, int k) const {
    return (long long)(k + NG) * plane + (long long)(j + NG) * px + (i + xoff);
  }
};

// Padded geometry of an n[0] x n[1] x n[2] patch on [lo, lo + n h] with
// elements of esize bytes.
inline Geom padded_geom(const int n[3], const double lo[3], const double h[3], int esize) {
  Geom g{};
  for (int a = 0; a < 3; ++a) {
    g.n[a] = n[a];
    g.lo[a] = lo[a];
    g.h[a] = h[a];
  }
  g.xoff = XOFF_BYTES / esize;
  const int row = 128 / esize;  // elements per 128 B
  g.px = ((n[0] + g.xoff + NG + 1) + row - 1) / row * row;
  g.py = n[1] + 2 * NG;
  g.plane = (long long)g.px * g.py;
  g.vol = g.plane * (n[2] + 2 * NG);
  return g;
}

// Covered box of one local patch in global index space (inclusive bounds);
// empty when lo > hi on any axis.
struct Box {
  int lo[3], hi[3];
};

// ---------------------------------------------------------------- K1
// Tensor maps of one patch buffer for the RHS kernel's TMA loads: `tile`
// covers a (32+8) x (8+6) x 1 x 2-field box (a column tile with its x/y halo,
// x start rounded down to a 16-byte boundary), `point` a 32 x 8 x 1 x 2 box.
struct RhsPatch {
  CUtensorMap ymap;  // tile map of the stencil input buffer
  CUtensorMap umap;  // point map of u
  CUtensorMap amap;  // point map of the accumulator
  const double* Y;   // stencil input (psi; Pi at +vol)
  const double* U;   // u_n
  double* ACC;       // accumulator
  double* OUT;       // next stage state (or u_{n+1} at the last substage)
  Geom g;
  double c1[3];      // w_a / (12 h_a)
  double c2[3];      // 1 / (12 h_a^2)
  double cko[3];     // eps / (64 h_a)
  int tiles_x, tiles_y, zchunks, zc;
  int block0;
  int moving;        // any w_a != 0
  int rot;           // rotating frame: c1 varies with the point,
  double c1g[3][3];  //   c1_a(i, j, k) = c1[a] + c1g[a][0] i + c1g[a][1] j + c1g[a][2] k
  int is_global;
  int iso;           // equal spacing on all axes (D2 and KO sums aggregated)
  int in_buf, out_buf;
};

struct RhsArgs {
  RhsPatch p[MAX_PATCHES];
  int np;
  int stage;            // 0..3
  double alpha, beta;   // OUT = base + alpha K ; ACC = base' + beta K
  const uint8_t* flags; // global cover flags
  int nbox;
  Box box[MAX_PATCHES];
  int* expo;            // tracked maximum biased exponents, [patch][buffer][field]
  int* err;             // device error word
  unsigned wait_limit;  // try-waits allowed to the TMA pipeline's waits (the drain after
                        // an expired wait always gets WAIT_LIMIT)
};

#ifndef MPW_RHS_TY
#define MPW_RHS_TY 8
#endif
#ifndef MPW_RHS_MINB
#define MPW_RHS_MINB 2
#endif
// Default planes per CTA chunk of the RHS kernels for a patch of n2 planes:
// deep chunks cut the z-halo re-reads of large patches (measured on GB300:
// 48 planes for binary64, 64 for binary32, against 32: 1.2 % and 2.6 % faster
// launches); small patches keep short chunks so that they still fill the GPU.
inline int default_rhs_chunk(int n2, bool f32) { return n2 >= 128 ? (f32 ? 64 : 48) : 8; }

constexpr int RHS_TX = 32;
constexpr int RHS_TY = MPW_RHS_TY;      // tile rows (threads per CTA = 32 x RHS_TY)
constexpr int RHS_MIN_BLOCKS = MPW_RHS_MINB;  // CTAs per SM the register budget is sized for

}  // namespace mpw
