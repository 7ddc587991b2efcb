// mpw_kernels.cu -- CUDA kernels of libmpw (sm_103a) besides the RHS and the
// ghost fill: cover flags with buffer (with poisoning and revival), the
// exponent scan, and the closed-form / pack / unpack helpers of the C ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "mpw_device.cuh"
#include "mpw_fixed.cuh"
#include "mpw_internal.cuh"

namespace mpw {

// ---------------------------------------------------------------------------
// Covered mask of the rotating local patches (Sec. 2.4.2, "Find Covered
// Zones"): a global cell is covered when its centre, taken to the patch's
// numeric coordinates, lies in the closed live box.  One thread per cell of
// each patch's bounding box; the mask is box-local, x fastest.
__global__ void __launch_bounds__(256) k_cover(const __grid_constant__ FlagArgs A) {
  long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= A.cov_off[A.nloc]) return;
  int q = 0;
  while (idx >= A.cov_off[q + 1]) ++q;
  const Box& b = A.box[q];
  const long long r = idx - A.cov_off[q];
  const int w0 = b.hi[0] - b.lo[0] + 1, w1 = b.hi[1] - b.lo[1] + 1;
  const int i = b.lo[0] + (int)(r % w0), j = b.lo[1] + (int)((r / w0) % w1), k = b.lo[2] + (int)(r / ((long long)w0 * w1));
  const Geom& gl = A.gl[q];
  if (A.sph[q]) {
    // a shell covers r_lo <= r <= r_hi and r cos(theta_hi) <= z' <= r cos(theta_lo),
    // rounded as written (the oracle's order); covered cells start at the
    // distance cap for the transform that follows
    double xl[3];
    to_local_rn(A.R[q], A.X0[q], node_rn(A.gg.lo[0], i, A.gg.h[0]), node_rn(A.gg.lo[1], j, A.gg.h[1]),
                node_rn(A.gg.lo[2], k, A.gg.h[2]), xl);
    const double rr =
        __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(xl[0], xl[0]), __dmul_rn(xl[1], xl[1])), __dmul_rn(xl[2], xl[2])));
    const bool in = gl.lo[0] <= rr && rr <= A.lhi[q][0] && __dmul_rn(rr, A.cth[q][1]) <= xl[2] &&
                    xl[2] <= __dmul_rn(rr, A.cth[q][0]);
    A.cov[idx] = in ? DIST_CAP : 0;
    return;
  }
  // binary32 screen: a cell whose screened position is at least the margin
  // from every face is decided by it (the margin exceeds 25 times the
  // screen's rounding error); the others take the exact test
  const float MARGIN = A.scrm[q];
  bool sure_in = true, sure_out = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float* c = A.scr[q][a];
    const float v = fmaf(c[0], (float)i, fmaf(c[1], (float)j, fmaf(c[2], (float)k, c[3])));
    const float lo = (float)gl.lo[a], hi = (float)A.lhi[q][a];
    sure_in = sure_in && v > lo + MARGIN && v < hi - MARGIN;
    sure_out = sure_out || v < lo - MARGIN || v > hi + MARGIN;
  }
  bool in = sure_in;
  if (!sure_in && !sure_out) {
    double xl[3];
    to_local_rn(A.R[q], A.X0[q], node_rn(A.gg.lo[0], i, A.gg.h[0]), node_rn(A.gg.lo[1], j, A.gg.h[1]),
                node_rn(A.gg.lo[2], k, A.gg.h[2]), xl);
    in = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) in = in && gl.lo[a] <= xl[a] && xl[a] <= A.lhi[q][a];
  }
  A.cov[idx] = in ? 1 : 0;
}

// One pass of the L-infinity distance transform over the bounding box of every
// spherical shell, along axis ax: out = min over |t| < DIST_CAP of
// max(|t|, in(cell + t e_ax)), cells outside the box reading 0 (uncovered).
// Three passes (x, y, z) from the covered mask (DIST_CAP / 0) give, per cell,
// the distance to the nearest uncovered cell capped at DIST_CAP: max(a,
// min f) = min max(a, f) makes the cube metric separable.
__global__ void __launch_bounds__(256) k_cdt(const __grid_constant__ FlagArgs A, int ax, const uint8_t* __restrict__ in,
                                             uint8_t* __restrict__ out) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= A.cov_off[A.nloc]) return;
  int q = 0;
  while (idx >= A.cov_off[q + 1]) ++q;
  if (!A.sph[q]) return;
  const Box& b = A.box[q];
  const long long r = idx - A.cov_off[q];
  const int w[3] = {b.hi[0] - b.lo[0] + 1, b.hi[1] - b.lo[1] + 1, b.hi[2] - b.lo[2] + 1};
  const int pos[3] = {(int)(r % w[0]), (int)((r / w[0]) % w[1]), (int)(r / ((long long)w[0] * w[1]))};
  const long long stride = ax == 0 ? 1 : (ax == 1 ? (long long)w[0] : (long long)w[0] * w[1]);
  int best = in[idx];
#pragma unroll
  for (int t = 1; t < DIST_CAP; ++t) {
    const int lo = pos[ax] - t, hi = pos[ax] + t;
    const int vl = lo >= 0 ? in[idx - t * stride] : 0;
    const int vh = hi < w[ax] ? in[idx + t * stride] : 0;
    best = min(best, max(t, min(vl, vh)));
  }
  out[idx] = (uint8_t)best;
}

// Covered state of global cell (i, j, k) for rotating patch q (cells outside
// its bounding box are uncovered).
__device__ __forceinline__ bool covered_rot(const FlagArgs& A, int q, int i, int j, int k) {
  const Box& b = A.box[q];
  if (i < b.lo[0] || i > b.hi[0] || j < b.lo[1] || j > b.hi[1] || k < b.lo[2] || k > b.hi[2]) return false;
  const long long w0 = b.hi[0] - b.lo[0] + 1, w1 = b.hi[1] - b.lo[1] + 1;
  return A.cov[A.cov_off[q] + ((long long)(k - b.lo[2]) * w1 + (j - b.lo[1])) * w0 + (i - b.lo[0])] != 0;
}

// Numeric coordinates in local patch q of the centre of global cell (i, j, k).
__device__ __forceinline__ void cell_in_local(const FlagArgs& A, int q, int i, int j, int k, double& x, double& y,
                                              double& z) {
  const double xb = A.gg.lo[0] + (i + 0.5) * A.gg.h[0], yb = A.gg.lo[1] + (j + 0.5) * A.gg.h[1],
               zb = A.gg.lo[2] + (k + 0.5) * A.gg.h[2];
  if (A.sph[q]) {
    double xl[3], qs[3];
    to_local_rn(A.R[q], A.X0[q], xb, yb, zb, xl);
    cart_to_sph(xl, qs);
    x = qs[0], y = qs[1], z = qs[2];
  } else if (A.rot[q]) {
    double xl[3];
    to_local_rn(A.R[q], A.X0[q], xb, yb, zb, xl);
    x = xl[0], y = xl[1], z = xl[2];
  } else {
    x = xb - A.X0[q][0], y = yb - A.X0[q][1], z = zb - A.X0[q][2];
  }
}

// ---------------------------------------------------------------------------
// Cover flags with buffer (Sec. 2.4.2), from the covered set of every local
// patch at t_n; d is a covered cell's L-infinity index distance to the
// nearest uncovered cell: LIVE if d <= buffer, GHOST if d <= buffer + NG,
// DEAD beyond.  Under translation the covered set is a box and d the
// distance to its faces plus one.  A rotating patch covers the cells of a
// rotated box, a convex set: the cube of half-width r around a cell holds
// only covered cells exactly when its eight corners are covered, so d is the
// first r whose corners are not all covered.  DEAD cells of u are poisoned
// with NaN; cells that turn LIVE after having been GHOST or DEAD are
// REVIVED: u_n there is interpolated from the owning local patch at t_n.
template <int P, typename ST>
__device__ __forceinline__ void flags_block(const FlagArgs& A, long long bx) {
  long long idx = bx * (long long)blockDim.x + threadIdx.x;
  int i = 0, j = 0, k = 0;
  bool valid;
  if (A.nreg == 0) {
    const long long N = (long long)A.n[0] * A.n[1] * A.n[2];
    valid = idx < N;
    if (valid) {
      i = (int)(idx % A.n[0]);
      const long long r = idx / A.n[0];
      j = (int)(r % A.n[1]);
      k = (int)(r / A.n[1]);
    }
  } else {
    valid = idx < A.reg_begin[A.nreg];
    if (valid) {
      int g = 0;
      while (idx >= A.reg_begin[g + 1]) ++g;
      idx -= A.reg_begin[g];
      const Box& R = A.reg[g];
      const int w0 = R.hi[0] - R.lo[0] + 1, w1 = R.hi[1] - R.lo[1] + 1;
      i = R.lo[0] + (int)(idx % w0);
      const long long r = idx / w0;
      j = R.lo[1] + (int)(r % w1);
      k = R.lo[2] + (int)(r / w1);
      idx = ((long long)k * A.n[1] + j) * A.n[0] + i;
    }
  }
  int owner = 0, d = 0;
  for (int q = 0; valid && q < A.nloc; ++q) {
    const Box& b = A.box[q];
    if (i >= b.lo[0] && i <= b.hi[0] && j >= b.lo[1] && j <= b.hi[1] && k >= b.lo[2] && k <= b.hi[2]) {
      if (A.sph[q]) {
        // the transform's distance (0: uncovered)
        const long long w0 = b.hi[0] - b.lo[0] + 1, w1 = b.hi[1] - b.lo[1] + 1;
        const int dd = A.cov[A.cov_off[q] + ((long long)(k - b.lo[2]) * w1 + (j - b.lo[1])) * w0 + (i - b.lo[0])];
        if (dd == 0) continue;
        owner = q + 1;
        d = dd;
        break;
      }
      if (A.rot[q]) {
        if (!covered_rot(A, q, i, j, k)) continue;
        owner = q + 1;
        const int rmax = A.buffer + NG;
        d = rmax + 1;
        for (int r = 1; r <= rmax; ++r) {
          bool all = true;
#pragma unroll
          for (int c = 0; c < 8; ++c)
            all = all && covered_rot(A, q, i + ((c & 1) ? r : -r), j + ((c & 2) ? r : -r), k + ((c & 4) ? r : -r));
          if (!all) {
            d = r;
            break;
          }
        }
        break;
      }
      owner = q + 1;
      d = min(min(min(i - b.lo[0], b.hi[0] - i), min(j - b.lo[1], b.hi[1] - j)), min(k - b.lo[2], b.hi[2] - k)) + 1;
      break;
    }
  }
  // effective ghosts of a rotating patch or a shell join that patch's list, one atomic
  // per warp and patch (every lane of the warp takes part)
  const bool ghost_rot = valid && A.glist && owner > 0 && (A.rot[owner - 1] || A.sph[owner - 1]) &&
                         d > A.buffer && d <= A.buffer + NG;
  const int gq = ghost_rot ? owner - 1 : -1;
  const unsigned peers = __match_any_sync(0xffffffffu, gq);
  if (gq >= 0) {
    const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&A.gcount[gq], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    A.glist[A.cov_off[gq] + base + __popc(peers & ((1u << lane) - 1u))] = idx;
  }
  if (!valid) return;
  int st = (owner == 0 || d <= A.buffer) ? FLAG_LIVE : (d <= A.buffer + NG ? FLAG_GHOST : FLAG_DEAD);
  if (A.old_valid && st == FLAG_LIVE) {
    const int os = A.flags[idx] & 3;
    if (os == FLAG_GHOST || os == FLAG_DEAD) st = FLAG_REVIVED;
  }
  A.flags[idx] = (uint8_t)(st | (owner << 2));
  const long long c = A.gg.at(i, j, k);
  ST* Ug = reinterpret_cast<ST*>(A.Ug);
  if (st == FLAG_DEAD) {
    Ug[c] = (ST)__longlong_as_double(0x7ff8000000000000LL);
    Ug[c + A.gg.vol] = (ST)__longlong_as_double(0x7ff8000000000000LL);
  } else if (st == FLAG_REVIVED) {
    const int q = owner - 1;
    // queue the cell: a warp holds about one revived cell, and a warp-wide
    // FP64 instruction costs the same with one active lane as with 32
    const int slot = atomicAdd(A.rev_count, 1);
    if (slot < A.rev_cap) {
      A.rev_list[slot] = idx | ((long long)q << 40);
      return;
    }
    double v0, v1, x, y, z;
    cell_in_local(A, q, i, j, k, x, y, z);
    const bool ok = A.sph[q] ? interp_point_shell<P>(reinterpret_cast<const ST*>(A.Uloc[q]), A.gl[q], x, y, z, v0, v1)
                             : interp_point<P>(reinterpret_cast<const ST*>(A.Uloc[q]), A.gl[q], x, y, z, v0, v1);
    if (!ok) {
      atomicOr(A.err, ERR_UNFILLED);
      return;
    }
    Ug[c] = (ST)v0;
    Ug[c + A.gg.vol] = (ST)v1;
    if (sizeof(ST) == 8) {
      atomicMax(&A.expo[BUF_U * 2], biased_exponent(v0));
      atomicMax(&A.expo[BUF_U * 2 + 1], biased_exponent(v1));
    }
  }
}

template <int P, typename ST>
__global__ void __launch_bounds__(256) k_flags(const __grid_constant__ FlagArgs A) {
  flags_block<P, ST>(A, blockIdx.x);
}

constexpr int REVIVE_BLOCKS = 4 * 152;  // four CTAs per SM of a GB300

// Revival (reading of Sec. 2.4.2): the queued cells take the Lagrange
// interpolant of their local patch at the current time, densely packed.
template <int P, typename ST>
__device__ __forceinline__ void revive_blocks(const FlagArgs& A, int bx, int gx) {
  const int count = min(*A.rev_count, A.rev_cap);
  int e0 = 0, e1 = 0;
  for (int base = bx * blockDim.x; base < count; base += gx * blockDim.x) {
    const int r = base + threadIdx.x;
    if (r < count) {
      const long long ent = A.rev_list[r];
      const long long idx = ent & ((1ll << 40) - 1);
      const int q = (int)(ent >> 40);
      const int i = (int)(idx % A.n[0]);
      const long long rr = idx / A.n[0];
      const int j = (int)(rr % A.n[1]);
      const int k = (int)(rr / A.n[1]);
      double v0, v1, x, y, z;
      cell_in_local(A, q, i, j, k, x, y, z);
      if (A.sph[q] ? interp_point_shell<P>(reinterpret_cast<const ST*>(A.Uloc[q]), A.gl[q], x, y, z, v0, v1)
                   : interp_point<P>(reinterpret_cast<const ST*>(A.Uloc[q]), A.gl[q], x, y, z, v0, v1)) {
        const long long c = A.gg.at(i, j, k);
        ST* Ug = reinterpret_cast<ST*>(A.Ug);
        Ug[c] = (ST)v0;
        Ug[c + A.gg.vol] = (ST)v1;
        e0 = max(e0, biased_exponent(v0));
        e1 = max(e1, biased_exponent(v1));
      } else {
        atomicOr(A.err, ERR_UNFILLED);
      }
    }
  }
  e0 = __reduce_max_sync(0xffffffffu, e0);
  e1 = __reduce_max_sync(0xffffffffu, e1);
  if (sizeof(ST) == 8 && (threadIdx.x & 31) == 0) {
    if (e0) atomicMax(&A.expo[BUF_U * 2], e0);
    if (e1) atomicMax(&A.expo[BUF_U * 2 + 1], e1);
  }
}

template <int P, typename ST>
__global__ void __launch_bounds__(256) k_revive(const __grid_constant__ FlagArgs A) {
  revive_blocks<P, ST>(A, blockIdx.x, gridDim.x);
}

// Batched cover flags of translating instances (argument tables in device
// memory): instance i owns flag blocks [blk0[i], blk0[i + 1]) (blocks from
// blk0[ninst] on pad a captured grid), REVIVE_PER revival blocks each, and
// its queue counter is cleared first by k_flags_reset.
constexpr int REVIVE_PER = 16;

__global__ void k_flags_reset(const FlagArgs* __restrict__ As, int ninst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ninst && As[i].rev_count) *As[i].rev_count = 0;
}

template <int P, typename ST>
__global__ void __launch_bounds__(256) k_flags_batch(const FlagArgs* __restrict__ As, const int* __restrict__ blk0,
                                                     int ninst) {
  if ((int)blockIdx.x >= blk0[ninst]) return;
  int lo = 0, hi = ninst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((int)blockIdx.x >= blk0[mid]) lo = mid; else hi = mid - 1;
  }
  flags_block<P, ST>(As[lo], blockIdx.x - blk0[lo]);
}

template <int P, typename ST>
__global__ void __launch_bounds__(256) k_revive_batch(const FlagArgs* __restrict__ As) {
  const FlagArgs& A = As[blockIdx.x / REVIVE_PER];
  if (!A.rev_count || !A.old_valid || A.skip_revive) return;
  revive_blocks<P, ST>(A, blockIdx.x % REVIVE_PER, REVIVE_PER);
}

template <int P, typename ST>
static void launch_flags_batch_t(const FlagArgs* d_args, const int* d_blk0, int ninst, int blocks, cudaStream_t s) {
  k_flags_reset<<<(ninst + 127) / 128, 128, 0, s>>>(d_args, ninst);
  if (blocks > 0) k_flags_batch<P, ST><<<blocks, 256, 0, s>>>(d_args, d_blk0, ninst);
  k_revive_batch<P, ST><<<ninst * REVIVE_PER, 256, 0, s>>>(d_args);
}

void launch_flags_batch(const FlagArgs* d_args, const int* d_blk0, int ninst, int blocks, int P, bool f32,
                        void* stream) {
  const cudaStream_t s = (cudaStream_t)stream;
  if (f32)
    P == 6 ? launch_flags_batch_t<6, float>(d_args, d_blk0, ninst, blocks, s)
           : launch_flags_batch_t<5, float>(d_args, d_blk0, ninst, blocks, s);
  else
    P == 6 ? launch_flags_batch_t<6, double>(d_args, d_blk0, ninst, blocks, s)
           : launch_flags_batch_t<5, double>(d_args, d_blk0, ninst, blocks, s);
}

long long flags_blocks(const FlagArgs& a) {
  const long long N = a.nreg ? a.reg_begin[a.nreg] : (long long)a.n[0] * a.n[1] * a.n[2];
  return (N + 255) / 256;
}

// Every DEAD global cell of buffer A.Ug takes the Lagrange interpolant of the
// local patch that covers it (A.Uloc: that patch's buffer).  Dead cells take
// no part in the method; the learned surrogate reads a complete field.
// Block row q of the grid walks the covered box of local patch q.
template <int P>
__global__ void __launch_bounds__(256) k_fill_dead(const __grid_constant__ FlagArgs A) {
  const int q = blockIdx.y;
  const Box& b = A.box[q];
  const int w0 = b.hi[0] - b.lo[0] + 1, w1 = b.hi[1] - b.lo[1] + 1, w2 = b.hi[2] - b.lo[2] + 1;
  if (w0 <= 0 || w1 <= 0 || w2 <= 0) return;
  const long long V = (long long)w0 * w1 * w2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < V; e += (long long)gridDim.x * blockDim.x) {
    const int i = b.lo[0] + (int)(e % w0), j = b.lo[1] + (int)((e / w0) % w1), k = b.lo[2] + (int)(e / ((long long)w0 * w1));
    const uint8_t f = A.flags[((long long)k * A.n[1] + j) * A.n[0] + i];
    if ((f & 3) != FLAG_DEAD || (f >> 2) != q + 1) continue;
    double v0, v1, x, y, z;
    cell_in_local(A, q, i, j, k, x, y, z);
    if (interp_point<P>(A.Uloc[q], A.gl[q], x, y, z, v0, v1)) {
      const long long c = A.gg.at(i, j, k);
      A.Ug[c] = v0;
      A.Ug[c + A.gg.vol] = v1;
    } else {
      atomicOr(A.err, ERR_UNFILLED);
    }
  }
}

void launch_fill_dead(const FlagArgs& a, void* stream) {
  long long vmax = 0;
  for (int q = 0; q < a.nloc; ++q) {
    const Box& b = a.box[q];
    vmax = std::max(vmax, (long long)std::max(b.hi[0] - b.lo[0] + 1, 0) * std::max(b.hi[1] - b.lo[1] + 1, 0) *
                              std::max(b.hi[2] - b.lo[2] + 1, 0));
  }
  if (vmax == 0 || a.nloc == 0) return;
  const dim3 grid((unsigned)std::min<long long>((vmax + 255) / 256, 1024), (unsigned)a.nloc);
  if (a.P == 6)
    k_fill_dead<6><<<grid, 256, 0, (cudaStream_t)stream>>>(a);
  else
    k_fill_dead<5><<<grid, 256, 0, (cudaStream_t)stream>>>(a);
}

template <int P, typename ST>
static void launch_flags_t(const FlagArgs& a, unsigned blocks, unsigned rblocks, cudaStream_t s) {
  const long long ncov = a.cov_off[a.nloc];
  if (ncov > 0) k_cover<<<(unsigned)((ncov + 255) / 256), 256, 0, s>>>(a);
  bool any_sph = false;
  for (int q = 0; q < a.nloc; ++q) any_sph = any_sph || a.sph[q];
  if (any_sph) {
    // distance transform: mask -> region 1 (x) -> region 2 (y) -> region 0 (z)
    const unsigned cb = (unsigned)((ncov + 255) / 256);
    k_cdt<<<cb, 256, 0, s>>>(a, 0, a.cov, a.cov + ncov);
    k_cdt<<<cb, 256, 0, s>>>(a, 1, a.cov + ncov, a.cov + 2 * ncov);
    k_cdt<<<cb, 256, 0, s>>>(a, 2, a.cov + 2 * ncov, a.cov);
  }
  k_flags<P, ST><<<blocks, 256, 0, s>>>(a);
  if (a.old_valid && !a.skip_revive) k_revive<P, ST><<<rblocks, 256, 0, s>>>(a);
}

int launch_flags(const FlagArgs& a, void* stream) {
  const long long N = a.nreg ? a.reg_begin[a.nreg] : (long long)a.n[0] * a.n[1] * a.n[2];
  if (N <= 0) return 0;
  const cudaStream_t s = (cudaStream_t)stream;
  cudaMemsetAsync(a.rev_count, 0, sizeof(int), s);
  if (a.gcount) cudaMemsetAsync(a.gcount, 0, sizeof(int) * MAX_PATCHES, s);
  const unsigned blocks = (unsigned)((N + 255) / 256);
  // the revival kernel walks the queue with a fixed grid (its length is
  // known on the device only); empty queues cost one short launch
  const unsigned rblocks = (unsigned)std::min<long long>((N + 255) / 256, REVIVE_BLOCKS);
  if (a.f32)
    a.P == 6 ? launch_flags_t<6, float>(a, blocks, rblocks, s) : launch_flags_t<5, float>(a, blocks, rblocks, s);
  else
    a.P == 6 ? launch_flags_t<6, double>(a, blocks, rblocks, s) : launch_flags_t<5, double>(a, blocks, rblocks, s);
  bool any_sph = false;
  for (int q = 0; q < a.nloc; ++q) any_sph = any_sph || a.sph[q];
  return (a.old_valid && !a.skip_revive ? 2 : 1) + (a.cov_off[a.nloc] > 0 ? 1 : 0) + (any_sph ? 3 : 0);
}

// ---------------------------------------------------------------------------
// Interior <- closed form at time t (positions X_B = numeric + X0).
template <typename ST>
__global__ void k_analytic(ST* buf, const Geom g, const Affine map, int rot, int sph, int akind, int acount,
                           const double* __restrict__ P, const float4* __restrict__ screen,
                           const double* __restrict__ apre, double t) {
  const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= N) return;
  const int i = (int)(idx % g.n[0]);
  const long long r = idx / g.n[0];
  const int j = (int)(r % g.n[1]);
  const int k = (int)(r / g.n[1]);
  const double x = g.lo[0] + (i + 0.5) * g.h[0], y = g.lo[1] + (j + 0.5) * g.h[1], z = g.lo[2] + (k + 0.5) * g.h[2];
  double xb, yb, zb;
  if (sph) {
    double xl[3];
    sph_to_cart(x, y, z, xl);
    affine(map.R, map.X0, xl[0], xl[1], xl[2], xb, yb, zb);
  } else if (rot) {
    double b[3];
    to_background_rn(map.R, map.X0, node_rn(g.lo[0], i, g.h[0]), node_rn(g.lo[1], j, g.h[1]),
                     node_rn(g.lo[2], k, g.h[2]), b);
    xb = b[0], yb = b[1], zb = b[2];
  } else {
    xb = x + map.X0[0], yb = y + map.X0[1], zb = z + map.X0[2];
  }
  double ps, pv;
  closed_form(akind, P, screen, apre, acount, t, xb, yb, zb, ps, pv);
  const long long c = g.at(i, j, k);
  buf[c] = (ST)ps;
  buf[c + g.vol] = (ST)pv;
}

void launch_analytic(void* buf, const Geom& g, const Affine& map, int akind, int acount, const double* aparams,
                     const float4* screen, const double* apre, double t, bool f32, void* stream, bool sph) {
  const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
  const unsigned blocks = (unsigned)((N + 255) / 256);
  int rot = 0;
  for (int e = 0; e < 9; ++e) rot |= map.R[e] != ((e % 4 == 0) ? 1.0 : 0.0);
  if (f32)
    k_analytic<float><<<blocks, 256, 0, (cudaStream_t)stream>>>(static_cast<float*>(buf), g, map, rot, sph, akind,
                                                                acount, aparams, screen, apre, t);
  else
    k_analytic<double><<<blocks, 256, 0, (cudaStream_t)stream>>>(static_cast<double*>(buf), g, map, rot, sph, akind,
                                                                 acount, aparams, screen, apre, t);
}

// Padded buffer -> dense array (interior, or the whole padded box).  With
// flags, global cells that are not live read as NaN.
template <typename ST>
__global__ void k_pack(const ST* __restrict__ buf, const Geom g, double* __restrict__ d0,
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
  double v0 = (double)buf[c], v1 = (double)buf[c + g.vol];
  if (flags) {
    const int f = flags[((long long)k * g.n[1] + j) * g.n[0] + i] & 3;
    if (f == FLAG_GHOST || f == FLAG_DEAD) v0 = v1 = __longlong_as_double(0x7ff8000000000000LL);
  }
  d0[idx] = v0;
  d1[idx] = v1;
}

void launch_pack(const void* buf, const Geom& g, double* d0, double* d1, int padded, const uint8_t* flags, bool f32,
                 void* stream) {
  const int e = padded ? 2 * NG : 0;
  const long long N = (long long)(g.n[0] + e) * (g.n[1] + e) * (g.n[2] + e);
  const unsigned blocks = (unsigned)((N + 255) / 256);
  if (f32)
    k_pack<float><<<blocks, 256, 0, (cudaStream_t)stream>>>(static_cast<const float*>(buf), g, d0, d1, padded,
                                                            padded ? nullptr : flags);
  else
    k_pack<double><<<blocks, 256, 0, (cudaStream_t)stream>>>(static_cast<const double*>(buf), g, d0, d1, padded,
                                                             padded ? nullptr : flags);
}

template <typename ST>
__global__ void k_unpack(ST* buf, const Geom g, const double* __restrict__ d0, const double* __restrict__ d1) {
  const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= N) return;
  const int i = (int)(idx % g.n[0]);
  const long long r = idx / g.n[0];
  const int j = (int)(r % g.n[1]);
  const int k = (int)(r / g.n[1]);
  const long long c = g.at(i, j, k);
  buf[c] = (ST)d0[idx];
  buf[c + g.vol] = (ST)d1[idx];
}

// k_unpack for binary64 buffers that also raises the buffer's exponent slots
// (slot2, cleared before the launch) with the largest biased exponent of the
// live values it writes, as k_expo_scan would, so that u needs no second
// pass.  flags (global patch, or null): cells flagged GHOST or DEAD are
// written but not counted.  Rows of the interior are spread over the blocks,
// the threads of a block along x; one atomic per field and block.
__global__ void __launch_bounds__(128) k_unpack_scan(double* buf, const Geom g, const double* __restrict__ d0,
                                                     const double* __restrict__ d1,
                                                     const uint8_t* __restrict__ flags, int* slot2) {
  const int n0 = g.n[0], n1 = g.n[1];
  const int rows = n1 * g.n[2];
  int e0 = 0, e1 = 0;
  for (int r = blockIdx.x; r < rows; r += gridDim.x) {
    const int j = r % n1, k = r / n1;
    const long long base = (long long)r * n0;
    const long long c0 = g.at(0, j, k);
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
      const double a = d0[base + i], b = d1[base + i];
      buf[c0 + i] = a;
      buf[c0 + i + g.vol] = b;
      if (flags) {
        const int f = flags[base + i] & 3;
        if (f == FLAG_GHOST || f == FLAG_DEAD) continue;
      }
      e0 = max(e0, biased_exponent(a));
      e1 = max(e1, biased_exponent(b));
    }
  }
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

void launch_unpack_scan(double* buf, const Geom& g, const double* d0, const double* d1, const uint8_t* flags,
                        int* slot2, void* stream) {
  const int rows = g.n[1] * g.n[2];
  const int blocks = rows < 152 * 16 ? rows : 152 * 16;
  if (blocks > 0) k_unpack_scan<<<blocks, 128, 0, (cudaStream_t)stream>>>(buf, g, d0, d1, flags, slot2);
}

void launch_unpack(void* buf, const Geom& g, const double* d0, const double* d1, bool f32, void* stream) {
  const long long N = (long long)g.n[0] * g.n[1] * g.n[2];
  const unsigned blocks = (unsigned)((N + 255) / 256);
  if (f32)
    k_unpack<float><<<blocks, 256, 0, (cudaStream_t)stream>>>(static_cast<float*>(buf), g, d0, d1);
  else
    k_unpack<double><<<blocks, 256, 0, (cudaStream_t)stream>>>(static_cast<double*>(buf), g, d0, d1);
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
