// mpw_noalloc.cu -- an entry point that allocates no memory at all.
//
// Some callers cannot call cudaMalloc (or any allocating routine) when they
// want to advance a field: plugins that live inside a host application whose
// allocator owns all device memory, and timing-critical loops that must not
// enter the driver's allocator.  mpw_step_periodic_noalloc serves them for the simplest
// layout the library supports, one periodic Cartesian patch.  It runs the same
// ghost-fill and fused RHS + RK4 stage kernels as mpw_step, but every work
// buffer (the padded state, accumulator and stage buffers, the exponent slots
// and the error word) lives in one file-scope __device__ array of fixed size
// that every GPU loading the library holds until the process exits.  The
// caller still owns and passes the field arrays it reads and writes.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/mpw.h"
#include "mpw_fixed.cuh"
#include "mpw_internal.cuh"

using namespace mpw;

namespace {

// Largest padded field array: (48 + 6) planes x (48 + 6) rows x 64 doubles.
constexpr int NOALLOC_MAX_N = MPW_NOALLOC_MAX_N;
constexpr long long NOALLOC_MAX_VOL = 64LL * (NOALLOC_MAX_N + 2 * NG) * (NOALLOC_MAX_N + 2 * NG);
// 4 buffers x 2 fields, then exponent slots and the error word (in doubles)
constexpr long long NOALLOC_WORDS = 8 * NOALLOC_MAX_VOL + 64;

// The scratch array (about 12 MB, held by every GPU that loads the library
// until the process exits).  Host code must not pass its name to a kernel: on
// the host it is only a stand-in, and a kernel given it would fault or read
// the wrong memory.  The device address comes from cudaGetSymbolAddress,
// looked up once per device on that device's first call (so that first call
// belongs before any stream capture).  Every call reuses the array and keeps
// the previous call's contents; the exponent slots and the error word are
// cleared at the start of each call.  Calls that overlap on the GPU race.
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_WORDS];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[MAX_DEVICES] = {nullptr};

mpw_status fail(mpw_status st, const char* msg) {
  set_last_error(msg);
  return st;
}

}  // namespace

extern "C" mpw_status mpw_step_periodic_noalloc(const int n[3], const double lo[3], const double hi[3],
                                                double ko_eps, double dt, int nsteps, double* psi, double* pi,
                                                void* stream) {
  if (!n || !lo || !hi || !psi || !pi) return fail(MPW_ERR_ARG, "null argument");
  for (int a = 0; a < 3; ++a) {
    if (n[a] < 2 * NG || n[a] > NOALLOC_MAX_N)
      return fail(MPW_ERR_ARG, "mpw_step_periodic_noalloc: each n must be in [6, MPW_NOALLOC_MAX_N = 48]");
    if (!(hi[a] > lo[a])) return fail(MPW_ERR_ARG, "mpw_step_periodic_noalloc: hi must exceed lo");
  }
  if (!(dt > 0.0) || nsteps < 0 || !(ko_eps >= 0.0)) return fail(MPW_ERR_ARG, "bad dt, nsteps or ko_eps");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return fail(MPW_ERR_CUDA, "cudaGetDevice");
  // one-time set-up per device: the device address of the scratch array
  double* base;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) return fail(MPW_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
      g_scratch_ptr[dev] = static_cast<double*>(ptr);
    }
    base = g_scratch_ptr[dev];
  }
  // padded geometry (same layout as the context path)
  double h[3];
  for (int a = 0; a < 3; ++a) h[a] = (hi[a] - lo[a]) / n[a];
  const Geom g = padded_geom(n, lo, h, 8);
  double lap = 0.0;
  for (int a = 0; a < 3; ++a) lap += 16.0 / (3.0 * g.h[a] * g.h[a]);
  if (dt * std::sqrt(lap) > 2.8) return fail(MPW_ERR_CFL, "dt exceeds the RK4 stability estimate");
  double* buf[4];
  for (int b = 0; b < 4; ++b) buf[b] = base + (long long)b * 2 * g.vol;
  // TMA maps of the scratch buffers (host-side encoding, no allocation)
  CUtensorMap tile_map[4], point_map[2];
  for (int b = 0; b < 4; ++b)
    if (!encode_rhs_map(&tile_map[b], buf[b], g, true)) return fail(MPW_ERR_CUDA, "tensor map encoding failed");
  if (!encode_rhs_map(&point_map[0], buf[BUF_U], g, false) || !encode_rhs_map(&point_map[1], buf[BUF_ACC], g, false))
    return fail(MPW_ERR_CUDA, "tensor map encoding failed");
  int* expo = reinterpret_cast<int*>(base + 8 * NOALLOC_MAX_VOL);
  int* err = expo + 32;
  cudaStream_t s = (cudaStream_t)stream;
  // state in; exponent slots and error word start at zero on every call
  launch_unpack(buf[BUF_U], g, psi, pi, false, s);
  if (cudaMemsetAsync(expo, 0, 64 * sizeof(int), s) != cudaSuccess) return fail(MPW_ERR_CUDA, "memset");
  launch_expo_scan(buf[BUF_U], g, nullptr, expo + BUF_U * 2, s);
  static const double RK_C[4] = {0.0, 0.5, 0.5, 1.0};
  static const int in_buf[4] = {BUF_U, BUF_YA, BUF_YB, BUF_YA};
  static const int out_buf[4] = {BUF_YA, BUF_YB, BUF_YA, BUF_U};
  double t = 0.0;
  for (int step = 0; step < nsteps; ++step) {
    for (int l = 0; l < 4; ++l) {
      FillArgs f{};
      f.Yg = buf[in_buf[l]];
      f.gg = g;
      f.outer_bc = 1;
      f.t = t + RK_C[l] * dt;
      f.outer_count = (long long)(n[0] + 2 * NG) * (n[1] + 2 * NG) * (n[2] + 2 * NG) - (long long)n[0] * n[1] * n[2];
      f.outer_blocks = (int)((f.outer_count + fill_threads() - 1) / fill_threads());
      f.nseg = 0;
      f.P = 6;
      f.err = err;
      f.expo = expo;
      f.y_buf = in_buf[l];
      f.reset_buf = out_buf[l];
      f.np = 1;
      f.total_blocks = f.outer_blocks;
      f.fixed = 1;
      f.f32 = 0;
      launch_fill(f, s);
      RhsArgs r{};
      r.np = 1;
      r.stage = l;
      const double alpha[4] = {0.5 * dt, 0.5 * dt, dt, dt / 6.0};
      const double beta[4] = {dt / 6.0, dt / 3.0, dt / 3.0, 0.0};
      r.alpha = alpha[l];
      r.beta = beta[l];
      r.expo = expo;
      r.err = err;
      r.wait_limit = WAIT_LIMIT;
      RhsPatch& R = r.p[0];
      R.ymap = tile_map[in_buf[l]];
      R.umap = point_map[0];
      R.amap = point_map[1];
      R.Y = buf[in_buf[l]];
      R.U = buf[BUF_U];
      R.ACC = buf[BUF_ACC];
      R.OUT = buf[out_buf[l]];
      R.g = g;
      for (int k = 0; k < 3; ++k) {
        R.c1[k] = 0.0;
        R.c2[k] = 1.0 / (12.0 * g.h[k] * g.h[k]);
        R.cko[k] = ko_eps / (64.0 * g.h[k]);
      }
      R.moving = 0;
      R.is_global = 0;
      R.iso = g.h[0] == g.h[1] && g.h[1] == g.h[2];
      R.in_buf = in_buf[l];
      R.out_buf = out_buf[l];
      R.tiles_x = (n[0] + RHS_TX - 1) / RHS_TX;
      R.tiles_y = (n[1] + RHS_TY - 1) / RHS_TY;
      R.zc = 8;
      R.zchunks = (n[2] + R.zc - 1) / R.zc;
      R.block0 = 0;
      launch_rhs(r, R.tiles_x * R.tiles_y * R.zchunks, true, false, s);
    }
    t += dt;
  }
  launch_pack(buf[BUF_U], g, psi, pi, 0, nullptr, false, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(MPW_ERR_CUDA, cudaGetErrorString(e));
  // The device error word, read into a host stack variable once the work has
  // run: a copy into pageable host memory stages through the driver's own
  // buffers, so nothing is allocated here either.
  int word = 0;
  e = cudaMemcpyAsync(&word, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(MPW_ERR_CUDA, cudaGetErrorString(e));
  if (word & ERR_TIMEOUT) return fail(MPW_ERR_TIMEOUT, "a bounded device wait ran out; psi and pi are incomplete");
  if (word & ERR_UNFILLED) return fail(MPW_ERR_GHOST_UNFILLED, "a ghost point could not be filled");
  if (word) return fail(MPW_ERR_CUDA, "unexpected device error word");
  return MPW_OK;
}
