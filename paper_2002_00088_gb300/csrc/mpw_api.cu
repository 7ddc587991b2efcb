// mpw_api.cu -- host side of libmpw: the C ABI of include/mpw.h, patch
// storage, motion laws, validation and the per-step launch schedule.
//
// Per step (Sec. 2.3-2.4): cover flags from the maps at t_n (recomputed every
// step while any local patch moves, once for static layouts), then for each
// RK4 substage l = 1..4 at t_l = t_n + c_l dt one ghost-fill launch (outer
// BC, Local-to-Global, Global-to-Local with the maps at t_l) and one fused
// RHS + stage launch covering every patch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mpw.h"
#include "../../include/mpw_surrogate.h"
#include "mpw_fixed.cuh"
#include "mpw_internal.cuh"

using namespace mpw;

namespace {

thread_local std::string g_last_error;

mpw_status set_err(mpw_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

#define CUDA_TRY(call)                                                                              \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) return set_err(MPW_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Classic RK4 (Table 1): c_l.
const double RK_C[4] = {0.0, 0.5, 0.5, 1.0};

struct PatchState {
  mpw_patch_desc d;
  Geom g;
  bool u_expo_valid = false;  // exponent slots of u track its live values
  double* base = nullptr;     // 4 buffers x 2 fields x vol elements (binary64, or binary32 when esize = 4)
  double* tab = nullptr;      // spherical shell: node tables of the RHS (see ShellPatch)
  size_t esize = 8;           // bytes per element
  CUtensorMap tile_map[4];    // RHS input tiles of each buffer (TMA)
  CUtensorMap point_map[2];   // RHS stage operands: u, ACC (TMA)
  // asynchronous host IO (mpw_set_fields_async / mpw_get_fields_async):
  // device staging of the next input and of the last result (2 n doubles
  // each), and the events that order them with the copy streams
  double* io_in = nullptr;
  double* io_out = nullptr;
  cudaEvent_t in_copied = nullptr, in_free = nullptr, out_packed = nullptr, out_free = nullptr;
  bool in_pending = false;
  bool sph() const { return d.topology == MPW_TOPOLOGY_SPHERICAL; }
  // device address of buffer b (its element type follows esize)
  double* buf(int b) const {
    return reinterpret_cast<double*>(reinterpret_cast<char*>(base) + (size_t)b * 2 * (size_t)g.vol * esize);
  }
};

}  // namespace

struct mpw_ctx {
  mpw_config cfg{};
  cudaStream_t stream = nullptr;
  int P = 6, buffer = NG + 1;
  std::vector<PatchState> p;
  int akind = -1, acount = 0;
  std::vector<double> aparams;
  std::vector<float4> screen;
  std::vector<double> apre;
  double* d_aparams = nullptr;
  float4* d_ascreen = nullptr;  // FP32 screening data of Gaussian pulses
  double* d_apre = nullptr;     // 1/width^2 of every Gaussian pulse
  bool screen_ok = false;
  uint8_t* d_flags = nullptr;
  bool flags_valid = false;
  std::vector<Box> boxes;  // covered boxes at the last flag computation
  int* d_err = nullptr;
  int* h_err = nullptr;
  unsigned wait_limit = WAIT_LIMIT;  // try-waits of the RHS kernels' TMA pipeline waits
  int* d_expo = nullptr;  // [patch][buffer][field] maximum biased exponent
  long long* d_rev = nullptr;  // queue of revived cells (REVIVE_CAP entries); its length lives in d_err[32]
  uint8_t* d_cov = nullptr;    // covered masks of the rotating patches' bounding boxes
  size_t cov_bytes = 0;
  long long* d_glist = nullptr;  // effective ghosts of the rotating patches (same offsets as d_cov)
  int* d_gcount = nullptr;       // their counts, MAX_PATCHES entries
  std::vector<long long> glist_off;  // per local patch, from the last flag computation
  bool glist_valid = false;          // lists match the current flags
  int2* d_mirror = nullptr;          // fixed-point mirrors of the shells' donor regions
  size_t mirror_cap = 0;             // entries
  // Time whose closed form each global buffer's outer shell holds (NaN: none).
  // The RK4 substage times repeat (c = 0, 1/2, 1/2, 1, and t_n + dt starts the
  // next step), so half of the analytic shell evaluations become copies.
  double shell_time[4] = {NAN, NAN, NAN, NAN};
  double* d_stage = nullptr;
  size_t stage_bytes = 0;
  double* d_sur = nullptr;  // hybrid stepping: dense global states, Laplacians, Hermite coefficients
  size_t sur_bytes = 0;
  // copy streams of the asynchronous host IO: inputs in, results out
  cudaStream_t io_in = nullptr, io_out = nullptr;
  double t = 0.0;
  bool stepped = false;
  // measurement: per kernel family, a pool of event pairs and a launch count
  bool prof = false;
  std::vector<cudaEvent_t> ev[MPW_KERNEL_FAMILIES];
  size_t ev_used[MPW_KERNEL_FAMILIES] = {0, 0, 0};
  long long launches[MPW_KERNEL_FAMILIES] = {0, 0, 0};

  // Record the start event of a launch of family f (when timing is on).
  void launch_begin(int f) {
    ++launches[f];
    if (!prof) return;
    if (ev[f].size() < 2 * (ev_used[f] + 1)) {
      cudaEvent_t a, b;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      ev[f].push_back(a);
      ev[f].push_back(b);
    }
    cudaEventRecord(ev[f][2 * ev_used[f]], stream);
  }
  void launch_end(int f) {
    if (!prof) return;
    cudaEventRecord(ev[f][2 * ev_used[f] + 1], stream);
    ++ev_used[f];
  }

  void* dalloc(size_t bytes) {
    if (cfg.alloc) return cfg.alloc(bytes, cfg.alloc_user);
    void* ptr = nullptr;
    return cudaMalloc(&ptr, bytes) == cudaSuccess ? ptr : nullptr;
  }
  void dfree(void* ptr) {
    if (!ptr) return;
    if (cfg.free)
      cfg.free(ptr, cfg.alloc_user);
    else
      cudaFree(ptr);
  }
};

namespace {

void rotation(const mpw_patch_desc& d, double t, double R[9]);

// Rigid motion of a patch: X_B = R(t) X' + X0(t), R = I except for ROTATING;
// w = R^T dX0/dt is the frame velocity at X' = 0.  The rounding order is
// fixed (no contraction) because the cover flags depend on it.
void motion(const mpw_patch_desc& d, double t, double X0[3], double w[3]) {
  const double* mp = d.motion_params;
  if (d.motion == MPW_MOTION_ROTATING) {
    double R[9];
    rotation(d, t, R);
    for (int a = 0; a < 3; ++a) X0[a] = mp[a] + t * mp[3 + a];
    for (int a = 0; a < 3; ++a) w[a] = R[a] * mp[3] + R[3 + a] * mp[4] + R[6 + a] * mp[5];
  } else if (d.motion == MPW_MOTION_LINEAR) {
    for (int a = 0; a < 3; ++a) {
      X0[a] = mp[a] + t * mp[3 + a];
      w[a] = mp[3 + a];
    }
  } else if (d.motion == MPW_MOTION_CIRCULAR) {
    const double ph = mp[4] * t + mp[5];
    const double c = std::cos(ph), s = std::sin(ph);
    X0[0] = mp[0] + mp[3] * c;
    X0[1] = mp[1] + mp[3] * s;
    X0[2] = mp[2];
    w[0] = -(mp[3] * mp[4]) * s;
    w[1] = (mp[3] * mp[4]) * c;
    w[2] = 0.0;
  } else {
    for (int a = 0; a < 3; ++a) {
      X0[a] = mp[a];
      w[a] = 0.0;
    }
  }
}

// Rotation by theta = p9 t + p10 about the unit axis n = (p6, p7, p8)
// (Rodrigues: R = cos I + sin [n]_x + (1 - cos) n n^T, row-major), the
// entries formed in a fixed order: the cover flags depend on their last bit.
void rotation(const mpw_patch_desc& d, double t, double R[9]) {
  const double* mp = d.motion_params;
  const double* n = mp + 6;
  const double th = mp[9] * t + mp[10];
  const double c = std::cos(th), sn = std::sin(th), omc = 1.0 - c;
  const double K[9] = {0.0, -n[2], n[1], n[2], 0.0, -n[0], -n[1], n[0], 0.0};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) R[3 * a + b] = ((a == b ? c : 0.0) + sn * K[3 * a + b]) + (omc * n[a]) * n[b];
}

// Map of a patch at time t and its frame velocity as an affine function of
// the patch point: X_B = R X' + X0, w(X') = w0 + W X' (patch components;
// W = Omega [n]_x for a rotating patch, 0 otherwise).
struct Frame {
  bool rot = false;
  double R[9], X0[3], w0[3], W[9];
};

Frame frame(const mpw_patch_desc& d, double t) {
  Frame f;
  f.rot = d.motion == MPW_MOTION_ROTATING;
  motion(d, t, f.X0, f.w0);
  for (int e = 0; e < 9; ++e) {
    f.R[e] = (e % 4 == 0) ? 1.0 : 0.0;
    f.W[e] = 0.0;
  }
  if (f.rot) {
    rotation(d, t, f.R);
    const double* n = d.motion_params + 6;
    const double om = d.motion_params[9];
    const double K[9] = {0.0, -n[2], n[1], n[2], 0.0, -n[0], -n[1], n[0], 0.0};
    for (int e = 0; e < 9; ++e) f.W[e] = om * K[e];
  }
  return f;
}

// X_B of the patch point xl (interpolation positions; host side).
void to_background(const Frame& f, const double xl[3], double xb[3]) {
  for (int a = 0; a < 3; ++a)
    xb[a] = f.rot ? ((f.R[3 * a] * xl[0] + f.R[3 * a + 1] * xl[1]) + f.R[3 * a + 2] * xl[2]) + f.X0[a] : xl[a] + f.X0[a];
}

// Background bounding box of the patch box [lo - e h, hi + e h] at time t
// (exact for translation).
void background_extent(const mpw_patch_desc& d, double t, double e, double lo[3], double hi[3]) {
  const Frame f = frame(d, t);
  if (d.topology == MPW_TOPOLOGY_SPHERICAL) {
    // a shell lies in the ball of radius r_hi (+ e radial cells) about X0
    const double R = d.hi[0] + e * (d.hi[0] - d.lo[0]) / d.n[0];
    for (int a = 0; a < 3; ++a) {
      lo[a] = f.X0[a] - R;
      hi[a] = f.X0[a] + R;
    }
    return;
  }
  double h[3];
  for (int a = 0; a < 3; ++a) {
    h[a] = (d.hi[a] - d.lo[a]) / d.n[a];
    lo[a] = 1e300;
    hi[a] = -1e300;
  }
  for (int c = 0; c < 8; ++c) {
    double xl[3], xb[3];
    for (int a = 0; a < 3; ++a) xl[a] = ((c >> a) & 1) ? d.hi[a] + e * h[a] : d.lo[a] - e * h[a];
    to_background(f, xl, xb);
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], xb[a]);
      hi[a] = std::max(hi[a], xb[a]);
    }
  }
}

// Largest speed of a point of the live box in the background frame (the
// Euclidean bound |Omega| r_max + |V| for a rotating patch).
double max_point_speed(const mpw_patch_desc& d) {
  const double* mp = d.motion_params;
  if (d.topology == MPW_TOPOLOGY_SPHERICAL) {
    // points of the shell lie within r_hi of the patch origin
    double v = 0.0;
    if (d.motion == MPW_MOTION_LINEAR) v = std::sqrt(mp[3] * mp[3] + mp[4] * mp[4] + mp[5] * mp[5]);
    if (d.motion == MPW_MOTION_CIRCULAR) v = std::fabs(mp[3] * mp[4]);
    if (d.motion == MPW_MOTION_ROTATING)
      v = std::fabs(mp[9]) * d.hi[0] + std::sqrt(mp[3] * mp[3] + mp[4] * mp[4] + mp[5] * mp[5]);
    return v;
  }
  if (d.motion == MPW_MOTION_LINEAR) return std::sqrt(mp[3] * mp[3] + mp[4] * mp[4] + mp[5] * mp[5]);
  if (d.motion == MPW_MOTION_CIRCULAR) return std::fabs(mp[3] * mp[4]);
  if (d.motion != MPW_MOTION_ROTATING) return 0.0;
  double r2 = 0.0;
  for (int c = 0; c < 8; ++c) {
    double q = 0.0;
    for (int a = 0; a < 3; ++a) {
      const double x = ((c >> a) & 1) ? d.hi[a] : d.lo[a];
      q += x * x;
    }
    r2 = std::max(r2, q);
  }
  return std::fabs(mp[9]) * std::sqrt(r2) + std::sqrt(mp[3] * mp[3] + mp[4] * mp[4] + mp[5] * mp[5]);
}

// Largest |w_a| per axis the motion law can reach (a rotating patch: the
// bound over the live box, |Omega| |(n x X')_a| + |V| at the corners).
void max_speed(const mpw_patch_desc& d, double v[3]) {
  const double* mp = d.motion_params;
  for (int a = 0; a < 3; ++a) v[a] = 0.0;
  if (d.motion == MPW_MOTION_LINEAR)
    for (int a = 0; a < 3; ++a) v[a] = std::fabs(mp[3 + a]);
  if (d.motion == MPW_MOTION_CIRCULAR) v[0] = v[1] = std::fabs(mp[3] * mp[4]);
  if (d.motion == MPW_MOTION_ROTATING) {
    const double* n = mp + 6;
    const double vv = std::sqrt(mp[3] * mp[3] + mp[4] * mp[4] + mp[5] * mp[5]);
    for (int c = 0; c < 8; ++c) {
      double x[3];
      for (int a = 0; a < 3; ++a) x[a] = ((c >> a) & 1) ? d.hi[a] : d.lo[a];
      const double cr[3] = {n[1] * x[2] - n[2] * x[1], n[2] * x[0] - n[0] * x[2], n[0] * x[1] - n[1] * x[0]};
      for (int a = 0; a < 3; ++a) v[a] = std::max(v[a], std::fabs(mp[9]) * std::fabs(cr[a]) + vv);
    }
  }
}

bool is_moving(const mpw_patch_desc& d) {
  double v[3];
  max_speed(d, v);
  return v[0] != 0.0 || v[1] != 0.0 || v[2] != 0.0;
}

Geom make_geom(const mpw_patch_desc& d, int esize = 8) {
  double h[3];
  for (int a = 0; a < 3; ++a) h[a] = (d.hi[a] - d.lo[a]) / d.n[a];
  return padded_geom(d.n, d.lo, h, esize);
}

// Covered box of local patch l on the global grid at time t (Sec. 2.4.2,
// "Find Covered Zones"): global cell centres inside the closed live box of l,
// tested in l's numeric coordinates.  Under translation the covered set is a
// product of one index interval per axis.  A rotating patch covers a rotated
// box: the result is then a bounding box of its cells (one cell of margin
// around the cells whose centres lie in the background extent), and the
// cover kernel tests every cell in it.
Box covered_box(const PatchState& g, const PatchState& l, double t) {
  double X0[3], w[3];
  motion(l.d, t, X0, w);
  Box b;
  if (l.d.motion == MPW_MOTION_ROTATING || l.sph()) {
    double lo[3], hi[3];
    background_extent(l.d, t, 0.0, lo, hi);
    for (int a = 0; a < 3; ++a) {
      const double h = (g.d.hi[a] - g.d.lo[a]) / g.d.n[a];
      b.lo[a] = std::max(0, (int)std::ceil((lo[a] - g.d.lo[a]) / h - 0.5) - 1);
      b.hi[a] = std::min(g.d.n[a] - 1, (int)std::floor((hi[a] - g.d.lo[a]) / h - 0.5) + 1);
    }
    return b;
  }
  for (int a = 0; a < 3; ++a) {
    b.lo[a] = 1 << 30;
    b.hi[a] = -1;
    const double h = (g.d.hi[a] - g.d.lo[a]) / g.d.n[a];
    for (int i = 0; i < g.d.n[a]; ++i) {
      const double x = g.d.lo[a] + (i + 0.5) * h;
      const double xl = x - X0[a];
      if (l.d.lo[a] <= xl && xl <= l.d.hi[a]) {
        b.lo[a] = std::min(b.lo[a], i);
        b.hi[a] = std::max(b.hi[a], i);
      }
    }
  }
  return b;
}

bool box_empty(const Box& b) { return b.lo[0] > b.hi[0] || b.lo[1] > b.hi[1] || b.lo[2] > b.hi[2]; }

mpw_status check_ctx(const mpw_ctx* c) {
  if (!c) return set_err(MPW_ERR_ARG, "null context");
  return MPW_OK;
}

mpw_status use_device(mpw_ctx* c) {
  CUDA_TRY(cudaSetDevice(c->cfg.device));
  return MPW_OK;
}

mpw_status ensure_stage(mpw_ctx* c, size_t bytes) {
  if (c->stage_bytes >= bytes) return MPW_OK;
  c->dfree(c->d_stage);
  c->d_stage = (double*)c->dalloc(bytes);
  c->stage_bytes = c->d_stage ? bytes : 0;
  if (!c->d_stage) return set_err(MPW_ERR_CUDA, "staging allocation of %zu bytes failed", bytes);
  return MPW_OK;
}

// Validation of a step of size dt from time t (the checks the paper leaves to
// the user, Sec. 2.4.2, plus the RK4 stability estimate).
mpw_status validate_step(mpw_ctx* c, double dt, double t) {
  if (!(dt > 0.0) || !std::isfinite(dt)) return set_err(MPW_ERR_ARG, "dt must be positive and finite");
  const PatchState& g = c->p[0];
  const double h0 = std::min(g.g.h[0], std::min(g.g.h[1], g.g.h[2]));
  for (size_t q = 0; q < c->p.size(); ++q) {
    const PatchState& P = c->p[q];
    double v[3];
    max_speed(P.d, v);
    const double sp = max_point_speed(P.d);
    // RK4 stays stable on the imaginary axis up to 2 sqrt(2); the 4th-order
    // Laplacian reaches 16/(3 h^2) per axis, the 4th-order first derivative
    // 1.372/h.
    double lap = 0.0, adv = 0.0;
    if (P.sph()) {
      // physical spacings at the smallest radius and sin(theta)
      const double smin = std::min(std::sin(P.d.lo[1]), std::sin(P.d.hi[1]));
      const double L[3] = {P.g.h[0], P.d.lo[0] * P.g.h[1], P.d.lo[0] * smin * P.g.h[2]};
      for (int a = 0; a < 3; ++a) {
        lap += 16.0 / (3.0 * L[a] * L[a]);
        adv += 1.372 * sp / L[a];
      }
    } else {
      for (int a = 0; a < 3; ++a) {
        lap += 16.0 / (3.0 * P.g.h[a] * P.g.h[a]);
        adv += 1.372 * v[a] / P.g.h[a];
      }
    }
    if (dt * (std::sqrt(lap) + adv) > 2.8)
      return set_err(MPW_ERR_CFL, "patch %zu: dt = %g exceeds the RK4 stability estimate", q, dt);
    if (q == 0) continue;
    // the buffer of B live cells lets a patch cross B - NG global cells per
    // step (a rotating patch: its fastest point, on every axis)
    for (int a = 0; a < 3; ++a)
      if ((P.d.motion == MPW_MOTION_ROTATING || P.sph() ? sp : v[a]) * dt > (c->buffer - NG) * g.g.h[a])
        return set_err(MPW_ERR_TRAVERSAL, "patch %zu crosses more than %d global cell(s) per step", q,
                       c->buffer - NG);
  }
  const double ts[3] = {t, t + 0.5 * dt, t + dt};
  for (double tt : ts) {
    for (size_t q = 1; q < c->p.size(); ++q) {
      const PatchState& P = c->p[q];
      double X0[3], w[3];
      motion(P.d, tt, X0, w);
      if (P.d.motion == MPW_MOTION_ROTATING || P.sph()) {
        // the ghost-extended box, rotated (a shell: its ball); the samples are dt/2 apart
        double lo[3], hi[3];
        background_extent(P.d, tt, NG, lo, hi);
        const double slack = max_point_speed(P.d) * 0.5 * dt;
        for (int a = 0; a < 3; ++a) {
          const double margin = (NG + 2) * g.g.h[a] + slack;
          if (lo[a] - margin < g.d.lo[a] || hi[a] + margin > g.d.hi[a])
            return set_err(MPW_ERR_OUTSIDE, "patch %zu leaves the global interior at t = %g", q, tt);
        }
      }
      for (int a = 0; a < 3; ++a) {
        const double margin = NG * P.g.h[a] + (NG + 2) * g.g.h[a];
        if (P.d.motion != MPW_MOTION_ROTATING && !P.sph() &&
            (P.d.lo[a] + X0[a] - margin < g.d.lo[a] || P.d.hi[a] + X0[a] + margin > g.d.hi[a]))
          return set_err(MPW_ERR_OUTSIDE, "patch %zu leaves the global interior at t = %g", q, tt);
      }
      double plo[3], phi[3];
      background_extent(P.d, tt, 0.0, plo, phi);
      for (size_t r = q + 1; r < c->p.size(); ++r) {
        const PatchState& R = c->p[r];
        double rlo[3], rhi[3];
        background_extent(R.d, tt, 0.0, rlo, rhi);
        double gap = -1e300;
        for (int a = 0; a < 3; ++a) {
          const double g1 = rlo[a] - phi[a];
          const double g2 = plo[a] - rhi[a];
          gap = std::max(gap, std::max(g1, g2));
        }
        if (gap < 2.0 * h0)
          return set_err(MPW_ERR_OVERLAP, "patches %zu and %zu are closer than 2 global cells at t = %g", q, r, tt);
      }
    }
  }
  return MPW_OK;
}

// Cover flags at time t; revival uses the previous flags when valid.
// revive = false: the cells that turn live keep what u holds there (the NaN
// of a dead cell).  Only for the steps inside a hybrid call, where u of the
// global is not read before it is rewritten: every Global-to-Local donor lies
// in the boxes the Hermite stage states overwrite, and the call ends by
// writing the surrogate's state over all of u.
// The arguments of the cover-flag launch at time t (covered boxes, visited
// regions, revival queue); launch = false when no flag can change (then the
// flags are already valid).  run_flags launches them; a batched step gathers
// them for one launch over its instances.
mpw_status prep_flags(mpw_ctx* c, double t, bool revive, FlagArgs& a, bool& launch) {
  const PatchState& g = c->p[0];
  launch = false;
  a = FlagArgs{};
  a.flags = c->d_flags;
  for (int k = 0; k < 3; ++k) a.n[k] = g.d.n[k];
  a.nloc = (int)c->p.size() - 1;
  const std::vector<Box> old_boxes = c->boxes;
  const bool restrict_cells = c->flags_valid && (int)old_boxes.size() == a.nloc;
  c->boxes.assign(a.nloc, Box{});
  long long ncov = 0;
  for (int q = 0; q < a.nloc; ++q) {
    const PatchState& L = c->p[q + 1];
    c->boxes[q] = covered_box(g, L, t);
    a.box[q] = c->boxes[q];
    a.Uloc[q] = L.buf(BUF_U);
    a.gl[q] = L.g;
    const Frame f = frame(L.d, t);
    a.rot[q] = f.rot ? 1 : 0;
    a.sph[q] = L.sph() ? 1 : 0;
    a.cth[q][0] = std::cos(L.d.lo[1]);
    a.cth[q][1] = std::cos(L.d.hi[1]);
    for (int e = 0; e < 9; ++e) a.R[q][e] = f.R[e];
    for (int k = 0; k < 3; ++k) {
      a.X0[q][k] = f.X0[k];
      a.lhi[q][k] = L.d.hi[k];
    }
    // X'_a = sum_b R_ba (lo_b + (idx_b + 1/2) h_b - X0_b), affine in the
    // global cell indices, rounded to binary32 for the screen.  Its error is
    // at most about 6 units of 2^-24 of the largest |term| sum, E; the
    // margin is 1e-5 E, above 25 times that.
    double E = 0.0;
    for (int r = 0; r < 3; ++r) {
      double c = 0.0, e = 0.0;
      for (int m = 0; m < 3; ++m) {
        a.scr[q][r][m] = (float)(f.R[3 * m + r] * g.g.h[m]);
        c += f.R[3 * m + r] * (g.g.lo[m] + 0.5 * g.g.h[m] - f.X0[m]);
        e += std::fabs(f.R[3 * m + r] * g.g.h[m]) * g.d.n[m];
      }
      a.scr[q][r][3] = (float)c;
      E = std::max(E, e + std::fabs(c) + std::fabs(L.d.lo[r]) + std::fabs(L.d.hi[r]));
    }
    a.scrm[q] = (float)(1e-5 * E);
    a.cov_off[q] = ncov;
    if ((f.rot || L.sph()) && !box_empty(c->boxes[q])) {
      const Box& b = c->boxes[q];
      ncov += (long long)(b.hi[0] - b.lo[0] + 1) * (b.hi[1] - b.lo[1] + 1) * (b.hi[2] - b.lo[2] + 1);
    }
  }
  a.cov_off[a.nloc] = ncov;
  c->glist_valid = false;
  if ((size_t)ncov > c->cov_bytes) {
    c->dfree(c->d_cov);
    c->dfree(c->d_glist);
    // the shells' distance transform uses two more regions of the same size
    c->d_cov = (uint8_t*)c->dalloc(3 * (size_t)ncov);
    c->d_glist = (long long*)c->dalloc(sizeof(long long) * (size_t)ncov);
    c->cov_bytes = c->d_cov && c->d_glist ? (size_t)ncov : 0;
    if (!c->cov_bytes) return set_err(MPW_ERR_CUDA, "covered-mask allocation for %lld cells failed", ncov);
  }
  if (ncov > 0 && !c->d_gcount) {
    c->d_gcount = (int*)c->dalloc(sizeof(int) * MAX_PATCHES);
    if (!c->d_gcount) return set_err(MPW_ERR_CUDA, "ghost-list counter allocation failed");
  }
  a.cov = c->d_cov;
  a.glist = ncov > 0 ? c->d_glist : nullptr;
  a.gcount = ncov > 0 ? c->d_gcount : nullptr;
  c->glist_off.assign(a.cov_off, a.cov_off + a.nloc);
  // With valid flags only cells inside an old or a new covered box can change:
  // visit the bounding box of each pair, merging regions until disjoint.
  a.nreg = 0;
  if (restrict_cells) {
    std::vector<Box> reg;
    for (int q = 0; q < a.nloc; ++q) {
      const Box& o = old_boxes[q];
      const Box& nw = c->boxes[q];
      Box r{};
      bool any = false;
      for (const Box* bx : {&o, &nw}) {
        if (box_empty(*bx)) continue;
        for (int k = 0; k < 3; ++k) {
          r.lo[k] = any ? std::min(r.lo[k], bx->lo[k]) : bx->lo[k];
          r.hi[k] = any ? std::max(r.hi[k], bx->hi[k]) : bx->hi[k];
        }
        any = true;
      }
      if (any) reg.push_back(r);
    }
    for (bool merged = true; merged;) {
      merged = false;
      for (size_t x = 0; x < reg.size() && !merged; ++x)
        for (size_t y = x + 1; y < reg.size() && !merged; ++y) {
          bool overlap = true;
          for (int k = 0; k < 3; ++k) overlap = overlap && reg[x].lo[k] <= reg[y].hi[k] && reg[y].lo[k] <= reg[x].hi[k];
          if (!overlap) continue;
          for (int k = 0; k < 3; ++k) {
            reg[x].lo[k] = std::min(reg[x].lo[k], reg[y].lo[k]);
            reg[x].hi[k] = std::max(reg[x].hi[k], reg[y].hi[k]);
          }
          reg.erase(reg.begin() + y);
          merged = true;
        }
    }
    long long pos = 0;
    for (size_t q = 0; q < reg.size(); ++q) {
      a.reg[q] = reg[q];
      a.reg_begin[q] = pos;
      pos += (long long)(reg[q].hi[0] - reg[q].lo[0] + 1) * (reg[q].hi[1] - reg[q].lo[1] + 1) *
             (reg[q].hi[2] - reg[q].lo[2] + 1);
    }
    a.reg_begin[reg.size()] = pos;
    a.nreg = (int)reg.size();
    if (a.nreg == 0) {  // nothing covered before or now: no flag can change
      c->flags_valid = true;
      return MPW_OK;
    }
  }
  a.buffer = c->buffer;
  a.old_valid = c->flags_valid ? 1 : 0;
  a.skip_revive = revive ? 0 : 1;
  a.Ug = g.buf(BUF_U);
  a.gg = g.g;
  a.P = c->P;
  a.err = c->d_err;
  a.expo = c->d_expo;
  a.rev_list = c->d_rev;
  a.rev_count = c->d_err + 32;
  a.rev_cap = REVIVE_CAP;
  a.f32 = c->cfg.precision == 32;
  launch = true;
  return MPW_OK;
}

mpw_status run_flags(mpw_ctx* c, double t, bool revive = true) {
  FlagArgs a;
  bool launch;
  const std::vector<Box> old_boxes = c->boxes;
  const bool old_valid = c->flags_valid, old_glist = c->glist_valid;
  if (mpw_status st = prep_flags(c, t, revive, a, launch)) {
    // nothing launched: the device flags still belong to the old boxes
    c->boxes = old_boxes;
    c->flags_valid = old_valid;
    c->glist_valid = old_glist;
    return st;
  }
  if (!launch) return MPW_OK;
  c->launch_begin(MPW_KERNEL_FLAGS);
  const int kernels = launch_flags(a, c->stream);  // flags kernel, plus the revival kernel when old flags exist
  c->launches[MPW_KERNEL_FLAGS] += kernels - 1;
  c->launch_end(MPW_KERNEL_FLAGS);
  CUDA_TRY(cudaGetLastError());
  c->flags_valid = true;
  c->glist_valid = a.glist != nullptr;
  return MPW_OK;
}

// Tile extent for one slab of an interpolation segment: the thin axis takes
// the slab thickness, the two wide axes the largest candidate whose blocks
// fit the separable kernel's budget.  Donor extents are bounded as the
// kernel computes them: (T - 1) * ratio spans at most floor of that plus one
// donor, plus the P nodes of the last window.
void choose_tile(const double ratio[3], int P, int thin, const int extent[3], int td[3]) {
  static const int cand[][2] = {{32, 32}, {32, 16}, {16, 32}, {16, 16}, {32, 8}, {8, 32}, {16, 8}, {8, 16},
                                {8, 8},   {8, 4},   {4, 8},   {4, 4},   {2, 2}, {1, 1}};
  const int wa = thin == 0 ? 1 : 0, wb = thin == 2 ? 1 : 2;
  for (const auto& cd : cand) {
    int T[3];
    T[thin] = extent[thin];
    T[wa] = std::min(cd[0], extent[wa]);
    T[wb] = std::min(cd[1], extent[wb]);
    long long Dn[3];
    for (int a = 0; a < 3; ++a) Dn[a] = (long long)std::floor((T[a] - 1) * ratio[a]) + 1 + P;
    const long long r1 = T[thin] * Dn[wa] * Dn[wb];
    const long long r2 = std::min(T[thin] * T[wa] * Dn[wb], T[thin] * Dn[wa] * T[wb]);
    const bool ok = T[wa] <= fill_max_tile() && T[wb] <= fill_max_tile() && T[thin] <= NG &&
                    Dn[thin] <= fill_max_thin_donors() && r1 <= fill_cap_r1() && r2 <= fill_cap_r2();
    if (ok || (cd[0] == 1 && cd[1] == 1)) {
      for (int a = 0; a < 3; ++a) td[a] = std::max(T[a], 1);
      return;
    }
  }
}

// Tile extent for one slab of a rotated ghost shell: the largest candidate
// whose donor box fits the shared-memory block of the fixed-point tile path.
// The donor index is affine in the target index with slopes M_ab h_t[b] /
// h_d[a]; the kernel widens the covered range by the window (P) and three
// cells of margin.
void choose_tile_affine(const InterpSeg& S, int P, int thin, const int extent[3], int td[3]) {
  static const int cand[][2] = {{16, 16}, {16, 8}, {8, 16}, {8, 8}, {8, 4}, {4, 8}, {4, 4}, {2, 2}, {1, 1}};
  const int wa = thin == 0 ? 1 : 0, wb = thin == 2 ? 1 : 2;
  const long long cap = fill_cap_r1() + fill_cap_r2();
  for (const auto& cd : cand) {
    int T[3];
    T[thin] = extent[thin];
    T[wa] = std::min(cd[0], extent[wa]);
    T[wb] = std::min(cd[1], extent[wb]);
    long long vol = 1;
    for (int a = 0; a < 3; ++a) {
      double span = 0.0;
      for (int b = 0; b < 3; ++b) span += std::fabs(S.M[3 * a + b]) * (T[b] - 1) * S.gt.h[b] / S.gd.h[a];
      vol *= (long long)std::floor(span * (1.0 + 1e-12)) + 1 + P + 3;
    }
    if (vol <= cap || (cd[0] == 1 && cd[1] == 1)) {
      for (int a = 0; a < 3; ++a) td[a] = std::max(T[a], 1);
      return;
    }
  }
}

// Affine map of a rotated segment from target cell indices to donor index
// coordinates: s_a = sum_b (M_ab h_t[b] / h_d[a]) idx_b
//                    + (sum_b M_ab (lo_t[b] + h_t[b] / 2) + shift_a - lo_d[a]) / h_d[a] - 1/2.
void set_index_map(InterpSeg& S) {
  for (int a = 0; a < 3; ++a) {
    double c = S.shift[a];
    for (int b = 0; b < 3; ++b) {
      S.sidx[a][b] = S.M[3 * a + b] * S.gt.h[b] / S.gd.h[a];
      c += S.M[3 * a + b] * (S.gt.lo[b] + 0.5 * S.gt.h[b]);
    }
    S.sidx[a][3] = (c - S.gd.lo[a]) / S.gd.h[a] - 0.5;
  }
}

// Cut the hollow box (origin O0, extent O, walls NG thick) into six slabs and
// tile them; returns the number of CTAs.
int build_segment(InterpSeg& S, const int O0[3], const int O[3], int P) {
  int lo[3], hi[3];  // wall thickness at the low / high end of each axis
  for (int a = 0; a < 3; ++a) {
    lo[a] = std::min(NG, O[a]);
    hi[a] = std::min(NG, O[a] - lo[a]);
  }
  const int mid0[3] = {lo[0], lo[1], lo[2]};
  const int midn[3] = {O[0] - lo[0] - hi[0], O[1] - lo[1] - hi[1], O[2] - lo[2] - hi[2]};
  int sb[6][3], se[6][3];
  // z-, z+
  for (int k = 0; k < 2; ++k) {
    sb[k][0] = 0, se[k][0] = O[0];
    sb[k][1] = 0, se[k][1] = O[1];
    sb[k][2] = k ? O[2] - hi[2] : 0, se[k][2] = k ? hi[2] : lo[2];
  }
  // y-, y+ (between the z walls)
  for (int k = 0; k < 2; ++k) {
    sb[2 + k][0] = 0, se[2 + k][0] = O[0];
    sb[2 + k][1] = k ? O[1] - hi[1] : 0, se[2 + k][1] = k ? hi[1] : lo[1];
    sb[2 + k][2] = mid0[2], se[2 + k][2] = midn[2];
  }
  // x-, x+ (between the z and y walls)
  for (int k = 0; k < 2; ++k) {
    sb[4 + k][0] = k ? O[0] - hi[0] : 0, se[4 + k][0] = k ? hi[0] : lo[0];
    sb[4 + k][1] = mid0[1], se[4 + k][1] = midn[1];
    sb[4 + k][2] = mid0[2], se[4 + k][2] = midn[2];
  }
  double ratio[3];
  for (int a = 0; a < 3; ++a) ratio[a] = S.gt.h[a] / S.gd.h[a];
  int blocks = 0;
  for (int sl = 0; sl < 6; ++sl) {
    S.slab_block0[sl] = blocks;
    for (int a = 0; a < 3; ++a) {
      S.sb[sl][a] = O0[a] + sb[sl][a];
      S.se[sl][a] = se[sl][a];
    }
    if (se[sl][0] <= 0 || se[sl][1] <= 0 || se[sl][2] <= 0) {
      S.tn[sl][0] = S.tn[sl][1] = 0;
      for (int a = 0; a < 3; ++a) S.td[sl][a] = 1;
      continue;
    }
    if (S.kind == SEG_AFFINE)
      choose_tile_affine(S, P, sl / 2 == 0 ? 2 : (sl / 2 == 1 ? 1 : 0), se[sl], S.td[sl]);
    else
      choose_tile(ratio, P, sl / 2 == 0 ? 2 : (sl / 2 == 1 ? 1 : 0), se[sl], S.td[sl]);
    int n[3];
    for (int a = 0; a < 3; ++a) n[a] = (se[sl][a] + S.td[sl][a] - 1) / S.td[sl][a];
    S.tn[sl][0] = n[0];
    S.tn[sl][1] = n[1];
    blocks += n[0] * n[1] * n[2];
  }
  return blocks;
}

// CTAs that stride over one rotating patch's list of effective ghosts.
constexpr int L2G_LIST_BLOCKS = 152;

// Ghost fill of the stage buffer `b` at time t; clears the exponent slots of
// buffer reset_buf (the output of the following RHS launch), if >= 0.
// Fixed-point mirrors for the shells of c at time t (fill of buffer b): per
// shell, the global cells its ghost nodes' windows can reach (the ball of
// its ghost-extended radius, widened by the window) and its own padded box.
// mir_global[q] / mir_shell[q]: region of local patch q, or -1.
mpw_status prep_mirrors(mpw_ctx* c, int b, double t, MirrorArgs& m, int mir_global[], int mir_shell[]) {
  m = MirrorArgs{};
  const PatchState& g = c->p[0];
  const int nloc = (int)c->p.size() - 1;
  for (int q = 0; q < nloc; ++q) mir_global[q] = mir_shell[q] = -1;
  if (c->cfg.arith == 1 || c->cfg.precision != 64) return MPW_OK;
  // capacity from the shells' radii, the same at every substage (a batch
  // prepares four substages before it enqueues them)
  size_t need = 0;
  for (int q = 0; q < nloc; ++q) {
    const PatchState& L = c->p[q + 1];
    if (!L.sph()) continue;
    const double R = L.d.hi[0] + NG * L.g.h[0];
    size_t vg = 1, vs = 1;
    for (int a = 0; a < 3; ++a) {
      vg *= (size_t)std::ceil(2.0 * R / g.g.h[a]) + 9;
      vs *= (size_t)(L.d.n[a] + 2 * NG);
    }
    need += 2 * (vg + vs);
  }
  for (int q = 0; q < nloc; ++q) {
    const PatchState& L = c->p[q + 1];
    if (!L.sph()) continue;
    double lo[3], hi[3];
    background_extent(L.d, t, NG, lo, hi);
    MirrorRegion& G = m.r[m.nr];
    G.src = g.buf(b);
    G.g = g.g;
    G.patch = 0;
    for (int a = 0; a < 3; ++a) {
      const int l0 = (int)std::floor((lo[a] - g.g.lo[a]) / g.g.h[a] - 0.5) - 3;
      const int h0 = std::min((int)std::floor((hi[a] - g.g.lo[a]) / g.g.h[a] - 0.5) + 4,
                              l0 + (int)std::ceil(2.0 * (hi[a] - lo[a]) / 2.0 / g.g.h[a]) + 8);
      G.box.lo[a] = std::max(-NG, l0);
      G.box.hi[a] = std::min(g.d.n[a] + NG - 1, h0);
    }
    mir_global[q] = m.nr++;
    MirrorRegion& S = m.r[m.nr];
    S.src = L.buf(b);
    S.g = L.g;
    S.patch = q + 1;
    for (int a = 0; a < 3; ++a) {
      S.box.lo[a] = -NG;
      S.box.hi[a] = L.d.n[a] + NG - 1;
    }
    mir_shell[q] = m.nr++;
  }
  long long blocks = 0;
  for (int r = 0; r < m.nr; ++r) {
    const Box& bx = m.r[r].box;
    const long long vol = (long long)(bx.hi[0] - bx.lo[0] + 1) * (bx.hi[1] - bx.lo[1] + 1) * (bx.hi[2] - bx.lo[2] + 1);
    m.r[r].block0 = blocks;
    blocks += (vol + 255) / 256;
  }
  m.blocks = blocks;
  m.expo = c->d_expo;
  m.y_buf = b;
  if (need > c->mirror_cap) {
    c->dfree(c->d_mirror);
    c->d_mirror = (int2*)c->dalloc(sizeof(int2) * need);
    c->mirror_cap = c->d_mirror ? need : 0;
    if (!c->d_mirror) return set_err(MPW_ERR_CUDA, "mirror allocation of %zu entries failed", need);
  }
  size_t off = 0;
  for (int r = 0; r < m.nr; ++r) {
    const Box& bx = m.r[r].box;
    m.r[r].dst = c->d_mirror + off;
    off += 2 * (size_t)(bx.hi[0] - bx.lo[0] + 1) * (bx.hi[1] - bx.lo[1] + 1) * (bx.hi[2] - bx.lo[2] + 1);
  }
  return MPW_OK;
}

// Which segments a fill runs: all of them (the method's substages), the
// Global-to-Local ones only (the hybrid substages of mpw_step_surrogate, where
// nothing reads the global's outer ghosts or its Local-to-Global ring), or the
// Local-to-Global ones only (the start of a hybrid call, where only the
// global's covered cells are read).
enum FillParts { FILL_ALL = 0, FILL_G2L = 1, FILL_L2G = 2 };

// gdonor >= 0 (Global-to-Local fills only): the global patch donates from
// buffer gdonor instead of b, and the fill clears no exponent slot of the
// global patch (the hybrid step lays the global's stage states out in their
// own buffers ahead of the substages).
mpw_status prep_fill(mpw_ctx* c, int b, double t, int reset_buf, FillArgs& a, MirrorArgs* mirrors = nullptr,
                     int parts = FILL_ALL, int gdonor = -1) {
  const bool g2l_only = parts == FILL_G2L, l2g_only = parts == FILL_L2G;
  if (gdonor >= 0 && !g2l_only) return set_err(MPW_ERR_STATE, "a global donor buffer needs a Global-to-Local fill");
  const PatchState& g = c->p[0];
  a = FillArgs{};
  int mir_global[MAX_PATCHES], mir_shell[MAX_PATCHES];
  for (int q = 0; q < MAX_PATCHES; ++q) mir_global[q] = mir_shell[q] = -1;
  MirrorArgs local_m{};
  MirrorArgs& m = mirrors ? *mirrors : local_m;  // without a launch slot: the per-tap path
  if (mirrors)
    if (mpw_status st = prep_mirrors(c, b, t, m, mir_global, mir_shell)) return st;
  a.Yg = g.buf(b);
  a.gg = g.g;
  a.outer_bc = g.d.outer_bc == MPW_BC_PERIODIC ? 1 : 0;
  if (a.outer_bc == 0 && c->akind < 0) return set_err(MPW_ERR_STATE, "analytic outer BC without mpw_set_analytic");
  a.akind = c->akind;
  a.acount = c->acount;
  a.aparams = c->d_aparams;
  a.ascreen = c->screen_ok ? c->d_ascreen : nullptr;
  a.apre = c->screen_ok ? c->d_apre : nullptr;
  a.shell_src = nullptr;
  if (a.outer_bc == 0 && parts == FILL_ALL) {
    for (int k = 0; k < 4; ++k)
      if (k != b && c->shell_time[k] == t) a.shell_src = g.buf(k);
    c->shell_time[b] = t;
  }
  a.t = t;
  a.outer_count = (long long)(g.d.n[0] + 2 * NG) * (g.d.n[1] + 2 * NG) * (g.d.n[2] + 2 * NG) -
                  (long long)g.d.n[0] * g.d.n[1] * g.d.n[2];
  if (parts != FILL_ALL) a.outer_count = 0;
  a.outer_blocks = (int)((a.outer_count + fill_threads() - 1) / fill_threads());
  int blocks = a.outer_blocks;
  a.nseg = 0;
  const int nloc = (int)c->p.size() - 1;
  // Local-to-Global: the effective-ghost shell of each covered box
  for (int q = 0; q < (g2l_only ? 0 : nloc); ++q) {
    const Box& bx = c->boxes[q];
    if (box_empty(bx)) continue;
    int O0[3], O[3];
    bool any = true;
    for (int k = 0; k < 3; ++k) {
      O0[k] = bx.lo[k] + c->buffer;
      O[k] = bx.hi[k] - bx.lo[k] + 1 - 2 * c->buffer;
      any = any && O[k] > 0;
    }
    if (!any) continue;
    const PatchState& L = c->p[q + 1];
    InterpSeg& S = a.seg[a.nseg++];
    S.T = g.buf(b);
    S.gt = g.g;
    S.tpatch = 0;
    S.dpatch = q + 1;
    S.D = L.buf(b);
    S.gd = L.g;
    const Frame f = frame(L.d, t);
    S.block0 = blocks;
    S.sph = L.sph() ? 1 : 0;
    if (f.rot || L.sph()) {
      // the effective ghosts of a rotated box, mapped by X' = R^T X_B - R^T X0:
      // the list the cover-flag kernel wrote, or (flags set through the ABI)
      // every cell of the covered bounding box whose flag says GHOST of this
      // patch
      for (int r = 0; r < 3; ++r) {
        S.shift[r] = 0.0;
        for (int k = 0; k < 3; ++k) {
          S.M[3 * r + k] = f.R[3 * k + r];
          S.shift[r] -= f.R[3 * k + r] * f.X0[k];
        }
      }
      set_index_map(S);
      S.mir = nullptr;
      if (L.sph() && mir_shell[q] >= 0) {
        S.mir = m.r[mir_shell[q]].dst;
        S.mbox = m.r[mir_shell[q]].box;
      }
      if (c->glist_valid && q < (int)c->glist_off.size()) {
        S.kind = SEG_LIST;
        S.list = c->d_glist + c->glist_off[q];
        S.count = c->d_gcount + q;
        S.list_blocks = L2G_LIST_BLOCKS;
        blocks += L2G_LIST_BLOCKS;
        continue;
      }
      S.kind = SEG_MASKED;
      S.box = bx;
      S.flags = c->d_flags;
      S.want = FLAG_GHOST | ((q + 1) << 2);
      const long long vol = (long long)(bx.hi[0] - bx.lo[0] + 1) * (bx.hi[1] - bx.lo[1] + 1) * (bx.hi[2] - bx.lo[2] + 1);
      blocks += (int)((vol + fill_threads() - 1) / fill_threads());
      continue;
    }
    S.kind = SEG_SHELL;
    for (int k = 0; k < 3; ++k) S.shift[k] = -f.X0[k];
    blocks += build_segment(S, O0, O, c->P);
  }
  // Global-to-Local: the ghost shell of each local patch
  for (int q = 0; q < (l2g_only ? 0 : nloc); ++q) {
    const PatchState& L = c->p[q + 1];
    InterpSeg& S = a.seg[a.nseg++];
    S.T = L.buf(b);
    S.gt = L.g;
    S.tpatch = q + 1;
    S.dpatch = 0;
    S.D = g.buf(gdonor >= 0 ? gdonor : b);
    S.gd = g.g;
    const Frame f = frame(L.d, t);
    // a rotated ghost shell: per-point sums through X_B = R X' + X0 (fixed-point
    // tiles with the donor box in shared memory, or direct FP64 sums)
    S.kind = f.rot ? SEG_AFFINE : SEG_SHELL;
    for (int e = 0; e < 9; ++e) S.M[e] = f.R[e];
    for (int k = 0; k < 3; ++k) S.shift[k] = f.X0[k];
    if (L.sph()) {
      // every ghost node of a spherical shell, one thread each
      S.kind = SEG_SPH_GHOSTS;
      S.mir = nullptr;
      if (mir_global[q] >= 0) {
        S.mir = m.r[mir_global[q]].dst;
        S.mbox = m.r[mir_global[q]].box;
      }
      S.block0 = blocks;
      const long long cnt = (long long)(L.d.n[0] + 2 * NG) * (L.d.n[1] + 2 * NG) * (L.d.n[2] + 2 * NG) -
                            (long long)L.d.n[0] * L.d.n[1] * L.d.n[2];
      blocks += (int)((cnt + fill_threads() - 1) / fill_threads());
      continue;
    }
    if (f.rot) set_index_map(S);
    const int O0[3] = {-NG, -NG, -NG};
    const int O[3] = {L.d.n[0] + 2 * NG, L.d.n[1] + 2 * NG, L.d.n[2] + 2 * NG};
    S.block0 = blocks;
    blocks += build_segment(S, O0, O, c->P);
  }
  a.total_blocks = blocks;
  a.P = c->P;
  a.err = c->d_err;
  a.expo = c->d_expo;
  a.y_buf = b;
  a.reset_buf = reset_buf;
  a.reset_first = gdonor >= 0 ? 1 : 0;
  a.gdonor_use = gdonor >= 0 ? 1 : 0;
  a.gdonor_buf = gdonor >= 0 ? gdonor : 0;
  a.np = (int)c->p.size();
  a.fixed = c->cfg.arith != 1;
  a.f32 = c->cfg.precision == 32;
  return MPW_OK;
}

mpw_status run_fill(mpw_ctx* c, int b, double t, int reset_buf, int parts = FILL_ALL, int gdonor = -1) {
  FillArgs a;
  MirrorArgs m;
  if (mpw_status st = prep_fill(c, b, t, reset_buf, a, &m, parts, gdonor)) return st;
  c->launch_begin(MPW_KERNEL_FILL);
  if (m.nr > 0) {
    launch_mirror(m, c->stream);
    c->launches[MPW_KERNEL_FILL] += 1;
  }
  launch_fill(a, c->stream);
  c->launch_end(MPW_KERNEL_FILL);
  CUDA_TRY(cudaGetLastError());
  return MPW_OK;
}

// One fused RHS + RK4 stage launch over every patch (substage l at t).
// RHS + stage arguments of substage l for every patch of c; returns the
// number of CTAs.  zc: planes per CTA chunk (0: the default).
// The fixed-point RHS body converts one x/y halo point per thread: the
// 6 TX + 6 TY halo points of a tile need that many of its TX TY threads.
static_assert(6 * RHS_TX + 6 * RHS_TY <= RHS_TX * RHS_TY, "RHS tile too small for its halo (MPW_RHS_TY >= 8)");

int prep_rhs(mpw_ctx* c, int l, double t, double dt, RhsArgs& a, int zc = 0, bool skip_global = false) {
  static const int in_buf[4] = {BUF_U, BUF_YA, BUF_YB, BUF_YA};
  static const int out_buf[4] = {BUF_YA, BUF_YB, BUF_YA, BUF_U};
  a = RhsArgs{};
  a.np = (int)c->p.size();
  a.stage = l;
  // OUT = U + alpha K (l < 3) or ACC + alpha K (l = 3); ACC = base + beta K
  const double alpha[4] = {0.5 * dt, 0.5 * dt, dt, dt / 6.0};
  const double beta[4] = {dt / 6.0, dt / 3.0, dt / 3.0, 0.0};
  a.alpha = alpha[l];
  a.beta = beta[l];
  a.flags = c->d_flags;
  a.nbox = (int)c->boxes.size();
  for (int q = 0; q < a.nbox; ++q) a.box[q] = c->boxes[q];
  a.expo = c->d_expo;
  a.err = c->d_err;
  a.wait_limit = c->wait_limit;
  int blocks = 0;
  for (int q = 0; q < a.np; ++q) {
    const PatchState& P = c->p[q];
    RhsPatch& R = a.p[q];
    R.ymap = P.tile_map[in_buf[l]];
    R.umap = P.point_map[0];
    R.amap = P.point_map[1];
    R.Y = P.buf(in_buf[l]);
    R.U = P.buf(BUF_U);
    R.ACC = P.buf(BUF_ACC);
    R.OUT = P.buf(out_buf[l]);
    R.g = P.g;
    const Frame f = frame(P.d, t);
    R.moving = 0;
    R.rot = f.rot && is_moving(P.d) ? 1 : 0;
    for (int k = 0; k < 3; ++k) {
      const double h = P.g.h[k];
      // c1 at cell (0, 0, 0): w0 + W X'(0, 0, 0); steps W_kb h_b per index
      double wk = f.w0[k];
      for (int m = 0; m < 3; ++m) wk += f.W[3 * k + m] * (P.g.lo[m] + 0.5 * P.g.h[m]);
      R.c1[k] = wk / (12.0 * h);
      for (int m = 0; m < 3; ++m) R.c1g[k][m] = f.W[3 * k + m] * P.g.h[m] / (12.0 * h);
      R.c2[k] = 1.0 / (12.0 * h * h);
      R.cko[k] = c->cfg.ko_eps / (64.0 * h);
      if (wk != 0.0) R.moving = 1;
    }
    if (R.rot) R.moving = 1;
    R.is_global = q == 0 && c->flags_valid && !c->boxes.empty();
    R.iso = P.g.h[0] == P.g.h[1] && P.g.h[1] == P.g.h[2];
    R.in_buf = in_buf[l];
    R.out_buf = out_buf[l];
    R.tiles_x = (P.d.n[0] + RHS_TX - 1) / RHS_TX;
    R.tiles_y = (P.d.n[1] + RHS_TY - 1) / RHS_TY;
    R.zc = zc > 0 ? zc : default_rhs_chunk(P.d.n[2], c->cfg.precision == 32);
    R.zchunks = (P.d.n[2] + R.zc - 1) / R.zc;
    R.block0 = blocks;
    if (P.sph()) continue;  // spherical shells: k_rhs_shell
    if (skip_global && q == 0) continue;  // the global patch advanced by other means
    blocks += R.tiles_x * R.tiles_y * R.zchunks;
  }
  return blocks;
}

// RHS + stage arguments of substage l for the spherical shells of c, appended
// to a (a.np shells so far, `blocks` CTAs so far: one launch may cover the
// shells of several contexts); returns the new CTA count, or -1 when a
// would overflow (nothing appended then).
long long prep_rhs_shell(mpw_ctx* c, int l, double t, double dt, ShellArgs& a, long long blocks = 0) {
  static const int in_buf[4] = {BUF_U, BUF_YA, BUF_YB, BUF_YA};
  static const int out_buf[4] = {BUF_YA, BUF_YB, BUF_YA, BUF_U};
  const double alpha[4] = {0.5 * dt, 0.5 * dt, dt, dt / 6.0};
  const double beta[4] = {dt / 6.0, dt / 3.0, dt / 3.0, 0.0};
  int ns = 0;
  for (size_t q = 1; q < c->p.size(); ++q) ns += c->p[q].sph() ? 1 : 0;
  if (a.np + ns > MAX_SHELLS) return -1;
  a.stage = l;
  a.in_buf = in_buf[l];
  a.out_buf = out_buf[l];
  for (size_t q = 1; q < c->p.size(); ++q) {
    const PatchState& P = c->p[q];
    if (!P.sph()) continue;
    ShellPatch& S = a.p[a.np++];
    S.expo = c->d_expo;
    S.alpha = alpha[l];
    S.beta = beta[l];
    S.tab = P.tab;
    for (int a2 = 0; a2 < 3; ++a2) {
      S.id1[a2] = 1.0 / (12.0 * P.g.h[a2]);
      S.id2[a2] = 1.0 / (12.0 * P.g.h[a2] * P.g.h[a2]);
      S.iko[a2] = c->cfg.ko_eps / (64.0 * P.g.h[a2]);
    }
    S.Y = P.buf(in_buf[l]);
    S.U = P.buf(BUF_U);
    S.ACC = P.buf(BUF_ACC);
    S.OUT = P.buf(out_buf[l]);
    S.g = P.g;
    const Frame f = frame(P.d, t);
    for (int e = 0; e < 9; ++e) {
      S.R[e] = f.R[e];
      S.W[e] = f.W[e];
    }
    for (int k = 0; k < 3; ++k) S.w0[k] = f.w0[k];
    S.moving = is_moving(P.d) ? 1 : 0;
    S.patch = (int)q;
    S.block0 = blocks;
    blocks += ((long long)P.d.n[0] * P.d.n[1] * P.d.n[2] + 255) / 256;
  }
  return blocks;
}

mpw_status run_rhs(mpw_ctx* c, int l, double t, double dt, bool skip_global = false) {
  RhsArgs a;
  const int blocks = prep_rhs(c, l, t, dt, a, 0, skip_global);
  bool rot = false;
  for (int q = 0; q < a.np; ++q) rot = rot || a.p[q].rot;
  ShellArgs sa{};
  const long long sblocks = prep_rhs_shell(c, l, t, dt, sa);
  c->launch_begin(MPW_KERNEL_RHS);
  if (blocks == 0)
    c->launches[MPW_KERNEL_RHS] -= 1;  // nothing to launch (only shells, or the skipped global patch)
  else if (c->cfg.precision == 32)
    launch_rhs32(a, blocks, rot, c->stream);
  else
    launch_rhs(a, blocks, c->cfg.arith != 1, rot, c->stream);
  if (sblocks > 0) {
    launch_rhs_shell(sa, sblocks, c->stream);
    c->launches[MPW_KERNEL_RHS] += 1;
  }
  c->launch_end(MPW_KERNEL_RHS);
  CUDA_TRY(cudaGetLastError());
  return MPW_OK;
}

// Recompute the exponent slots of u for patches whose u was written from
// outside a step (creation, set_fields, fill_analytic).
mpw_status ensure_u_exponents(mpw_ctx* c) {
  if (c->cfg.precision == 32) return MPW_OK;  // the slots scale binary64 fixed-point arithmetic only
  for (size_t q = 0; q < c->p.size(); ++q) {
    PatchState& P = c->p[q];
    if (P.u_expo_valid) continue;
    int* slot2 = c->d_expo + q * EXP_SLOTS_PER_PATCH + BUF_U * 2;
    CUDA_TRY(cudaMemsetAsync(slot2, 0, 2 * sizeof(int), c->stream));
    launch_expo_scan(P.buf(BUF_U), P.g, (q == 0 && c->flags_valid) ? c->d_flags : nullptr, slot2, c->stream);
    CUDA_TRY(cudaGetLastError());
    P.u_expo_valid = true;
  }
  return MPW_OK;
}

// FP32 screening data of Gaussian pulses (centre, radius): sqrt(50) widths
// plus a slack that covers FP32 rounding of coordinates of magnitude up to
// the largest patch or centre coordinate.
mpw_status upload_screen(mpw_ctx* c) {
  c->screen_ok = false;
  if ((c->akind != MPW_ANALYTIC_GAUSS_SUM && c->akind != MPW_ANALYTIC_PLANE_GAUSS) || c->acount <= 0) return MPW_OK;
  // the pulses' parameters (after the plane wave for PLANE_GAUSS)
  const double* params = c->aparams.data() + (c->akind == MPW_ANALYTIC_PLANE_GAUSS ? 6 : 0);
  double extent = 1.0;
  for (const auto& P : c->p)
    for (int a = 0; a < 3; ++a) extent = std::max(extent, std::max(std::fabs(P.d.lo[a]), std::fabs(P.d.hi[a])));
  for (int q = 0; q < c->acount; ++q)
    for (int a = 0; a < 3; ++a) extent = std::max(extent, std::fabs(params[5 * q + 2 + a]));
  c->screen.resize(c->acount);
  c->apre.resize(c->acount);
  for (int q = 0; q < c->acount; ++q) {
    const double* g = params + 5 * q;
    const double R = std::sqrt(50.0) * std::fabs(g[1]) * (1.0 + 1e-5) + 1e-5 * (4.0 * extent);
    c->screen[q] = make_float4((float)g[2], (float)g[3], (float)g[4], (float)R);
    c->apre[q] = 1.0 / (g[1] * g[1]);
  }
  CUDA_TRY(cudaMemcpyAsync(c->d_ascreen, c->screen.data(), sizeof(float4) * c->acount, cudaMemcpyHostToDevice,
                           c->stream));
  CUDA_TRY(cudaMemcpyAsync(c->d_apre, c->apre.data(), sizeof(double) * c->acount, cudaMemcpyHostToDevice,
                           c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  c->screen_ok = true;
  return MPW_OK;
}

mpw_status read_error_word(mpw_ctx* c) {
  CUDA_TRY(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  const int e = *c->h_err;
  if (e) {
    CUDA_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    if (e & ERR_TIMEOUT) return set_err(MPW_ERR_TIMEOUT, "a bounded device wait ran out (error word 0x%x)", e);
    if (e & ERR_UNFILLED) return set_err(MPW_ERR_GHOST_UNFILLED, "a ghost point could not be interpolated");
    return set_err(MPW_ERR_CUDA, "unexpected device error word 0x%x", e);
  }
  return MPW_OK;
}

}  // namespace

namespace mpw {
void set_last_error(const char* msg) { g_last_error = msg; }
}  // namespace mpw

// ============================================================================ C ABI

extern "C" {

static mpw_status apply_pending_inputs(mpw_ctx* c);

const char* mpw_last_error(void) { return g_last_error.c_str(); }

mpw_status mpw_create(const mpw_config* cfg, mpw_ctx** out) {
  if (!cfg || !out) return set_err(MPW_ERR_ARG, "null argument");
  *out = nullptr;
  if (cfg->precision != 64 && cfg->precision != 32) return set_err(MPW_ERR_ARG, "precision must be 64 or 32");
  if (cfg->ghost != NG) return set_err(MPW_ERR_ARG, "ghost must be %d", NG);
  if (cfg->interp_points != 5 && cfg->interp_points != 6) return set_err(MPW_ERR_ARG, "interp_points must be 5 or 6");
  if (!(cfg->ko_eps >= 0.0)) return set_err(MPW_ERR_ARG, "ko_eps must be >= 0");
  const int buffer = cfg->buffer > 0 ? cfg->buffer : NG + 1;
  if (buffer < NG + 1) return set_err(MPW_ERR_ARG, "buffer must be at least NG + 1 = %d", NG + 1);
  if ((cfg->alloc == nullptr) != (cfg->free == nullptr)) return set_err(MPW_ERR_ARG, "alloc and free go together");
  mpw_ctx* c = new mpw_ctx();
  c->cfg = *cfg;
  c->P = cfg->interp_points;
  c->buffer = buffer;
  c->stream = (cudaStream_t)cfg->stream;
  mpw_status st = use_device(c);
  if (st != MPW_OK) {
    delete c;
    return st;
  }
  c->d_err = (int*)c->dalloc(256);
  c->d_aparams = (double*)c->dalloc(sizeof(double) * MAX_APARAMS);
  c->d_ascreen = (float4*)c->dalloc(sizeof(float4) * (MAX_APARAMS / 5 + 1));
  c->d_apre = (double*)c->dalloc(sizeof(double) * (MAX_APARAMS / 5 + 1));
  c->d_expo = (int*)c->dalloc(sizeof(int) * MAX_PATCHES * EXP_SLOTS_PER_PATCH);
  c->d_rev = (long long*)c->dalloc(sizeof(long long) * REVIVE_CAP);
  if (!c->d_err || !c->d_aparams || !c->d_ascreen || !c->d_apre || !c->d_expo || !c->d_rev ||
      cudaMallocHost(&c->h_err, sizeof(int)) != cudaSuccess) {
    mpw_destroy(c);
    return set_err(MPW_ERR_CUDA, "context allocation failed");
  }
  if (cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->d_expo, 0, sizeof(int) * MAX_PATCHES * EXP_SLOTS_PER_PATCH, c->stream) != cudaSuccess) {
    mpw_destroy(c);
    return set_err(MPW_ERR_CUDA, "memset failed");
  }
  *out = c;
  return MPW_OK;
}

void mpw_destroy(mpw_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->cfg.device);
  cudaStreamSynchronize(c->stream);
  if (c->io_in) cudaStreamSynchronize(c->io_in);
  if (c->io_out) cudaStreamSynchronize(c->io_out);
  for (auto& P : c->p) {
    c->dfree(P.base);
    c->dfree(P.tab);
    c->dfree(P.io_in);
    c->dfree(P.io_out);
    for (cudaEvent_t e : {P.in_copied, P.in_free, P.out_packed, P.out_free})
      if (e) cudaEventDestroy(e);
  }
  if (c->io_in) cudaStreamDestroy(c->io_in);
  if (c->io_out) cudaStreamDestroy(c->io_out);
  c->dfree(c->d_flags);
  c->dfree(c->d_err);
  c->dfree(c->d_aparams);
  c->dfree(c->d_ascreen);
  c->dfree(c->d_apre);
  c->dfree(c->d_expo);
  c->dfree(c->d_rev);
  c->dfree(c->d_cov);
  c->dfree(c->d_glist);
  c->dfree(c->d_gcount);
  c->dfree(c->d_mirror);
  c->dfree(c->d_stage);
  c->dfree(c->d_sur);
  if (c->h_err) cudaFreeHost(c->h_err);
  for (auto& v : c->ev)
    for (cudaEvent_t e : v) cudaEventDestroy(e);
  delete c;
}

mpw_status mpw_create_patch(mpw_ctx* c, const mpw_patch_desc* d, int* patch_id) {
  mpw_status st = check_ctx(c);
  if (st) return st;
  if (!d || !patch_id) return set_err(MPW_ERR_ARG, "null argument");
  if (c->stepped) return set_err(MPW_ERR_STATE, "patches must be created before the first step");
  if ((c->p.empty()) != (d->kind == MPW_PATCH_GLOBAL))
    return set_err(MPW_ERR_STATE, "the global patch must be created first, and only once");
  if ((int)c->p.size() >= MAX_PATCHES) return set_err(MPW_ERR_ARG, "at most %d patches", MAX_PATCHES);
  for (int a = 0; a < 3; ++a) {
    if (d->n[a] < 2 * NG) return set_err(MPW_ERR_ARG, "n[%d] must be >= %d", a, 2 * NG);
    if (!(d->hi[a] > d->lo[a])) return set_err(MPW_ERR_ARG, "hi must exceed lo");
  }
  if (d->motion < MPW_MOTION_STATIC || d->motion > MPW_MOTION_ROTATING) return set_err(MPW_ERR_ARG, "bad motion law");
  if (d->motion == MPW_MOTION_ROTATING) {
    const double* n = d->motion_params + 6;
    if (!(std::fabs(n[0] * n[0] + n[1] * n[1] + n[2] * n[2] - 1.0) <= 1e-12))
      return set_err(MPW_ERR_ARG, "the rotation axis must be a unit vector");
    if (d->kind == MPW_PATCH_GLOBAL) return set_err(MPW_ERR_ARG, "the global patch cannot rotate");
  }
  if (d->kind == MPW_PATCH_GLOBAL) {
    if (d->topology != MPW_TOPOLOGY_CARTESIAN) return set_err(MPW_ERR_ARG, "the global patch is Cartesian");
    if (d->outer_bc != MPW_BC_ANALYTIC && d->outer_bc != MPW_BC_PERIODIC)
      return set_err(MPW_ERR_ARG, "global outer_bc must be ANALYTIC or PERIODIC");
  } else {
    if (d->outer_bc != MPW_BC_INTERPATCH) return set_err(MPW_ERR_ARG, "local outer_bc must be INTERPATCH");
    const mpw_patch_desc& g = c->p[0].d;
    if (g.motion != MPW_MOTION_STATIC || g.motion_params[0] != 0.0 || g.motion_params[1] != 0.0 ||
        g.motion_params[2] != 0.0)
      return set_err(MPW_ERR_ARG, "with local patches the global patch must be static at the origin");
    const Geom gg = make_geom(g);
    if (d->topology == MPW_TOPOLOGY_SPHERICAL) {
      const double hr = (d->hi[0] - d->lo[0]) / d->n[0], ht = (d->hi[1] - d->lo[1]) / d->n[1];
      const double hp = (d->hi[2] - d->lo[2]) / d->n[2], pi = 3.14159265358979323846;
      const double hg = std::min(gg.h[0], std::min(gg.h[1], gg.h[2])) * (1.0 + 1e-12);
      if (c->cfg.precision != 64) return set_err(MPW_ERR_ARG, "spherical shells run in precision 64 only");
      if (d->lo[0] - NG * hr <= 0.0 || d->lo[1] - NG * ht <= 0.0 || d->hi[1] + NG * ht >= pi)
        return set_err(MPW_ERR_ARG, "shell ghost nodes must stay off the origin and the poles");
      if (d->lo[2] != 0.0 || std::fabs(d->hi[2] - 2.0 * pi) > 1e-12)
        return set_err(MPW_ERR_ARG, "a shell spans the full azimuth [0, 2 pi)");
      if (hr > hg || d->hi[0] * ht > hg || d->hi[0] * hp > hg)
        return set_err(MPW_ERR_ARG, "a shell's physical spacings must not exceed the global spacing");
    } else if (d->topology != MPW_TOPOLOGY_CARTESIAN) {
      return set_err(MPW_ERR_ARG, "bad topology");
    } else {
      for (int a = 0; a < 3; ++a)
        if ((d->hi[a] - d->lo[a]) / d->n[a] > gg.h[a] * (1.0 + 1e-12))
          return set_err(MPW_ERR_ARG, "a local patch must not be coarser than the global patch");
    }
  }
  if (use_device(c)) return MPW_ERR_CUDA;
  PatchState P;
  P.d = *d;
  const bool f32 = c->cfg.precision == 32;
  P.esize = f32 ? 4 : 8;
  P.g = make_geom(*d, (int)P.esize);
  const size_t bytes = P.esize * 8 * (size_t)P.g.vol;
  P.base = (double*)c->dalloc(bytes);
  if (!P.base) return set_err(MPW_ERR_CUDA, "allocation of %zu bytes failed", bytes);
  // every failure below frees what this call allocated
  auto undo = [&](const char* msg) {
    c->dfree(P.base);
    return set_err(MPW_ERR_CUDA, "%s", msg);
  };
  if (cudaMemsetAsync(P.base, 0, bytes, c->stream) != cudaSuccess) return undo("memset of the new patch failed");
  for (int b = 0; b < 4; ++b)
    if (!encode_rhs_map(&P.tile_map[b], P.buf(b), P.g, true, f32)) return undo("tensor map encoding failed");
  if (!encode_rhs_map(&P.point_map[0], P.buf(BUF_U), P.g, false, f32) ||
      !encode_rhs_map(&P.point_map[1], P.buf(BUF_ACC), P.g, false, f32))
    return undo("tensor map encoding failed");
  if (d->topology == MPW_TOPOLOGY_SPHERICAL) {
    // node tables: r, 1/r; sin, cos, 1/sin of theta; sin, cos of phi
    std::vector<double> t;
    for (int i = 0; i < d->n[0]; ++i) t.push_back(P.g.lo[0] + (i + 0.5) * P.g.h[0]);
    for (int i = 0; i < d->n[0]; ++i) t.push_back(1.0 / (P.g.lo[0] + (i + 0.5) * P.g.h[0]));
    for (int j = 0; j < d->n[1]; ++j) t.push_back(std::sin(P.g.lo[1] + (j + 0.5) * P.g.h[1]));
    for (int j = 0; j < d->n[1]; ++j) t.push_back(std::cos(P.g.lo[1] + (j + 0.5) * P.g.h[1]));
    for (int j = 0; j < d->n[1]; ++j) t.push_back(1.0 / std::sin(P.g.lo[1] + (j + 0.5) * P.g.h[1]));
    for (int k = 0; k < d->n[2]; ++k) t.push_back(std::sin(P.g.lo[2] + (k + 0.5) * P.g.h[2]));
    for (int k = 0; k < d->n[2]; ++k) t.push_back(std::cos(P.g.lo[2] + (k + 0.5) * P.g.h[2]));
    P.tab = (double*)c->dalloc(sizeof(double) * t.size());
    if (!P.tab) return undo("shell table allocation failed");
    if (cudaMemcpy(P.tab, t.data(), sizeof(double) * t.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
      c->dfree(P.tab);
      return undo("shell table upload failed");
    }
  }
  if (d->kind == MPW_PATCH_GLOBAL) {
    const size_t nb = (size_t)d->n[0] * d->n[1] * d->n[2];
    c->d_flags = (uint8_t*)c->dalloc(nb);
    if (!c->d_flags) return undo("flag allocation failed");
    if (cudaMemsetAsync(c->d_flags, 0, nb, c->stream) != cudaSuccess) {
      c->dfree(c->d_flags);
      c->d_flags = nullptr;
      return undo("memset of the cover flags failed");
    }
  }
  c->p.push_back(P);
  c->flags_valid = false;
  if (mpw_status st2 = upload_screen(c)) return st2;
  *patch_id = (int)c->p.size() - 1;
  return MPW_OK;
}

mpw_status mpw_set_analytic(mpw_ctx* c, int kind, const double* params, int count) {
  mpw_status st = check_ctx(c);
  if (st) return st;
  int need = 0;
  if (kind == MPW_ANALYTIC_GAUSS_SUM)
    need = 5 * count;
  else if (kind == MPW_ANALYTIC_PLANE_SUM)
    need = 1 + 5 * count;
  else if (kind == MPW_ANALYTIC_HARMONIC_POLY)
    need = count;
  else if (kind == MPW_ANALYTIC_PLANE_GAUSS)
    need = 6 + 5 * count;
  else
    return set_err(MPW_ERR_ARG, "unknown analytic kind %d", kind);
  if (count < 0 || need > MAX_APARAMS || (kind == MPW_ANALYTIC_HARMONIC_POLY && count > 14) || (need && !params))
    return set_err(MPW_ERR_ARG, "bad analytic parameter count");
  if (use_device(c)) return MPW_ERR_CUDA;
  c->akind = kind;
  c->acount = count;
  for (double& st2 : c->shell_time) st2 = NAN;
  c->aparams.assign(params, params + need);
  if (need) CUDA_TRY(cudaMemcpyAsync(c->d_aparams, c->aparams.data(), sizeof(double) * need, cudaMemcpyHostToDevice,
                                     c->stream));
  if ((st = upload_screen(c))) return st;
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return MPW_OK;
}

mpw_status mpw_fill_analytic(mpw_ctx* c, double t) {
  mpw_status st = check_ctx(c);
  if (st) return st;
  if (c->akind < 0) return set_err(MPW_ERR_STATE, "no analytic function set");
  if (use_device(c)) return MPW_ERR_CUDA;
  if ((st = apply_pending_inputs(c))) return st;
  for (auto& P : c->p) {
    const Frame f = frame(P.d, t);
    Affine map;
    for (int e = 0; e < 9; ++e) map.R[e] = f.R[e];
    for (int k = 0; k < 3; ++k) map.X0[k] = f.X0[k];
    launch_analytic(P.buf(BUF_U), P.g, map, c->akind, c->acount, c->d_aparams,
                    c->screen_ok ? c->d_ascreen : nullptr, c->screen_ok ? c->d_apre : nullptr, t,
                    c->cfg.precision == 32, c->stream, P.sph());
    CUDA_TRY(cudaGetLastError());
    P.u_expo_valid = false;
  }
  c->t = t;
  return MPW_OK;
}

static mpw_status get_patch(mpw_ctx* c, int patch, PatchState** out) {
  mpw_status st = check_ctx(c);
  if (st) return st;
  if (patch < 0 || patch >= (int)c->p.size()) return set_err(MPW_ERR_ARG, "bad patch id %d", patch);
  *out = &c->p[patch];
  return use_device(c);
}

// Staging buffers, events and copy streams of the asynchronous host IO of
// patch P (allocated on first use).
static mpw_status ensure_async_io(mpw_ctx* c, PatchState& P) {
  if (!c->io_in) {
    CUDA_TRY(cudaStreamCreateWithFlags(&c->io_in, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamCreateWithFlags(&c->io_out, cudaStreamNonBlocking));
  }
  if (!P.io_in) {
    const size_t bytes = 2 * sizeof(double) * (size_t)P.d.n[0] * P.d.n[1] * P.d.n[2];
    P.io_in = (double*)c->dalloc(bytes);
    P.io_out = (double*)c->dalloc(bytes);
    if (!P.io_in || !P.io_out) return set_err(MPW_ERR_CUDA, "IO staging allocation of %zu bytes failed", bytes);
    for (cudaEvent_t* e : {&P.in_copied, &P.in_free, &P.out_packed, &P.out_free})
      CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  }
  return MPW_OK;
}

// Inputs queued by mpw_set_fields_async enter u, in stream order, before
// anything reads or writes u.
// Unpack new values into u of patch q.  On binary64 contexts the same pass
// raises u's live exponent slots when it can tell the live cells: every cell
// of a local patch, and the global's by the current cover flags (a cell those
// flags exclude and the next flags make live is revived, which raises the
// slot itself; a cell they count and the next flags drop only raises the
// bound).  Otherwise the slots are recomputed before the next step.
static mpw_status unpack_u(mpw_ctx* c, size_t q, const double* s0, const double* s1) {
  PatchState& P = c->p[q];
  const bool single = c->p.size() == 1;
  if (c->cfg.precision == 64 && (q > 0 || single || c->flags_valid)) {
    int* slot2 = c->d_expo + q * EXP_SLOTS_PER_PATCH + BUF_U * 2;
    CUDA_TRY(cudaMemsetAsync(slot2, 0, 2 * sizeof(int), c->stream));
    launch_unpack_scan(static_cast<double*>(P.buf(BUF_U)), P.g, s0, s1, q == 0 && !single ? c->d_flags : nullptr,
                       slot2, c->stream);
    CUDA_TRY(cudaGetLastError());
    P.u_expo_valid = true;
    return MPW_OK;
  }
  launch_unpack(P.buf(BUF_U), P.g, s0, s1, c->cfg.precision == 32, c->stream);
  CUDA_TRY(cudaGetLastError());
  P.u_expo_valid = false;
  return MPW_OK;
}

static mpw_status apply_pending_inputs(mpw_ctx* c) {
  for (size_t q = 0; q < c->p.size(); ++q) {
    PatchState& P = c->p[q];
    if (!P.in_pending) continue;
    const size_t n = (size_t)P.d.n[0] * P.d.n[1] * P.d.n[2];
    CUDA_TRY(cudaStreamWaitEvent(c->stream, P.in_copied, 0));
    if (mpw_status st = unpack_u(c, q, P.io_in, P.io_in + n)) return st;
    CUDA_TRY(cudaEventRecord(P.in_free, c->stream));
    P.in_pending = false;
  }
  return MPW_OK;
}

// Device alias of a page-locked host array (cudaHostAlloc, cudaMallocHost or
// cudaHostRegister'ed memory mapped into the device address space), or null
// for pageable memory.  The pack and unpack kernels read and write such an
// array in place, so the host copy needs no staging buffer and no copy engine.
static void* pinned_alias(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // pageable memory on older drivers reports an error
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

mpw_status mpw_set_fields(mpw_ctx* c, int patch, const double* psi, const double* pi, int on_device) {
  PatchState* P;
  mpw_status st = get_patch(c, patch, &P);
  if (st) return st;
  if (!psi || !pi) return set_err(MPW_ERR_ARG, "null field pointer");
  if ((st = apply_pending_inputs(c))) return st;
  const size_t n = (size_t)P->d.n[0] * P->d.n[1] * P->d.n[2];
  const double *s0 = psi, *s1 = pi;
  const double* a0 = on_device ? nullptr : (const double*)pinned_alias(psi);
  const double* a1 = on_device ? nullptr : (const double*)pinned_alias(pi);
  if (a0 && a1) {
    s0 = a0;
    s1 = a1;
  } else if (!on_device) {
    if ((st = ensure_stage(c, 2 * n * sizeof(double)))) return st;
    CUDA_TRY(cudaMemcpyAsync(c->d_stage, psi, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaMemcpyAsync(c->d_stage + n, pi, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    s0 = c->d_stage;
    s1 = c->d_stage + n;
  }
  if ((st = unpack_u(c, (size_t)patch, s0, s1))) return st;
  if (!on_device) CUDA_TRY(cudaStreamSynchronize(c->stream));
  return MPW_OK;
}

static mpw_status get_impl(mpw_ctx* c, int patch, double* psi, double* pi, int on_device, int padded) {
  PatchState* P;
  mpw_status st = get_patch(c, patch, &P);
  if (st) return st;
  if (!psi || !pi) return set_err(MPW_ERR_ARG, "null field pointer");
  if ((st = apply_pending_inputs(c))) return st;
  const int e = padded ? 2 * NG : 0;
  const size_t n = (size_t)(P->d.n[0] + e) * (P->d.n[1] + e) * (P->d.n[2] + e);
  const uint8_t* flags = (patch == 0 && c->flags_valid) ? c->d_flags : nullptr;
  double* a0 = on_device ? nullptr : (double*)pinned_alias(psi);
  double* a1 = on_device ? nullptr : (double*)pinned_alias(pi);
  if (on_device || (a0 && a1)) {
    launch_pack(P->buf(BUF_U), P->g, on_device ? psi : a0, on_device ? pi : a1, padded, flags,
                c->cfg.precision == 32, c->stream);
    CUDA_TRY(cudaGetLastError());
  } else {
    if ((st = ensure_stage(c, 2 * n * sizeof(double)))) return st;
    launch_pack(P->buf(BUF_U), P->g, c->d_stage, c->d_stage + n, padded, flags, c->cfg.precision == 32, c->stream);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(psi, c->d_stage, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaMemcpyAsync(pi, c->d_stage + n, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return MPW_OK;
}

mpw_status mpw_get_fields(mpw_ctx* c, int patch, double* psi, double* pi, int on_device) {
  return get_impl(c, patch, psi, pi, on_device, 0);
}

mpw_status mpw_set_fields_async(mpw_ctx* c, int patch, const double* psi, const double* pi) {
  PatchState* P;
  mpw_status st = get_patch(c, patch, &P);
  if (st) return st;
  if (!psi || !pi) return set_err(MPW_ERR_ARG, "null field pointer");
  if (!pinned_alias(psi) || !pinned_alias(pi))
    return set_err(MPW_ERR_ARG, "asynchronous host transfers need page-locked host arrays");
  if ((st = ensure_async_io(c, *P))) return st;
  const size_t n = (size_t)P->d.n[0] * P->d.n[1] * P->d.n[2];
  // the previous input has left the staging buffer (its unpack ran)
  CUDA_TRY(cudaStreamWaitEvent(c->io_in, P->in_free, 0));
  CUDA_TRY(cudaMemcpyAsync(P->io_in, psi, n * sizeof(double), cudaMemcpyHostToDevice, c->io_in));
  CUDA_TRY(cudaMemcpyAsync(P->io_in + n, pi, n * sizeof(double), cudaMemcpyHostToDevice, c->io_in));
  CUDA_TRY(cudaEventRecord(P->in_copied, c->io_in));
  P->in_pending = true;
  return MPW_OK;
}

mpw_status mpw_get_fields_async(mpw_ctx* c, int patch, double* psi, double* pi) {
  PatchState* P;
  mpw_status st = get_patch(c, patch, &P);
  if (st) return st;
  if (!psi || !pi) return set_err(MPW_ERR_ARG, "null field pointer");
  if (!pinned_alias(psi) || !pinned_alias(pi))
    return set_err(MPW_ERR_ARG, "asynchronous host transfers need page-locked host arrays");
  if ((st = ensure_async_io(c, *P))) return st;
  if ((st = apply_pending_inputs(c))) return st;
  const size_t n = (size_t)P->d.n[0] * P->d.n[1] * P->d.n[2];
  const uint8_t* flags = (patch == 0 && c->flags_valid) ? c->d_flags : nullptr;
  // the previous result has left the staging buffer (its copy ran)
  CUDA_TRY(cudaStreamWaitEvent(c->stream, P->out_free, 0));
  launch_pack(P->buf(BUF_U), P->g, P->io_out, P->io_out + n, 0, flags, c->cfg.precision == 32, c->stream);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaEventRecord(P->out_packed, c->stream));
  CUDA_TRY(cudaStreamWaitEvent(c->io_out, P->out_packed, 0));
  CUDA_TRY(cudaMemcpyAsync(psi, P->io_out, n * sizeof(double), cudaMemcpyDeviceToHost, c->io_out));
  CUDA_TRY(cudaMemcpyAsync(pi, P->io_out + n, n * sizeof(double), cudaMemcpyDeviceToHost, c->io_out));
  CUDA_TRY(cudaEventRecord(P->out_free, c->io_out));
  return MPW_OK;
}

mpw_status mpw_sync(mpw_ctx* c) {
  mpw_status st = check_ctx(c);
  if (st) return st;
  if (use_device(c)) return MPW_ERR_CUDA;
  if (c->io_in) CUDA_TRY(cudaStreamSynchronize(c->io_in));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (c->io_out) CUDA_TRY(cudaStreamSynchronize(c->io_out));
  return read_error_word(c);  // device-side errors of mpw_step_async calls
}

mpw_status mpw_get_padded(mpw_ctx* c, int patch, double* psi, double* pi, int on_device) {
  return get_impl(c, patch, psi, pi, on_device, 1);
}

mpw_status mpw_set_time(mpw_ctx* c, double t) {
  mpw_status st = check_ctx(c);
  if (st) return st;
  c->t = t;
  return MPW_OK;
}

double mpw_time(const mpw_ctx* c) { return c ? c->t : NAN; }

mpw_status mpw_compute_flags(mpw_ctx* c) {
  mpw_status st = check_ctx(c);
  if (st) return st;
  if (c->p.empty()) return set_err(MPW_ERR_STATE, "no global patch");
  if (use_device(c)) return MPW_ERR_CUDA;
  if ((st = apply_pending_inputs(c))) return st;
  if ((st = run_flags(c, c->t))) return st;
  return read_error_word(c);
}

mpw_status mpw_get_flags(mpw_ctx* c, uint8_t* flags) {
  mpw_status st = check_ctx(c);
  if (st) return st;
  if (c->p.empty() || !flags) return set_err(MPW_ERR_ARG, "no global patch or null pointer");
  if (use_device(c)) return MPW_ERR_CUDA;
  const size_t nb = (size_t)c->p[0].d.n[0] * c->p[0].d.n[1] * c->p[0].d.n[2];
  CUDA_TRY(cudaMemcpyAsync(flags, c->d_flags, nb, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return MPW_OK;
}

mpw_status mpw_set_flags(mpw_ctx* c, const uint8_t* flags) {
  mpw_status st = check_ctx(c);
  if (st) return st;
  if (c->p.empty() || !flags) return set_err(MPW_ERR_ARG, "no global patch or null pointer");
  if (use_device(c)) return MPW_ERR_CUDA;
  const PatchState& g = c->p[0];
  const size_t nb = (size_t)g.d.n[0] * g.d.n[1] * g.d.n[2];
  CUDA_TRY(cudaMemcpyAsync(c->d_flags, flags, nb, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  c->boxes.assign(c->p.size() - 1, Box{});
  for (size_t q = 1; q < c->p.size(); ++q) c->boxes[q - 1] = covered_box(g, c->p[q], c->t);
  c->flags_valid = true;
  c->glist_valid = false;  // the ghost lists come from the flags kernel only
  return MPW_OK;
}

mpw_status mpw_set_wait_limit(mpw_ctx* c, unsigned limit) {
  mpw_status st = check_ctx(c);
  if (st) return st;
  c->wait_limit = limit;
  return MPW_OK;
}

mpw_status mpw_fill_ghosts(mpw_ctx* c, double t) {
  mpw_status st = check_ctx(c);
  if (st) return st;
  if (c->p.empty()) return set_err(MPW_ERR_STATE, "no global patch");
  if (use_device(c)) return MPW_ERR_CUDA;
  if ((st = apply_pending_inputs(c))) return st;
  if (!c->flags_valid && (st = run_flags(c, c->t))) return st;
  if ((st = ensure_u_exponents(c))) return st;
  if ((st = run_fill(c, BUF_U, t, -1))) return st;
  return read_error_word(c);
}

}  // extern "C"

namespace {
const int FILL_BUF[4] = {BUF_U, BUF_YA, BUF_YB, BUF_YA};
const int NEXT_BUF[4] = {BUF_YA, BUF_YB, BUF_YA, BUF_U};

bool any_moving(const mpw_ctx* c) {
  for (size_t q = 1; q < c->p.size(); ++q)
    if (is_moving(c->p[q].d)) return true;
  return false;
}

// What a step does before its substages: validation at t_n, the cover flags
// (every step when a patch moves, once otherwise) and the exponent slots of u.
mpw_status step_prologue(mpw_ctx* c, double dt, bool revive = true) {
  mpw_status st;
  const double tn = c->t;
  if ((st = validate_step(c, dt, tn))) return st;
  if (any_moving(c) || !c->flags_valid)
    if ((st = run_flags(c, tn, revive))) return st;
  return ensure_u_exponents(c);
}
}  // namespace

extern "C" {

static mpw_status step_impl(mpw_ctx* c, double dt, int nsteps, bool check_errors);

mpw_status mpw_step(mpw_ctx* c, double dt, int nsteps) { return step_impl(c, dt, nsteps, true); }

mpw_status mpw_step_async(mpw_ctx* c, double dt, int nsteps) { return step_impl(c, dt, nsteps, false); }

static mpw_status step_impl(mpw_ctx* c, double dt, int nsteps, bool check_errors) {
  mpw_status st = check_ctx(c);
  if (st) return st;
  if (c->p.empty()) return set_err(MPW_ERR_STATE, "no global patch");
  if (nsteps < 0) return set_err(MPW_ERR_ARG, "nsteps must be >= 0");
  if (use_device(c)) return MPW_ERR_CUDA;
  if ((st = apply_pending_inputs(c))) return st;
  for (int s = 0; s < nsteps; ++s) {
    const double tn = c->t;
    if ((st = step_prologue(c, dt))) return st;
    const int* fill_buf = FILL_BUF;
    const int* next_buf = NEXT_BUF;
    for (int l = 0; l < 4; ++l) {
      const double tl = tn + RK_C[l] * dt;
      if ((st = run_fill(c, fill_buf[l], tl, next_buf[l]))) return st;
      if ((st = run_rhs(c, l, tl, dt))) return st;
    }
    c->t = tn + dt;
    c->stepped = true;
  }
  return check_errors ? read_error_word(c) : MPW_OK;
}

// The dead global cells of the U buffer from their local patches (the cover
// flags and boxes of t_n; translating Cartesian local patches).
static mpw_status fill_dead_cells(mpw_ctx* c) {
  const PatchState& g = c->p[0];
  FlagArgs a{};
  a.flags = c->d_flags;
  for (int k = 0; k < 3; ++k) a.n[k] = g.d.n[k];
  a.nloc = (int)c->p.size() - 1;
  if (a.nloc == 0 || (int)c->boxes.size() != a.nloc) return MPW_OK;
  for (int q = 0; q < a.nloc; ++q) {
    const PatchState& L = c->p[q + 1];
    a.box[q] = c->boxes[q];
    a.Uloc[q] = L.buf(BUF_U);
    a.gl[q] = L.g;
    const Frame f = frame(L.d, c->t);
    for (int k = 0; k < 3; ++k) a.X0[q][k] = f.X0[k];
  }
  a.Ug = g.buf(BUF_U);
  a.gg = g.g;
  a.P = c->P;
  a.err = c->d_err;
  launch_fill_dead(a, c->stream);
  CUDA_TRY(cudaGetLastError());
  return MPW_OK;
}

// Quintic Hermite basis on [0, 1] as coefficients of tau^0..tau^5: value,
// first and second derivative at 0, then at 1.
static const double HERMITE5[6][6] = {{1, 0, 0, -10, 15, -6}, {0, 1, 0, -6, 8, -3},  {0, 0, 0.5, -1.5, 1.5, -0.5},
                                      {0, 0, 0, 10, -15, 6},  {0, 0, 0, -4, 7, -3}, {0, 0, 0, 0.5, -1.0, 0.5}};

// k-th derivative in tau of the polynomial c at tau
static double poly_derivative(const double c[6], int k, double tau) {
  double s = 0.0;
  for (int p = 5; p >= k; --p) {
    double f = 1.0;
    for (int r = 0; r < k; ++r) f *= p - r;
    s = s * tau + c[p] * f;
  }
  return s;
}

// Weights of (y0, y0', y0'', y1, y1', y1'') -- the state at both ends of a
// call and its first two time derivatives -- in the input of RK4 stage l of
// step m (of the four one call spans).  For the linear system u' = A u the
// stage inputs of the method are u, u + dt/2 u', u + dt/2 u' + dt^2/4 u'' and
// u + dt u' + dt^2/2 u'' + dt^3/4 u''' (Table 1 applied to A); u and its
// derivatives are those of the interpolant at t_n + m dt.
static void stage_coefficients(int m, int l, double D, double cf[6]) {
  static const double mult[4][4] = {{1, 0, 0, 0}, {1, 0.5, 0, 0}, {1, 0.5, 0.25, 0}, {1, 1, 0.5, 0.25}};
  const double tau = m / 4.0, r = 0.25;  // dt / Delta
  const double unit[6] = {1.0, D, D * D, 1.0, D, D * D};
  for (int j = 0; j < 6; ++j) {
    double w = 0.0, rk = 1.0;
    for (int k = 0; k < 4; ++k, rk *= r) w += mult[l][k] * rk * poly_derivative(HERMITE5[j], k, tau);
    cf[j] = w * unit[j];
  }
}

mpw_status mpw_sur_stage_weights(int m, int l, double delta, double* w6) {
  if (m < 0 || m > 3 || l < 0 || l > 3 || !w6) return set_err(MPW_ERR_ARG, "stage weights: m, l in 0..3 and w6 non-null");
  stage_coefficients(m, l, delta, w6);
  return MPW_OK;
}

mpw_status mpw_step_surrogate(mpw_ctx* c, mpw_sur* s, double dt, int calls, double tol, int* accepted,
                              double* max_residual) {
  mpw_status st = check_ctx(c);
  if (st) return st;
  double sdt = 0.0, sh = 0.0;
  void* sstream = nullptr;
  if (!sur_geometry(s, &sdt, &sh, &sstream)) return set_err(MPW_ERR_ARG, "null surrogate handle");
  if (c->p.empty()) return set_err(MPW_ERR_STATE, "no global patch");
  if (calls < 0) return set_err(MPW_ERR_ARG, "calls must be >= 0");
  if (c->cfg.precision != 64) return set_err(MPW_ERR_ARG, "the surrogate path runs on binary64 contexts");
  PatchState& G = c->p[0];
  if (G.d.outer_bc != MPW_BC_PERIODIC) return set_err(MPW_ERR_ARG, "the surrogate needs a periodic global patch");
  for (int a = 0; a < 3; ++a)
    if (std::fabs(G.g.h[a] - sh) > 1e-12 * sh) return set_err(MPW_ERR_ARG, "global spacing differs from the surrogate's");
  if (std::fabs(dt - sdt) > 1e-12 * sdt) return set_err(MPW_ERR_ARG, "dt differs from the surrogate's");
  for (size_t q = 1; q < c->p.size(); ++q)
    if (c->p[q].sph() || c->p[q].d.motion == MPW_MOTION_ROTATING)
      return set_err(MPW_ERR_ARG, "the surrogate path takes translating Cartesian local patches only");
  if (use_device(c)) return MPW_ERR_CUDA;
  if ((st = apply_pending_inputs(c))) return st;
  const int n[3] = {G.d.n[0], G.d.n[1], G.d.n[2]};
  const long long P = (long long)n[0] * n[1] * n[2];
  const size_t need = (size_t)8 * P * sizeof(double) + 16 * 6 * sizeof(double) + 4 * sizeof(float);
  if (c->sur_bytes < need) {
    c->dfree(c->d_sur);
    c->sur_bytes = 0;
    if (!(c->d_sur = (double*)c->dalloc(need))) return set_err(MPW_ERR_CUDA, "device allocation failed");
    c->sur_bytes = need;
  }
  double* U = c->d_sur;  // psi0, Pi0, psi1, Pi1, then L psi0, L Pi0, L psi1, L Pi1
  double* coef = U + 8 * P;
  float* chk = (float*)(coef + 16 * 6);
  const cudaStream_t ss = (cudaStream_t)sstream;
  const double D = 4.0 * dt;
  double hc[16 * 6];
  for (int m = 0; m < 4; ++m)
    for (int l = 0; l < 4; ++l) stage_coefficients(m, l, D, hc + (4 * m + l) * 6);
  CUDA_TRY(cudaMemcpyAsync(coef, hc, sizeof(hc), cudaMemcpyHostToDevice, c->stream));
  int acc = 0;
  double rmax = 0.0;
  for (int call = 0; call < calls; ++call) {
    if ((st = step_prologue(c, dt))) return st;
    {
      // the state at t_n, its covered cells refilled from the local patches
      // (Local-to-Global, Sec. 2.4.2) as the method refills them at every
      // substage: local-patch data enters the global once per call
      if ((st = run_fill(c, FILL_BUF[0], c->t, NEXT_BUF[0], FILL_L2G))) return st;
      if ((st = fill_dead_cells(c))) return st;
      launch_pack(G.buf(BUF_U), G.g, U, U + P, 0, nullptr, false, c->stream);
      CUDA_TRY(cudaGetLastError());
    }
    if (ss != c->stream) CUDA_TRY(cudaStreamSynchronize(c->stream));
    if ((st = mpw_sur_predict(s, U, U + P, 1, n, U + 2 * P, U + 3 * P))) return st;
    if ((st = sur_check_after_predict(s, U, U + P, U + 2 * P, U + 3 * P, n, U + 4 * P, chk))) return st;
    float h2[2];
    CUDA_TRY(cudaMemcpyAsync(h2, chk, sizeof(h2), cudaMemcpyDeviceToHost, ss));
    CUDA_TRY(cudaStreamSynchronize(ss));
    const double r = h2[1] > 0.0f ? (double)h2[0] / h2[1] : (double)h2[0];
    rmax = std::isfinite(r) ? std::max(rmax, r) : INFINITY;
    if (!(r <= tol)) {
      // fall back: the method's own four steps from the same state
      if ((st = step_impl(c, dt, 4, false))) return st;
      continue;
    }
    ++acc;
    for (int m = 0; m < 4; ++m) {
      // flags of the step; no revival (its values would be overwritten before
      // any read, see run_flags)
      if (m > 0 && (st = step_prologue(c, dt, false))) return st;
      const double tn = c->t;
      // Global-to-Local reads the global only around each local patch: its
      // covered box of this step, widened by the interpolation window, the
      // ghost depth and the motion within a step (clipped to the patch)
      std::vector<Box> donors;
      const int margin = c->P / 2 + NG + 2;
      for (const Box& bx : c->boxes) {
        if (box_empty(bx)) continue;
        Box w{};
        for (int a = 0; a < 3; ++a) {
          w.lo[a] = std::max(bx.lo[a] - margin, 0);
          w.hi[a] = std::min(bx.hi[a] + margin, n[a] - 1);
        }
        donors.push_back(w);
      }
      // the global's four stage states of the step (the stage inputs the
      // method would form there, from the interpolant), laid out in its four
      // buffers at once: substages 0-2 in the buffers the fills read, the
      // last in ACC (the global's own RHS is skipped, so ACC is free), which
      // the last fill takes as the global's donor buffer
      static const int GBUF[4] = {BUF_U, BUF_YA, BUF_YB, BUF_ACC};
      double* gb[4];
      int* gs[4];
      for (int l = 0; l < 4; ++l) {
        gb[l] = G.buf(GBUF[l]);
        gs[l] = c->d_expo + GBUF[l] * 2;
      }
      CUDA_TRY(cudaMemsetAsync(c->d_expo, 0, 8 * sizeof(int), c->stream));  // live slots of the global's 4 buffers
      launch_hermite(gb, gs, G.g, U, coef + 4 * m * 6, donors.data(), (int)donors.size(), c->stream);
      CUDA_TRY(cudaGetLastError());
      for (int l = 0; l < 4; ++l) {
        const double tl = tn + RK_C[l] * dt;
        // only the local patches take an RHS + stage update
        if ((st = run_fill(c, FILL_BUF[l], tl, NEXT_BUF[l], FILL_G2L, GBUF[l]))) return st;
        if ((st = run_rhs(c, l, tl, dt, true))) return st;
      }
      c->t = tn + dt;
      c->stepped = true;
    }
    launch_unpack(G.buf(BUF_U), G.g, U + 2 * P, U + 3 * P, false, c->stream);
    CUDA_TRY(cudaGetLastError());
    G.u_expo_valid = false;
  }
  if (accepted) *accepted = acc;
  if (max_residual) *max_residual = rmax;
  return read_error_word(c);
}

mpw_status mpw_live_points(mpw_ctx* c, long long* count) {
  mpw_status st = check_ctx(c);
  if (st) return st;
  if (c->p.empty() || !count) return set_err(MPW_ERR_ARG, "no global patch or null pointer");
  long long n = 0;
  for (const auto& P : c->p) n += (long long)P.d.n[0] * P.d.n[1] * P.d.n[2];
  bool rot = false;
  for (size_t q = 1; q < c->p.size(); ++q) rot = rot || c->p[q].d.motion == MPW_MOTION_ROTATING || c->p[q].sph();
  if (rot) {
    // a rotated covered set is no box: count the live global cells
    if (use_device(c)) return MPW_ERR_CUDA;
    if ((st = apply_pending_inputs(c))) return st;
    if (!c->flags_valid && (st = run_flags(c, c->t))) return st;
    const PatchState& g = c->p[0];
    std::vector<uint8_t> fl((size_t)g.d.n[0] * g.d.n[1] * g.d.n[2]);
    CUDA_TRY(cudaMemcpyAsync(fl.data(), c->d_flags, fl.size(), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    n -= (long long)fl.size();
    for (uint8_t f : fl) n += ((f & 3) == FLAG_LIVE || (f & 3) == FLAG_REVIVED) ? 1 : 0;
    *count = n;
    return MPW_OK;
  }
  for (size_t q = 1; q < c->p.size(); ++q) {
    const Box b = c->flags_valid && q - 1 < c->boxes.size() ? c->boxes[q - 1] : covered_box(c->p[0], c->p[q], c->t);
    long long inner = 1;
    for (int a = 0; a < 3; ++a) inner *= std::max(b.hi[a] - b.lo[a] + 1 - 2 * c->buffer, 0);
    if (!box_empty(b)) n -= inner;
  }
  *count = n;
  return MPW_OK;
}

mpw_status mpw_profile_enable(mpw_ctx* c, int enable) {
  mpw_status st = check_ctx(c);
  if (st) return st;
  c->prof = enable != 0;
  return MPW_OK;
}

mpw_status mpw_profile_read(mpw_ctx* c, double* ms, long long* launches, int n) {
  mpw_status st = check_ctx(c);
  if (st) return st;
  if (n < 0 || n > MPW_KERNEL_FAMILIES) return set_err(MPW_ERR_ARG, "n must be in [0, %d]", MPW_KERNEL_FAMILIES);
  if (use_device(c)) return MPW_ERR_CUDA;
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  for (int f = 0; f < MPW_KERNEL_FAMILIES; ++f) {
    double total = 0.0;
    for (size_t i = 0; i < c->ev_used[f]; ++i) {
      float m = 0.0f;
      CUDA_TRY(cudaEventElapsedTime(&m, c->ev[f][2 * i], c->ev[f][2 * i + 1]));
      total += m;
    }
    if (f < n) {
      if (ms) ms[f] = total;
      if (launches) launches[f] = c->launches[f];
    }
    c->ev_used[f] = 0;
    c->launches[f] = 0;
  }
  return MPW_OK;
}


// ============================================================================ batches
}  // extern "C"

struct mpw_batch {
  std::vector<mpw_ctx*> ctx;
  cudaStream_t stream = nullptr;
  int P = 6;
  bool f32 = false, fixed = true;
  // argument tables of the 8 launches of one step (4 fills, 4 RHS): device
  // copies, reused every step in stream order, and two pinned host halves,
  // alternated by step, each released by the event after its last copy
  size_t region = 0;            // bytes per launch region
  char* d_args = nullptr;
  char* h_args[2] = {nullptr, nullptr};
  cudaEvent_t copied[2] = {nullptr, nullptr};
  long long steps_done = 0;
  // chunk-depth tuning of the RHS launches
  std::vector<int> cand;
  std::vector<cudaEvent_t> tev;  // start/stop per candidate
  int zc = 0;                    // chosen chunk depth (0 until tuned)
  double zc_ms = 0.0;            // its measured RHS time per step
  long long launches = 0;
  // CUDA graphs of one step (one per pinned half).  The captured copies pick
  // up each step's arguments from the pinned half at replay, so a graph
  // serves every step whose launches fit its grids: a static batch has the
  // same grids every step; a moving one is captured with grids padded to a
  // capacity (spare blocks exit at once) and captured again only when a
  // grid outgrows it.  Launches whose arguments travel by value (mirrors and
  // shells of moving patches) rule the graph out.
  cudaStream_t cap = nullptr;    // capture stream
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  int gtot[2][9] = {};           // the grids each graph launches (8: batched flags)
  bool gflags[2] = {false, false};  // whether the graph holds the batched flags launches
  long long captures = 0;
  bool graphs = true;
  long long graph_steps = 0;
};

namespace {
const int ZC_CANDIDATES[] = {8, 16, 32, 64};
}

extern "C" {

mpw_status mpw_batch_create(mpw_ctx* const* ctxs, int n, mpw_batch** out) {
  if (!ctxs || !out || n < 1) return set_err(MPW_ERR_ARG, "need at least one context");
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (mpw_status st = check_ctx(ctxs[i])) return st;
    const mpw_ctx* c = ctxs[i];
    if (c->p.empty()) return set_err(MPW_ERR_STATE, "context %d has no global patch", i);
    if (c->cfg.device != ctxs[0]->cfg.device || c->stream != ctxs[0]->stream)
      return set_err(MPW_ERR_ARG, "batched contexts must share the device and the stream");
    if (c->cfg.precision != ctxs[0]->cfg.precision || c->P != ctxs[0]->P ||
        (c->cfg.arith != 1) != (ctxs[0]->cfg.arith != 1))
      return set_err(MPW_ERR_ARG, "batched contexts must share precision, interp_points and arith");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == c) return set_err(MPW_ERR_ARG, "a context appears twice in the batch");
  }
  mpw_batch* b = new mpw_batch();
  b->ctx.assign(ctxs, ctxs + n);
  b->stream = ctxs[0]->stream;
  b->P = ctxs[0]->P;
  b->f32 = ctxs[0]->cfg.precision == 32;
  b->fixed = ctxs[0]->cfg.arith != 1;
  const size_t table = std::max(sizeof(FillArgs), sizeof(RhsArgs)) * (size_t)n;
  b->region = (table + sizeof(int) * (size_t)(n + 1) + 255) / 256 * 256;
  if (use_device(ctxs[0])) {
    delete b;
    return MPW_ERR_CUDA;
  }
  // regions 0-7: the fill and RHS tables of the 4 substages; 8: the flags
  static_assert(sizeof(FlagArgs) <= sizeof(FillArgs), "the flags table must fit a region");
  bool ok = cudaMalloc(&b->d_args, 9 * b->region) == cudaSuccess;
  for (int h = 0; h < 2 && ok; ++h)
    ok = cudaMallocHost(&b->h_args[h], 9 * b->region) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->copied[h], cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess;
  for (int z : ZC_CANDIDATES) b->cand.push_back(z);
  b->tev.resize(2 * b->cand.size());
  for (auto& e : b->tev) ok = ok && cudaEventCreate(&e) == cudaSuccess;
  if (!ok) {
    mpw_batch_destroy(b);
    return set_err(MPW_ERR_CUDA, "batch allocation failed");
  }
  *out = b;
  return MPW_OK;
}

void mpw_batch_destroy(mpw_batch* b) {
  if (!b) return;
  if (b->stream || !b->ctx.empty()) cudaStreamSynchronize(b->stream);
  cudaFree(b->d_args);
  for (int h = 0; h < 2; ++h) {
    if (b->h_args[h]) cudaFreeHost(b->h_args[h]);
    if (b->copied[h]) cudaEventDestroy(b->copied[h]);
  }
  for (auto& e : b->tev)
    if (e) cudaEventDestroy(e);
  for (int h = 0; h < 2; ++h)
    if (b->gexec[h]) cudaGraphExecDestroy(b->gexec[h]);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

mpw_status mpw_batch_step(mpw_batch* b, const double* dt, int nsteps) {
  if (!b || !dt) return set_err(MPW_ERR_ARG, "null argument");
  if (nsteps < 0) return set_err(MPW_ERR_ARG, "nsteps must be >= 0");
  const int n = (int)b->ctx.size();
  for (mpw_ctx* c : b->ctx)
    if (mpw_status st = check_ctx(c)) return st;
  if (use_device(b->ctx[0])) return MPW_ERR_CUDA;
  mpw_status st;
  for (mpw_ctx* c : b->ctx)
    if ((st = apply_pending_inputs(c))) return st;
  const size_t nc = b->cand.size();
  for (int s = 0; s < nsteps; ++s) {
    // chunk depth: the first steps try every candidate, timing the RHS
    // launches; results do not depend on it (each point's arithmetic is the
    // same whatever chunk its CTA marches)
    const long long k = b->steps_done;
    const bool trial = b->zc == 0 && k < (long long)nc;
    const int zc = b->zc ? b->zc : (trial ? b->cand[k] : 0);
    double tn[64];
    std::vector<double> tnv;
    double* tnp = n <= 64 ? tn : (tnv.resize(n), tnv.data());
    const int h = (int)(k & 1);
    CUDA_TRY(cudaEventSynchronize(b->copied[h]));  // the pinned half from two steps ago has been copied
    // cover flags: when every patch of every instance is a translating
    // Cartesian one and the flags and (binary64) u's exponent slots are in
    // place, the
    // moving instances' flags go into the step's launches as one batched
    // flags launch and one revival launch (argument table in region 8);
    // otherwise each instance takes its own, here
    bool fl_batch = true;
    for (mpw_ctx* c : b->ctx) {
      fl_batch = fl_batch && c->flags_valid;
      for (const auto& P : c->p)
        fl_batch = fl_batch && !P.sph() && P.d.motion != MPW_MOTION_ROTATING &&
                   (c->cfg.precision == 32 || P.u_expo_valid);
    }
    // host cover-flag state of the contexts whose flags this step prepares,
    // put back if the step fails before its launches are queued: the device
    // flags are then still those of the last completed step, and the next
    // flag computation must start from that step's covered boxes
    struct FlagsUndo {
      std::vector<mpw_ctx*> ctx;
      std::vector<std::vector<Box>> boxes;
      std::vector<char> valid, glist;
      ~FlagsUndo() {
        for (size_t k = 0; k < ctx.size(); ++k) {
          ctx[k]->boxes = boxes[k];
          ctx[k]->flags_valid = valid[k] != 0;
          ctx[k]->glist_valid = glist[k] != 0;
        }
      }
    } undo;
    int nflag = 0;
    {
      char* freg = b->h_args[h] + (size_t)8 * b->region;
      FlagArgs* fa = reinterpret_cast<FlagArgs*>(freg);
      int* fblk0 = reinterpret_cast<int*>(freg + sizeof(FlagArgs) * n);
      long long ftotal = 0;
      for (int i = 0; i < n; ++i) {
        mpw_ctx* c = b->ctx[i];
        tnp[i] = c->t;
        fblk0[i] = (int)ftotal;
        if (!fl_batch) {
          if ((st = step_prologue(c, dt[i]))) return st;
          continue;
        }
        if ((st = validate_step(c, dt[i], tnp[i]))) return st;
        bool launch = false;
        if (any_moving(c)) {
          undo.ctx.push_back(c);
          undo.boxes.push_back(c->boxes);
          undo.valid.push_back(c->flags_valid ? 1 : 0);
          undo.glist.push_back(c->glist_valid ? 1 : 0);
          if ((st = prep_flags(c, tnp[i], true, fa[i], launch))) return st;
        }
        if (launch) {
          ftotal += flags_blocks(fa[i]);
          c->flags_valid = true;
          c->glist_valid = false;
          ++nflag;
        } else {
          fa[i] = FlagArgs{};  // no flags this step: the clear and the revival skip it
        }
      }
      fblk0[n] = (int)ftotal;
      if (ftotal > INT32_MAX / 2) return set_err(MPW_ERR_ARG, "batched flags grid too large");
    }
    const bool fl_on = fl_batch && nflag > 0;
    std::vector<MirrorArgs> mirs(4 * (size_t)n);    // fixed-point mirrors of each instance's fills
    // arguments of the 8 launches of this step into pinned half h
    int totals[9];
    totals[8] = fl_on ? reinterpret_cast<int*>(b->h_args[h] + (size_t)8 * b->region + sizeof(FlagArgs) * n)[n] : 0;
    for (int l = 0; l < 4; ++l) {
      for (int pass = 0; pass < 2; ++pass) {  // 0: ghost fill, 1: RHS + stage
        const int r = 2 * l + pass;
        char* hreg = b->h_args[h] + (size_t)r * b->region;
        const size_t esz = pass ? sizeof(RhsArgs) : sizeof(FillArgs);
        int* blk0 = reinterpret_cast<int*>(hreg + esz * n);
        int total = 0;
        for (int i = 0; i < n; ++i) {
          mpw_ctx* c = b->ctx[i];
          const double tl = tnp[i] + RK_C[l] * dt[i];
          blk0[i] = total;
          if (pass == 0) {
            FillArgs* fa = reinterpret_cast<FillArgs*>(hreg) + i;
            if ((st = prep_fill(c, FILL_BUF[l], tl, NEXT_BUF[l], *fa, &mirs[l * n + i]))) return st;
            total += fa->total_blocks;
          } else {
            RhsArgs* ra = reinterpret_cast<RhsArgs*>(hreg) + i;
            total += prep_rhs(c, l, tl, dt[i], *ra, zc);
          }
        }
        blk0[n] = total;
        totals[r] = total;
      }
    }
    bool rot = false;  // some patch rotates: the RHS kernels with a position-dependent w
    for (mpw_ctx* c : b->ctx)
      for (const auto& P : c->p) rot = rot || P.d.motion == MPW_MOTION_ROTATING;
    // spherical shells: after each batched RHS launch, one launch over the
    // shells of all instances (more launches when they exceed MAX_SHELLS)
    std::vector<ShellArgs> sargs;
    std::vector<long long> sblocks;
    std::vector<int> sfirst(5, 0);
    for (int l = 0; l < 4; ++l) {
      sfirst[l] = (int)sargs.size();
      sargs.emplace_back();
      sblocks.push_back(0);
      for (int i = 0; i < n; ++i) {
        long long nb = prep_rhs_shell(b->ctx[i], l, tnp[i] + RK_C[l] * dt[i], dt[i], sargs.back(), sblocks.back());
        if (nb < 0) {  // full: start another launch
          sargs.emplace_back();
          sblocks.push_back(0);
          nb = prep_rhs_shell(b->ctx[i], l, tnp[i] + RK_C[l] * dt[i], dt[i], sargs.back(), 0);
          if (nb < 0) return set_err(MPW_ERR_ARG, "an instance holds more than %d shells", MAX_SHELLS);
        }
        sblocks.back() = nb;
      }
    }
    sfirst[4] = (int)sargs.size();
    bool moving = false;
    for (mpw_ctx* c : b->ctx) moving = moving || any_moving(c);
    bool by_value = false;  // a launch of this step takes its arguments by value
    for (long long sb : sblocks) by_value = by_value || sb > 0;
    for (const MirrorArgs& ma : mirs) by_value = by_value || ma.nr > 0;
    const bool use_graph = b->graphs && !trial && !(moving && by_value);
    // the grids: the block totals, or while replaying a moving batch the
    // graph's padded capacities (a new capture when a total outgrows them)
    int grid[9];
    std::memcpy(grid, totals, sizeof(grid));
    bool recapture = false;
    if (use_graph) {
      if (!b->gexec[h] || b->gflags[h] != fl_on) {
        recapture = true;
      } else if (moving) {
        for (int r = 0; r < 9; ++r) recapture = recapture || totals[r] > b->gtot[h][r];
      } else {
        recapture = std::memcmp(b->gtot[h], totals, sizeof(totals)) != 0;
      }
      if (moving)
        for (int r = 0; r < 9; ++r)
          grid[r] = recapture ? totals[r] + totals[r] / 16 + 64 : std::max(totals[r], b->gtot[h][r]);
    }
    // copies and launches of the step, on stream sm
    auto enqueue = [&](cudaStream_t sm) -> cudaError_t {
      if (fl_on) {
        const char* hreg = b->h_args[h] + (size_t)8 * b->region;
        char* dreg = b->d_args + (size_t)8 * b->region;
        cudaError_t e = cudaMemcpyAsync(dreg, hreg, sizeof(FlagArgs) * n + sizeof(int) * (n + 1),
                                        cudaMemcpyHostToDevice, sm);
        if (e != cudaSuccess) return e;
        launch_flags_batch(reinterpret_cast<const FlagArgs*>(dreg),
                           reinterpret_cast<const int*>(dreg + sizeof(FlagArgs) * n), n, grid[8], b->P, b->f32, sm);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
      }
      for (int r = 0; r < 8; ++r) {
        const int l = r / 2, pass = r % 2;
        char* hreg = b->h_args[h] + (size_t)r * b->region;
        char* dreg = b->d_args + (size_t)r * b->region;
        const size_t esz = pass ? sizeof(RhsArgs) : sizeof(FillArgs);
        cudaError_t e = cudaMemcpyAsync(dreg, hreg, esz * n + sizeof(int) * (n + 1), cudaMemcpyHostToDevice, sm);
        if (e != cudaSuccess) return e;
        const int* d_blk0 = reinterpret_cast<const int*>(dreg + esz * n);
        if (pass == 0) {
          for (int i = 0; i < n; ++i) launch_mirror(mirs[l * n + i], sm);
          launch_fill_batch(reinterpret_cast<const FillArgs*>(dreg), d_blk0, n, grid[r], b->P, b->f32, sm);
        } else {
          if (trial && l == 0) cudaEventRecord(b->tev[2 * k], sm);
          if (b->f32)
            launch_rhs32_batch(reinterpret_cast<const RhsArgs*>(dreg), d_blk0, n, grid[r], rot, sm);
          else
            launch_rhs_batch(reinterpret_cast<const RhsArgs*>(dreg), d_blk0, n, grid[r], b->fixed, rot, sm);
          for (int k2 = sfirst[l]; k2 < sfirst[l + 1]; ++k2)
            if (sblocks[k2] > 0) launch_rhs_shell(sargs[k2], sblocks[k2], sm);
          if (trial && l == 3) cudaEventRecord(b->tev[2 * k + 1], sm);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
      }
      return cudaSuccess;
    };
    bool replayed = false;
    if (use_graph) {
      if (recapture) {
        if (b->gexec[h]) cudaGraphExecDestroy(b->gexec[h]);
        b->gexec[h] = nullptr;
        cudaGraph_t graph = nullptr;
        bool ok = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        const cudaError_t eq = ok ? enqueue(b->cap) : cudaErrorUnknown;
        ok = cudaStreamEndCapture(b->cap, &graph) == cudaSuccess && ok && eq == cudaSuccess && graph;
        ok = ok && cudaGraphInstantiate(&b->gexec[h], graph, 0) == cudaSuccess;
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        if (ok) {
          std::memcpy(b->gtot[h], grid, sizeof(grid));
          b->gflags[h] = fl_on;
          ++b->captures;
        } else {
          b->gexec[h] = nullptr;
          b->graphs = false;  // this configuration does not capture: launch directly from now on
        }
      }
      if (b->gexec[h]) {
        CUDA_TRY(cudaGraphLaunch(b->gexec[h], b->stream));
        ++b->graph_steps;
        replayed = true;
      }
    }
    if (!replayed) CUDA_TRY(enqueue(b->stream));
    undo.ctx.clear();  // queued: the prepared flags are the contexts' own now
    b->launches += 8 + (fl_on ? (grid[8] > 0 ? 3 : 2) : 0);
    for (long long sb : sblocks) b->launches += sb > 0 ? 1 : 0;
    for (const MirrorArgs& ma : mirs) b->launches += ma.nr > 0 ? 1 : 0;
    CUDA_TRY(cudaEventRecord(b->copied[h], b->stream));
    for (int i = 0; i < n; ++i) {
      b->ctx[i]->t = tnp[i] + dt[i];
      b->ctx[i]->stepped = true;
    }
    ++b->steps_done;
    if (trial && b->steps_done == (long long)nc) {
      // every candidate ran once (the fills in between are the same for all)
      double best = 0.0;
      for (size_t c = 0; c < nc; ++c) {
        float ms = 0.0f;
        CUDA_TRY(cudaEventSynchronize(b->tev[2 * c + 1]));
        CUDA_TRY(cudaEventElapsedTime(&ms, b->tev[2 * c], b->tev[2 * c + 1]));
        if (b->zc == 0 || ms < best) {
          best = ms;
          b->zc = b->cand[c];
        }
      }
      b->zc_ms = best;
    }
  }
  for (mpw_ctx* c : b->ctx)
    if ((st = read_error_word(c))) return st;
  return MPW_OK;
}

mpw_status mpw_batch_tuning(const mpw_batch* b, int* zc, double* rhs_ms, long long* launches,
                            long long* graph_steps) {
  if (!b) return set_err(MPW_ERR_ARG, "null batch");
  if (zc) *zc = b->zc;
  if (rhs_ms) *rhs_ms = b->zc_ms;
  if (launches) *launches = b->launches;
  if (graph_steps) *graph_steps = b->graph_steps;
  return MPW_OK;
}

}  // extern "C"
