// mpw_internal.cuh -- device data layout and kernel interfaces of libmpw
// (the layout and the RHS tables live in mpw_rhs_args.cuh).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/mpw.h"
#include "mpw_rhs_args.cuh"

struct mpw_sur;

namespace mpw {

// ---------------------------------------------------------------- fill
// One interpolation target set: the hollow box shell (walls NG thick) of a
// target patch, filled from a donor patch.  The shell is cut into six slabs
// (z-, z+, y-, y+, x-, x+), each tiled by boxes of td targets.
enum { SEG_SHELL = 0, SEG_AFFINE = 1, SEG_MASKED = 2, SEG_LIST = 3, SEG_SPH_GHOSTS = 4 };

struct InterpSeg {
  int kind;            // SEG_SHELL: hollow box under translation (separable passes);
                       // SEG_AFFINE: hollow box under a rotating map (direct sums);
                       // SEG_MASKED: the global cells of flag `want` inside `box`;
                       // SEG_LIST: the global cells listed by the cover-flag kernel;
                       // SEG_SPH_GHOSTS: every ghost node of a spherical shell (azimuthal
                       // ghosts copy their periodic image, the others interpolate the
                       // global patch through X_B = M X'(r, theta, phi) + shift)
  double M[9];         // SEG_AFFINE / SEG_MASKED / SEG_LIST: donor position = M target position + shift
  double sidx[3][4];   // the same as donor index coordinates of target cell (i, j, k):
                       // s_a = sidx[a][0] i + sidx[a][1] j + sidx[a][2] k + sidx[a][3]
  const long long* list;  // SEG_LIST: linear global cell indices, *count of them
  const int* count;
  int list_blocks;     // SEG_LIST: CTAs striding over the list
  int sph;             // SEG_MASKED / SEG_LIST: the donor is a spherical shell (M, shift map
                       // the target to the donor's Cartesian frame)
  const int2* mir;     // fixed-point mirror of the donor over mbox (donor indices, both fields,
  Box mbox;            // x fastest), or null: the per-point sums gather and convert the donors
  Box box;             // SEG_MASKED: target cells to test (global indices)
  const uint8_t* flags;
  int want;            // flag byte of the cells to fill (state | owner << 2)
  double* T;           // target buffer (psi; Pi at +vol)
  Geom gt;
  int tpatch;          // target patch id (exponent slots)
  int dpatch;          // donor patch id (exponent slots)
  const double* D;     // donor buffer (psi; Pi at +vol)
  Geom gd;
  double shift[3];     // X0_target - X0_donor at the substage time (translation), or the
                       // affine offset
  int sb[6][3];        // slab origin (target indices)
  int se[6][3];        // slab extent
  int td[6][3];        // tile extent
  int tn[6][2];        // tiles along x and y of each slab (z follows)
  int slab_block0[6];  // first CTA of each slab, relative to block0
  int block0;          // first CTA of the segment
};

constexpr int MAX_SEGS = 2 * (MAX_PATCHES - 1);

struct FillArgs {
  double* Yg;          // global stage buffer
  Geom gg;
  int outer_bc;        // 0 analytic, 1 periodic
  int akind, acount;
  const double* aparams;
  const float4* ascreen;  // FP32 screening data of Gaussian pulses (or null)
  const double* apre;     // 1/width^2 of every Gaussian pulse (or null)
  const double* shell_src;  // global buffer whose outer shell holds the closed form at t (or null)
  double t;
  long long outer_count;
  int outer_blocks;
  int nseg;
  InterpSeg seg[MAX_SEGS];
  int P;
  int* err;
  int* expo;
  int y_buf;           // buffer being filled (its exponent slots receive the ghost values)
  int reset_buf;       // buffer whose exponent slots are cleared (the next stage's output), or -1
  int reset_first;     // first patch whose slots that clears (0: every patch)
  int gdonor_use;      // 1: the global patch donates from buffer gdonor_buf, not y_buf
  int gdonor_buf;
  int np;
  int total_blocks;
  int fixed;           // 1: separable contractions in int64 fixed point, 0: native FP64
  int f32;             // field buffers hold binary32 (FP32 arithmetic; fixed is ignored)
};

// ---------------------------------------------------------------- fixed-point mirrors
// Before a ghost fill whose per-point sums read many donors (spherical
// shells), the donor cells they can reach are converted once to the split
// fixed-point form of the fill (a = 64 q on the scale of the donor's live
// exponent slot for the buffer being filled).
struct MirrorRegion {
  const double* src;   // donor buffer (psi; Pi at +vol)
  Geom g;
  Box box;             // donor indices, inclusive
  int2* dst;           // 2 x volume(box) entries, field-major, x fastest
  int patch;           // donor patch id (exponent slots)
  long long block0;
};
constexpr int MAX_MIRRORS = 2 * MAX_PATCHES;  // per shell: its global donor box and its own box
struct MirrorArgs {
  MirrorRegion r[MAX_MIRRORS];
  int nr;
  long long blocks;
  const int* expo;
  int y_buf;
};
void launch_mirror(const MirrorArgs& a, void* stream);

// ---------------------------------------------------------------- shell RHS
// Fused RHS + RK4 stage on spherical shells (plain FP64, one thread per point).
struct ShellPatch {
  const double* Y;     // stencil input (psi; Pi at +vol), ghosts filled
  const double* U;
  double* ACC;
  double* OUT;
  Geom g;              // numeric (r, theta, phi)
  // per-axis tables of the nodes: r, 1/r (n_r each), sin, cos, 1/sin of theta
  // (n_theta each), sin, cos of phi (n_phi each)
  const double* tab;
  double R[9];         // frame velocity w(X') = w0 + W X' (patch frame components)
  double w0[3], W[9];
  int moving;
  int patch;           // patch id (exponent slots)
  int* expo;           // the exponent slots of the shell's context
  double alpha, beta;  // stage coefficients (dt of the shell's context)
  double id1[3], id2[3];  // 1 / (12 h_a), 1 / (12 h_a^2) per numeric axis
  double iko[3];       // eps / (64 L_a) with L = h_r, h_theta, h_phi (times 1/r, 1/(r sin theta) per point)
  long long block0;
};

constexpr int MAX_SHELLS = 64;  // shells of one launch (a batch may span several contexts)

struct ShellArgs {
  ShellPatch p[MAX_SHELLS];
  int np;
  int stage;
  int in_buf, out_buf;
};

void launch_rhs_shell(const ShellArgs& a, long long blocks, void* stream);

// ---------------------------------------------------------------- flags
struct FlagArgs {
  uint8_t* flags;
  int n[3];
  int nloc;
  Box box[MAX_PATCHES];
  int buffer;
  int old_valid;
  int skip_revive;     // flags only: the revived cells keep what u holds (see run_flags)
  double* Ug;          // global u (psi; Pi at +vol)
  Geom gg;
  const double* Uloc[MAX_PATCHES];
  Geom gl[MAX_PATCHES];
  double X0[MAX_PATCHES][3];
  // rotating patches: box[q] bounds the covered cells, whose mask the cover
  // kernel writes to cov (cov_off[q] onwards, box-local x fastest)
  int rot[MAX_PATCHES];
  double R[MAX_PATCHES][9];
  double lhi[MAX_PATCHES][3];  // upper corner of the live box (the descriptor's hi)
  // binary32 screen of the coverage test: X'_a ~ scr[q][a][3] + sum_b scr[q][a][b] idx_b
  float scr[MAX_PATCHES][3][4];
  float scrm[MAX_PATCHES];     // decision margin of the screen (above 25 x its rounding error)
  uint8_t* cov;
  long long cov_off[MAX_PATCHES + 1];
  // spherical shells: cov holds, per cell of the bounding box, the L-infinity
  // distance to the nearest uncovered cell capped at DIST_CAP (0: uncovered),
  // from a separable transform over two more regions of cov_off[nloc] bytes
  int sph[MAX_PATCHES];
  double cth[MAX_PATCHES][2];  // cos(theta_lo), cos(theta_hi)
  // effective ghosts of each rotating patch, listed for Local-to-Global:
  // glist[cov_off[q] ...], gcount[q] entries (null: no lists)
  long long* glist;
  int* gcount;
  int P;
  int* err;
  int* expo;
  // cells to visit: disjoint boxes (global indices) covering every cell whose
  // flag can change (the old and new covered boxes); nreg = 0 means all cells
  int nreg;
  Box reg[MAX_PATCHES];
  long long reg_begin[MAX_PATCHES + 1];
  // revived cells, interpolated by a second kernel with full warps: entry =
  // global cell index | (local patch << 40); cells past rev_cap are
  // interpolated in place by the flags kernel
  long long* rev_list;
  int* rev_count;
  int rev_cap;
  int f32;             // field buffers hold binary32
};
constexpr int REVIVE_CAP = 1 << 16;  // queue entries (one box crossing revives a few thousand cells)
constexpr int DIST_CAP = 9;          // distances above buffer + NG (<= 8) read as "dead" 

// Record the thread-local message returned by mpw_last_error().
void set_last_error(const char* msg);

// learned surrogate: the four RK4 stage states of one step from the quintic
// Hermite interpolant in time of the global state between two calls, written
// into the cells of `boxes` of four padded buffers, their exponent slots
// raised (u: psi0, Pi0, psi1, Pi1, L psi0, L Pi0, L psi1, L Pi1, dense;
// coef_dev: 4 x 6 device doubles); and the step and spacing a surrogate was
// made for
void launch_hermite(double* const buf[4], int* const slot2[4], const Geom& g, const double* u, const double* coef_dev,
                    const Box* boxes, int nbox, void* stream);
bool sur_geometry(const mpw_sur* s, double* dt, double* h, void** stream);
// mpw_sur_check for batch 1 right after mpw_sur_predict(s, psi0, pi0, ...):
// L psi0 and L Pi0 are copied from the prediction's features instead of
// being computed again (the same kernel, so the same values)
mpw_status sur_check_after_predict(mpw_sur* s, const double* psi0, const double* pi0, const double* psi1,
                                   const double* pi1, const int n[3], double* lap, float* out);

// ---------------------------------------------------------------- tensor maps
// Encode the TMA maps of the RHS kernel for one field buffer (psi at base, Pi
// at base + vol) of geometry g: box (RHS_TX + 8) x (RHS_TY + 6) ("tile") or
// RHS_TX x RHS_TY ("point"), elements binary64 or (f32) binary32.  Returns
// false if the driver rejects the map.
bool encode_rhs_map(CUtensorMap* map, const void* base, const Geom& g, bool tile, bool f32 = false);

// ---------------------------------------------------------------- host entry points of the kernels
// rot: some patch of the launch rotates (selects the kernels with a
// position-dependent frame velocity)
void launch_rhs(const RhsArgs& a, int blocks, bool fixed, bool rot, void* stream);
void launch_rhs32(const RhsArgs& a, int blocks, bool rot, void* stream);  // binary32 storage and arithmetic
// Batched launches over independent instances: d_args[i] (device memory)
// describes instance i, whose blocks are [d_blk0[i], d_blk0[i + 1]).
void launch_rhs_batch(const RhsArgs* d_args, const int* d_blk0, int ninst, int blocks, bool fixed, bool rot,
                      void* stream);
void launch_rhs32_batch(const RhsArgs* d_args, const int* d_blk0, int ninst, int blocks, bool rot, void* stream);
void launch_fill_batch(const FillArgs* d_args, const int* d_blk0, int ninst, int blocks, int P, bool f32,
                       void* stream);
void launch_expo_scan(const double* buf, const Geom& g, const uint8_t* flags, int* slot2, void* stream);
void launch_fill(const FillArgs& a, void* stream);
int fill_max_thin_donors();
int fill_cap_r1();
int fill_cap_r2();
int fill_max_tile();
int fill_threads();
// Batched cover flags of translating instances: one clear of the revival
// counters, one flags launch over `blocks` (prefix table d_blk0, padded grids
// allowed) and one revival launch, for `ninst` argument sets in device memory.
void launch_flags_batch(const FlagArgs* d_args, const int* d_blk0, int ninst, int blocks, int P, bool f32,
                        void* stream);
long long flags_blocks(const FlagArgs& a);   // blocks of a's flags launch
int launch_flags(const FlagArgs& a, void* stream);  // returns the number of kernels launched
void launch_fill_dead(const FlagArgs& a, void* stream);  // binary64 buffers only
// buf: a field buffer of binary64, or of binary32 when f32; the dense arrays
// d0, d1 are binary64 in every case.
struct Affine {
  double R[9];  // row-major
  double X0[3];
};
// X_B = R X' + X0 for every interior point (the patch map at t).
// sph: g's numeric coordinates are (r, theta, phi) of a spherical shell.
void launch_analytic(void* buf, const Geom& g, const Affine& map, int akind, int acount, const double* aparams,
                     const float4* screen, const double* apre, double t, bool f32, void* stream, bool sph = false);
void launch_pack(const void* buf, const Geom& g, double* d0, double* d1, int padded, const uint8_t* flags, bool f32,
                 void* stream);
void launch_unpack(void* buf, const Geom& g, const double* d0, const double* d1, bool f32, void* stream);
// unpack into a binary64 u, raising its live exponent slots (slot2, cleared
// first by the caller) over the cells flags count as live (flags may be null)
void launch_unpack_scan(double* buf, const Geom& g, const double* d0, const double* d1, const uint8_t* flags,
                        int* slot2, void* stream);

}  // namespace mpw
