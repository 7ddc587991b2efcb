/*
 * mpw.h -- C ABI of libmpw, a single-GPU (sm_103a) implementation of the
 * data-parallel hot path of the multipatch scalar-wave method of
 * "PatchworkWave" (arXiv:2002.00088): 4th-order method-of-lines evolution of
 * the fields psi and Pi = d(psi)/dt on one global patch plus moving local
 * patches, with ghost zones refilled at every RK4 substage by tensor-product
 * Lagrange interpolation through the time-dependent patch maps and a buffer of
 * live global cells under each local patch edge (one-way data flow).
 *
 * Conventions shared by every entry point
 *  - Every call returns mpw_status; MPW_OK is 0.  On error a message is kept
 *    per thread and returned by mpw_last_error().
 *  - Floating point is IEEE binary64 throughout (psi, Pi, time, maps).
 *  - Field arrays exchanged with the library are dense interior boxes
 *    [k][j][i], i fastest, n[0]*n[1]*n[2] doubles.  A pointer flagged
 *    on_device = 1 is a CUDA device pointer on the context's device; 0 means
 *    host memory (pinned or pageable).  Page-locked host arrays that are
 *    mapped into the device address space are read or written in place by
 *    the library's kernels; pageable arrays go through a device staging
 *    buffer.  Either way a host-pointer call returns once the host array may
 *    be reused (set) or holds the result (get).  The library never keeps or
 *    frees a caller pointer.
 *  - Patch geometry: patch j has numeric coordinates X'_j; the live box is
 *    [lo, hi] per axis holding n cells of width h = (hi - lo)/n, nodes
 *    cell-centred at lo + (i + 1/2) h.  The background Cartesian frame of
 *    Sec. 2.4.1 is X_B = X'_j + X0_j(t) (rigid translation; the global patch,
 *    id 0, is the background frame itself).  Every patch carries NG = 3
 *    ghost cells per side.
 *  - All work is enqueued on the stream given in mpw_config (NULL = the legacy
 *    default stream).  mpw_step(), mpw_get_fields() and mpw_get_flags()
 *    synchronise that stream before returning.
 */
#ifndef MPW_H
#define MPW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpw_ctx mpw_ctx;

typedef enum {
  MPW_OK = 0,
  MPW_ERR_ARG = 1,            /* invalid argument or configuration */
  MPW_ERR_OVERLAP = 2,        /* local patches closer than the separation rule */
  MPW_ERR_CFL = 3,            /* dt beyond the RK4 stability estimate */
  MPW_ERR_TRAVERSAL = 4,      /* a patch would cross more than one global cell in a step */
  MPW_ERR_OUTSIDE = 5,        /* a local patch (with ghosts and stencils) leaves the global interior */
  MPW_ERR_GHOST_UNFILLED = 6, /* a ghost point could not be interpolated (Sec. 2.4.1 "skip") */
                              /* 7 is not used */
  MPW_ERR_TIMEOUT = 8,        /* a bounded device wait (the RHS kernels' TMA pipeline) ran
                                 out: the CTA drained its own copies and stopped early, so the
                                 step's result is incomplete; the context stays usable */
  MPW_ERR_CUDA = 9,           /* a CUDA runtime call failed */
  MPW_ERR_STATE = 10          /* call not valid in the current state */
} mpw_status;

enum { MPW_PATCH_GLOBAL = 0, MPW_PATCH_LOCAL = 1 };
enum { MPW_TOPOLOGY_CARTESIAN = 0, MPW_TOPOLOGY_SPHERICAL = 1 };
enum { MPW_BC_ANALYTIC = 0, MPW_BC_PERIODIC = 1, MPW_BC_INTERPATCH = 2 };
enum { MPW_MOTION_STATIC = 0, MPW_MOTION_LINEAR = 1, MPW_MOTION_CIRCULAR = 2, MPW_MOTION_ROTATING = 3 };
enum {
  MPW_ANALYTIC_GAUSS_SUM = 0,
  MPW_ANALYTIC_PLANE_SUM = 1,
  MPW_ANALYTIC_HARMONIC_POLY = 2,
  MPW_ANALYTIC_PLANE_GAUSS = 3
};
/* Cover-flag byte of a global interior cell: state | (owning local patch id << 2). */
enum { MPW_FLAG_LIVE = 0, MPW_FLAG_GHOST = 1, MPW_FLAG_DEAD = 2, MPW_FLAG_REVIVED = 3 };

/* Device allocator hook.  alloc returns device memory of at least `bytes`
 * bytes (256-byte aligned) or NULL; free releases it.  NULL hooks mean
 * cudaMalloc / cudaFree. */
typedef void* (*mpw_alloc_fn)(size_t bytes, void* user);
typedef void (*mpw_free_fn)(void* ptr, void* user);

typedef struct {
  int precision;      /* 64: fields stored in IEEE binary64 (the paper's precision);
                         32: fields stored in binary32 and the stencil, stage and
                         interpolation arithmetic done in binary32, with the maps, the
                         Lagrange weights (rounded once), the closed forms and time in
                         binary64.  Field arrays exchanged through the ABI stay binary64
                         either way (converted on the device). */
  int ghost;          /* NG, must be 3 (the reach of the KO stencil, Sec. 2.4.2) */
  int interp_points;  /* Lagrange window P: 6 (the paper's i_c-2..i_c+3) or 5 (i_c-2..i_c+2) */
  double ko_eps;      /* Kreiss-Oliger strength epsilon (Sec. 2.3; the paper uses 0.005) */
  int buffer;         /* live global cells under a local edge; 0 selects NG+1 (Sec. 2.4.2) */
  int device;         /* CUDA device ordinal */
  void* stream;       /* cudaStream_t to enqueue on, or NULL */
  mpw_alloc_fn alloc; /* optional device allocator hook */
  mpw_free_fn free;
  void* alloc_user;
  int arith;          /* 0 (default): exact int64 fixed-point stencil sums in the RHS with
                         FP64 stage updates, and int64 fixed-point separable contractions
                         in the ghost-zone interpolation; 1: native FP64 throughout */
} mpw_config;

typedef struct {
  int kind;                 /* MPW_PATCH_GLOBAL (must be created first, id 0) or MPW_PATCH_LOCAL */
  int n[3];                 /* interior cells per axis, >= 6 */
  double lo[3], hi[3];      /* live box in the patch's numeric coordinates */
  int outer_bc;             /* global: ANALYTIC or PERIODIC; local: INTERPATCH */
  int motion;               /* MPW_MOTION_*; the global patch must be STATIC at the origin
                               when local patches exist */
  double motion_params[16]; /* The map to the background frame is X_B = R(t) X' + X0(t) with
                               R = I except for ROTATING (Sec. 2.4, numeric -> background):
                               STATIC   : X0 = (p0,p1,p2)
                               LINEAR   : X0 = (p0,p1,p2) + t (p3,p4,p5)
                               CIRCULAR : X0 = (p0,p1,p2) + p3 (cos(p4 t + p5), sin(p4 t + p5), 0)
                               ROTATING : X0 = (p0,p1,p2) + t (p3,p4,p5) and R the rotation by
                                          theta = p9 t + p10 about the unit axis (p6,p7,p8),
                                          counter-clockwise seen from the axis tip (Rodrigues'
                                          formula); the rotating local patch of Sec. 3.2.  The
                                          axis must have unit length (within 1e-12).  The frame
                                          velocity entering the RHS is then position dependent,
                                          w(X') = p9 n x X' + R^T (p3,p4,p5).  Validation of a
                                          rotating patch (overlap, distance to the global faces)
                                          uses the bounding box of its rotated box. */
  int topology;             /* MPW_TOPOLOGY_CARTESIAN (numeric x, y, z), or MPW_TOPOLOGY_SPHERICAL for a
                               local shell (the paper's spherical local patch, Sec. 3.3) with numeric
                               coordinates (r, theta, phi): n = cells along r, theta, phi; lo = (r_lo,
                               theta_lo, 0), hi = (r_hi, theta_hi, 2 pi) (the full azimuth, periodic); the
                               ghost nodes must stay off the origin and the poles (r_lo - 3 h_r > 0,
                               theta_lo - 3 h_theta > 0, theta_hi + 3 h_theta < pi), and the physical
                               spacings h_r, r_hi h_theta and r_hi h_phi must not exceed the global
                               spacing.  X' = r (sin theta cos phi, sin theta sin phi, cos theta) is the
                               patch frame the motion law maps.  Precision 64 only.  Errors: MPW_ERR_ARG. */
} mpw_patch_desc;

/* Create a context on cfg->device.  cfg is copied.  Errors: MPW_ERR_ARG for
 * unsupported precision/ghost/interp_points, MPW_ERR_CUDA. */
mpw_status mpw_create(const mpw_config* cfg, mpw_ctx** out);

/* Add a patch (Sec. 2.4.1: one global patch id 0, local patches 1..N-1) and
 * allocate its device storage (4 padded state buffers x 2 fields).  Returns
 * its id in *patch_id.  Errors: MPW_ERR_ARG, MPW_ERR_STATE (global patch not
 * first / already stepped), MPW_ERR_CUDA (allocation). */
mpw_status mpw_create_patch(mpw_ctx* ctx, const mpw_patch_desc* desc, int* patch_id);

/* Closed-form solution used by the analytic outer BC and mpw_fill_analytic
 * (Sec. 3: analytic BCs at the physical edges of the global domain).
 *   GAUSS_SUM     count pulses, params 5 per pulse (A, width, cx, cy, cz):
 *                 psi = sum [g(t+r) - g(t-r)]/(2r), g(s) = A s exp(-s^2/width^2)
 *   PLANE_SUM     params (C, then 5 per wave: A, kx, ky, kz, phase):
 *                 psi = C + sum A sin(k.x - |k| t + phase)   (Sec. 3, Eq. wave_solution)
 *   HARMONIC_POLY count <= 14 coefficients of the static harmonic basis
 *                 1, x, y, z, xy, yz, zx, x^2-y^2, y^2-z^2, xyz, x^3-3xy^2,
 *                 y^3-3yz^2, z^3-3zx^2, x^4-6x^2y^2+y^4 (Pi = 0).
 *   PLANE_GAUSS   params (C, A, kx, ky, kz, phase) of one plane wave, then count
 *                 pulses of 5 params as in GAUSS_SUM: the sum of the two solutions.
 * params is host memory and is copied.  Errors: MPW_ERR_ARG. */
mpw_status mpw_set_analytic(mpw_ctx* ctx, int kind, const double* params, int count);

/* Set every patch's interior to the closed form at time t and the context time
 * to t.  Errors: MPW_ERR_STATE (no analytic function), MPW_ERR_CUDA. */
mpw_status mpw_fill_analytic(mpw_ctx* ctx, double t);

/* Copy the interior of both fields of `patch` in (psi, Pi dense [k][j][i]).
 * The cover flags are left as they are (a restart restores them with
 * mpw_set_flags). */
mpw_status mpw_set_fields(mpw_ctx* ctx, int patch, const double* psi, const double* pi, int on_device);

/* Copy the interior of both fields out.  Global cells that are not live
 * (effective ghost or deactivated, Sec. 2.4.2) read as NaN. */
mpw_status mpw_get_fields(mpw_ctx* ctx, int patch, double* psi, double* pi, int on_device);

/* Asynchronous host transfers for pipelined use (no counterpart in the
 * paper): the copies run on the GPU's copy engines, on two streams of the
 * context's own, so that the next step's input travels in and the last
 * step's result travels out while a step computes.  psi and pi must be
 * page-locked host arrays (dense interior, binary64); MPW_ERR_ARG otherwise.
 *   mpw_set_fields_async queues psi, pi as the new interior of `patch`: they
 *     are copied into a device staging buffer and enter u at the start of
 *     the next call that reads or writes u (mpw_step, a get, a fill ...).
 *     The host arrays must stay unchanged until mpw_sync.
 *   mpw_get_fields_async copies the current interior out (NaN on non-live
 *     global cells, as mpw_get_fields) through a device staging buffer; the
 *     host arrays hold it after mpw_sync.  A second get of the same patch
 *     waits on the device for the first to leave the staging buffer.
 *   mpw_sync waits for the context's stream and both copy streams, then
 *     reports device-side errors of earlier mpw_step_async calls.
 * Staging takes 2 x 2 x n0 n1 n2 doubles per patch, allocated on first use. */
mpw_status mpw_set_fields_async(mpw_ctx* ctx, int patch, const double* psi, const double* pi);
mpw_status mpw_get_fields_async(mpw_ctx* ctx, int patch, double* psi, double* pi);
mpw_status mpw_sync(mpw_ctx* ctx);

/* Copy the whole padded box of the state u (ghost zones included) out, dense
 * [k][j][i] over (n+6)^3, index (i+3) + (n0+6)((j+3) + (n1+6)(k+3)).  Ghost
 * values are those of the last boundary fill of substage 1 (or of
 * mpw_fill_ghosts).  For tests of the ghost-zone fill.  Host or device. */
mpw_status mpw_get_padded(mpw_ctx* ctx, int patch, double* psi, double* pi, int on_device);

/* Time of the state. */
mpw_status mpw_set_time(mpw_ctx* ctx, double t);
double mpw_time(const mpw_ctx* ctx);

/* Recompute the cover flags at the current time (Sec. 2.4.2), poisoning
 * deactivated cells with NaN and reviving cells that became live. */
mpw_status mpw_compute_flags(mpw_ctx* ctx);

/* Read / restore the global cover flags (n0*n1*n2 bytes, host memory).  A
 * checkpoint is fields + flags + time. */
mpw_status mpw_get_flags(mpw_ctx* ctx, uint8_t* flags);
mpw_status mpw_set_flags(mpw_ctx* ctx, const uint8_t* flags);

/* Test support for the bounded-wait error path (no counterpart in the
 * paper).  Every mbarrier wait of the RHS kernels' TMA pipeline gives up
 * after `limit` try-waits, sets the device error word and lets the CTA drain
 * its own copies in flight (that drain always uses the default limit) and
 * return; the step then reports MPW_ERR_TIMEOUT.  The default is 2^20
 * (about a second and more); 0 makes every such wait give up at once, which
 * is how the tests drive the error path without a real stall.
 * Errors: MPW_ERR_ARG for a null context. */
mpw_status mpw_set_wait_limit(mpw_ctx* ctx, unsigned limit);

/* Fill every ghost zone of the state u at time t (maps at t): physical BC,
 * Local-to-Global, Global-to-Local (Sec. 2.4).  Flags are computed first if
 * invalid. */
mpw_status mpw_fill_ghosts(mpw_ctx* ctx, double t);

/* Advance nsteps RK4 steps of size dt (Sec. 2.3, Table 1).  Validates CFL,
 * traversal, separation and containment before launching; reads the device
 * error word once at the end.  On a device-side error the call returns
 * MPW_ERR_GHOST_UNFILLED (a ghost point was skipped, Sec. 2.4.1) or
 * MPW_ERR_TIMEOUT (a bounded wait ran out).  The steps run to the end either
 * way, so the fields then hold an invalid result: restore a checkpoint
 * (fields, flags, time) before stepping on.  The error word is cleared once
 * it has been read. */
mpw_status mpw_step(mpw_ctx* ctx, double dt, int nsteps);

/* As mpw_step, but returns once the work is enqueued: the device error word
 * is read by the next mpw_sync (or mpw_step) instead, so the host can queue
 * the next step's transfers while this one computes.  Host-side validation
 * errors are still returned at once. */
mpw_status mpw_step_async(mpw_ctx* ctx, double dt, int nsteps);

/* ---- Batches: many independent multipatch instances advanced together.
 * The paper has no counterpart (it runs one instance per set of MPI ranks);
 * this is the batching pattern of serving many small simulations on one GPU.
 * Each instance is an ordinary context.  A batched step does per instance
 * what mpw_step does on the host (validation, the choice of the cells whose
 * cover flags can change, exponent slots), but every ghost fill and every
 * RHS + stage substage is ONE kernel launch over all instances (plus one RHS
 * launch over the spherical shells of up to 64 instances, when there are
 * shells), and when every patch translates the cover flags of all instances
 * are one batched launch too, so small instances share the GPU instead of
 * running one after the other.  Instances may hold rotating patches and
 * spherical shells (their flags are then launched per instance).  Results
 * are bit for bit those of mpw_step on each context.
 *
 * mpw_batch_create: ctxs[0..n) must be distinct, live, hold a global patch,
 *   and share device, stream, precision, interp_points and arith; the array
 *   is copied, the contexts stay owned by the caller and must outlive the
 *   batch.  Allocates the argument tables (device and page-locked host).
 *   Errors: MPW_ERR_ARG, MPW_ERR_STATE, MPW_ERR_CUDA.
 * mpw_batch_step: advance every instance i by nsteps steps of dt[i] (host
 *   array of n doubles).  The first steps of a batch also tune the RHS
 *   chunk depth (planes marched per CTA): each candidate (8, 16, 32, 64)
 *   runs one step, timed with CUDA events from the first RHS launch of the
 *   step to the end of its last one, and the fastest is kept.
 *   Errors as mpw_step, for the first instance that fails.  A step that
 *   fails before its launches are queued (a host-side check) leaves every
 *   instance at its last completed step.
 *   After the tuning steps the copies and launches of a step are captured in
 *   a CUDA graph (one per argument buffer) and replayed; the replayed copies
 *   pick up each step's arguments from the page-locked buffers.  With moving
 *   patches the grids are padded to a capacity (blocks past a step's own
 *   total exit at once) and a step whose grids outgrow it is captured anew.
 *   Batches with moving spherical shells launch directly.
 * mpw_batch_tuning: the chosen chunk depth (0 while tuning), its measured
 *   time per step in ms (first RHS launch to the end of the last; three ghost
 *   fills lie in between), the number of batched launches so far and the
 *   number of steps replayed from a captured graph.
 * mpw_batch_destroy: frees the tables (not the contexts). */
typedef struct mpw_batch mpw_batch;
mpw_status mpw_batch_create(mpw_ctx* const* ctxs, int n, mpw_batch** out);
mpw_status mpw_batch_step(mpw_batch* batch, const double* dt, int nsteps);
mpw_status mpw_batch_tuning(const mpw_batch* batch, int* chunk, double* rhs_ms, long long* launches,
                            long long* graph_steps);
void mpw_batch_destroy(mpw_batch* batch);

/* Number of live points summed over patches (the unit of the throughput
 * metric: one live point advanced through one RK4 substage). */
mpw_status mpw_live_points(mpw_ctx* ctx, long long* count);

/* Kernel families reported by mpw_profile_read. */
enum { MPW_KERNEL_RHS = 0, MPW_KERNEL_FILL = 1, MPW_KERNEL_FLAGS = 2, MPW_KERNEL_FAMILIES = 3 };

/* Measurement support (no counterpart in the paper, which reports no
 * timings).  While enabled (enable = 1) every kernel launch of the context is
 * bracketed by a pair of CUDA events on the context's stream.  Launch counts
 * are kept whether or not timing is enabled. */
mpw_status mpw_profile_enable(mpw_ctx* ctx, int enable);

/* Synchronise the stream, write for families 0..n-1 the device milliseconds
 * accumulated by timed launches (ms, may be NULL) and the number of launches
 * (launches, may be NULL) since the last read, then reset both. */
mpw_status mpw_profile_read(mpw_ctx* ctx, double* ms, long long* launches, int n);

/* Largest interior extent per axis accepted by mpw_step_periodic_noalloc. */
#define MPW_NOALLOC_MAX_N 48

/* Advance one periodic Cartesian patch (static frame) by nsteps RK4 steps
 * without allocating any memory.  The paper has no counterpart; the entry
 * point exists for callers that may not allocate device memory when they step
 * a field: plugins whose host application owns every device allocation, and
 * timing-critical loops that must not enter the driver's allocator.  It runs
 * the same ghost-fill and fused RHS + RK4 stage kernels as mpw_step on a single
 * periodic patch, with every work buffer (padded state, accumulator, stage
 * buffers, exponent slots, error word) in one file-scope device array of about
 * 12 MB that each GPU loading the library holds until the process exits.
 *   n, lo, hi  patch extents (host memory); each n must lie in
 *              [6, MPW_NOALLOC_MAX_N], larger sizes return MPW_ERR_ARG.
 *   ko_eps     Kreiss-Oliger strength; dt, nsteps as in mpw_step (dt is checked
 *              against the RK4 stability estimate, MPW_ERR_CFL).
 *   psi, pi    device pointers on the current device, dense [k][j][i]
 *              interiors; read at the start, overwritten with the result.
 *   stream     cudaStream_t to enqueue on (NULL: the legacy default stream).
 * No cudaMalloc/cudaFree (or other allocating routine) is called.
 * The first call on a device looks up the device address of the array
 * (cudaGetSymbolAddress); make that first call before any stream capture
 * begins.  All calls share the array, which keeps the last call's contents
 * (the exponent slots and error word are cleared at the start of each call):
 * calls whose work overlaps on the GPU (other streams, unordered host
 * threads) race and corrupt each other.  The call returns once the work has
 * finished on `stream`: it then reads the device error word into a host
 * stack variable (no allocation) and synchronises the stream.
 * Errors: MPW_ERR_ARG, MPW_ERR_CFL (before any work is enqueued),
 * MPW_ERR_TIMEOUT (a bounded device wait ran out) and
 * MPW_ERR_GHOST_UNFILLED (a ghost point could not be filled) with psi and
 * pi then holding an incomplete result, MPW_ERR_CUDA; a message is kept for
 * mpw_last_error(). */
mpw_status mpw_step_periodic_noalloc(const int n[3], const double lo[3], const double hi[3], double ko_eps,
                                     double dt, int nsteps, double* psi, double* pi, void* stream);

/* Thread-local message of the last failing call on this thread. */
const char* mpw_last_error(void);

/* Free all device storage of the context. */
void mpw_destroy(mpw_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
