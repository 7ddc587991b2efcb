/*
 * oracle.h -- plain FP64 CPU oracle for the multipatch scalar-wave method of
 * "PatchworkWave" (arXiv:2002.00088).
 *
 * TEST INFRASTRUCTURE ONLY.  This directory is the slow, obviously correct
 * restatement of the method that the CUDA library is checked against.  Only
 * the test suite, the package smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or constant with
 * the CUDA library (paper_2002_00088_gb300/csrc), and neither includes the
 * other.
 *
 * What it computes, in the paper's order (one full step, Sec. 2.3-2.4):
 *   1. cover flags at t_n with the buffer of live global cells under each
 *      local patch edge (Sec. 2.4.2, "Calculate Cover Flags with Buffer");
 *   2. for each RK4 substage l = 1..4 at t_n + c_l dt (Table 1, Eqs. k1-k4):
 *      stage state u_n + dt a_{l,l-1} K_{l-1};
 *      ghost zones in the order physical -> interpatch (Sec. 2.4), the
 *      interpatch part being Local-to-Global then Global-to-Local, each a
 *      tensor-product Lagrange interpolation (Eq. Pijk) through the patch
 *      maps at that substage time;
 *      slope K_l = RHS of the two-field wave system on live points, 4th-order
 *      centred differences plus 6th-derivative Kreiss-Oliger dissipation
 *      (Sec. 2.2, Eqs. eom1-eom3; Sec. 2.3, KO with n = 5);
 *   3. u_{n+1/2} = u_n + dt (b1 K1 + b2 K2 + b3 K3),
 *      u_{n+1}   = u_{n+1/2} + dt b4 K4            (Sec. 2.3).
 *
 * Layout: every patch stores each field as a padded box of (n+6)^3 doubles,
 * x fastest, with NG = 3 ghost cells per side; cell-centred nodes
 * x_i = lo + (i + 1/2) h, h = (hi - lo) / n.
 * Dense interior arrays exchanged through this API are [k][j][i], i fastest.
 *
 * Every function returns 0 on success and a negative code on error; the
 * message is available from orc_error().
 */
#ifndef PATCHWORK_ORACLE_H
#define PATCHWORK_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_NG 3
#define ORC_MAX_PATCHES 16
#define ORC_MAX_APARAMS 1024

enum { ORC_GLOBAL = 0, ORC_LOCAL = 1 };
/* patch topology: CARTESIAN (numeric x, y, z) or SPHERICAL (a local shell with
 * numeric (r, theta, phi), theta in (0, pi) away from the poles, phi periodic
 * over [0, 2 pi)) */
enum { ORC_CARTESIAN = 0, ORC_SPHERICAL = 1 };
enum { ORC_BC_ANALYTIC = 0, ORC_BC_PERIODIC = 1, ORC_BC_INTERPATCH = 2 };
enum { ORC_STATIC = 0, ORC_LINEAR = 1, ORC_CIRCULAR = 2, ORC_ROTATING = 3 };
enum { ORC_GAUSS_SUM = 0, ORC_PLANE_SUM = 1, ORC_HARMONIC_POLY = 2, ORC_PLANE_GAUSS = 3 };
/* flag byte of a global interior cell: state | (owning local patch << 2) */
enum { ORC_LIVE = 0, ORC_GHOST = 1, ORC_DEAD = 2, ORC_REVIVED = 3 };

enum {
  ORC_ERR_ARG = -1,
  ORC_ERR_OVERLAP = -2,
  ORC_ERR_UNFILLED = -3,   /* a ghost point could not be interpolated */
  ORC_ERR_DONOR = -4,      /* an interpolation window touched non-live data */
  ORC_ERR_STATE = -5
};

typedef struct {
  int kind;                 /* ORC_GLOBAL (id 0, exactly one) or ORC_LOCAL */
  int n[3];                 /* interior cells per axis */
  double lo[3], hi[3];      /* numeric-coordinate extent of the live box */
  int outer_bc;             /* global: ANALYTIC or PERIODIC; local: INTERPATCH */
  int motion;               /* ORC_STATIC / ORC_LINEAR / ORC_CIRCULAR / ORC_ROTATING */
  double motion_params[16]; /* see orc_motion() and orc_frame() */
  int topology;             /* ORC_CARTESIAN or ORC_SPHERICAL (local patches only) */
} orc_patch_desc;

typedef struct orc_sim orc_sim;

orc_sim* orc_create(int interp_points, double ko_eps, int buffer);
void orc_destroy(orc_sim* s);
const char* orc_error(const orc_sim* s);

int orc_add_patch(orc_sim* s, const orc_patch_desc* d);          /* returns id >= 0 */
int orc_set_analytic(orc_sim* s, int kind, const double* params, int count);
int orc_fill_analytic(orc_sim* s, double t);                       /* interiors <- closed form */
int orc_set_fields(orc_sim* s, int patch, const double* psi, const double* pi);
int orc_get_fields(const orc_sim* s, int patch, double* psi, double* pi);
/* which = 0: state u (U); which = 1: the last stage/ghost-filled state (Y) */
int orc_set_padded(orc_sim* s, int patch, int which, const double* psi, const double* pi);
int orc_get_padded(const orc_sim* s, int patch, int which, double* psi, double* pi);
void orc_set_time(orc_sim* s, double t);
double orc_time(const orc_sim* s);
int orc_set_threads(orc_sim* s, int nthreads);
/* 1 (default): Local-to-Global before Global-to-Local; 0: the reverse.
 * Sec. 2.4.1 states the two are interchangeable without overlapping patches. */
int orc_set_fill_order(orc_sim* s, int l2g_first);

int orc_compute_flags(orc_sim* s);                  /* flags + revival at current time */
int orc_get_flags(const orc_sim* s, unsigned char* flags);
int orc_set_flags(orc_sim* s, const unsigned char* flags);
int orc_fill_ghosts(orc_sim* s, double t);          /* Y <- U on live points, then all BCs at t */
int orc_eval_rhs(orc_sim* s, int patch, double t, double* kpsi, double* kpi);
int orc_step(orc_sim* s, double dt, int nsteps);
/* hybrid-step pieces (the learned surrogate, an extension of the method):
 * dead global cells of Y from their local patch's u at t; one RK4 step of
 * the local patches with the global's stage states prescribed
 * (gstage[2 l + f]: substage l, field f, interior in (k, j, i) order) */
int orc_fill_dead(orc_sim* s, double t);
int orc_step_locals(orc_sim* s, double dt, const double* const* gstage);
long orc_live_points(const orc_sim* s);
double orc_energy(const orc_sim* s, int patch);

/* building blocks, exposed for the pins */
void orc_motion(int motion, const double* mp, double t, double X0[3], double w[3]);
/* map of a patch at time t: X_B = R X' + X0, R row-major (identity unless
 * ORC_ROTATING) */
void orc_frame(int motion, const double* mp, double t, double R[9], double X0[3]);
/* frame velocity w (patch components) at the patch point X' */
void orc_frame_velocity(int motion, const double* mp, double t, const double xl[3], double w[3]);
int orc_lagrange(int P, double s, double* w);      /* returns the window start index */
void orc_closed_form(int kind, const double* params, int count, double t,
                     double x, double y, double z, double* psi, double* pi);

#ifdef __cplusplus
}
#endif
#endif
