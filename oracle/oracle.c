/*
 * oracle.c -- plain FP64 CPU oracle for the multipatch scalar-wave method of
 * "PatchworkWave" (arXiv:2002.00088).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark, never by the library.  It shares no code
 * with the CUDA path.  Every loop below is the plain definition: no blocking,
 * no fusion, no reordering beyond what the paper's formulas state.  The only
 * concession to speed is an optional OpenMP split of the outer k loop of the
 * per-point loops, which does not change any point's arithmetic.
 *
 * Pinned by tests/test_oracle_*.py (closed forms, exact Fourier-mode
 * evolution, polynomial exactness of the stencils and of the interpolation,
 * brute-force cover flags, energy, 4th-order convergence).
 */
#include "oracle.h"

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NG ORC_NG
#define ORC_PI 3.14159265358979323846

typedef struct {
  orc_patch_desc d;
  double h[3];
  int m[3];        /* padded extent n + 2 NG */
  long vol;        /* padded volume */
  double* U[2];    /* u_n (becomes u_{n+1} at the end of a step) */
  double* Y[2];    /* state of the current substage, ghost zones filled */
  double* K[4][2]; /* slopes K_1..K_4 */
} opatch;

struct orc_sim {
  int P, buffer, nthreads, l2g_first;
  double eps;
  int np;
  opatch p[ORC_MAX_PATCHES];
  int akind, acount;
  double ap[ORC_MAX_APARAMS];
  unsigned char* flags; /* global interior, [k][j][i] */
  int flags_valid;
  double t;
  char err[256];
};

/* Classic RK4, Butcher tableau of Table 1 (Sec. 2.3): c_l, a_{l,l-1}, b_l. */
static const double RK_C[4] = {0.0, 0.5, 0.5, 1.0};
static const double RK_A[4] = {0.0, 0.5, 0.5, 1.0};
static const double RK_B[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};

static int fail(orc_sim* s, int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(s->err, sizeof s->err, fmt, ap);
  va_end(ap);
  return code;
}

static long at(const opatch* p, int i, int j, int k) {
  return ((long)(k + NG) * p->m[1] + (j + NG)) * p->m[0] + (i + NG);
}

static int in_interior(const opatch* p, int i, int j, int k) {
  return i >= 0 && i < p->d.n[0] && j >= 0 && j < p->d.n[1] && k >= 0 && k < p->d.n[2];
}

static long gidx(const opatch* g, int i, int j, int k) {
  return ((long)k * g->d.n[1] + j) * g->d.n[0] + i;
}

/* Cell-centred node of index i on axis a (numeric coordinates). */
static double node(const opatch* p, int a, int i) { return p->d.lo[a] + (i + 0.5) * p->h[a]; }

/* A point of patch pi is evolved ("live") unless it is a global cell that is
 * covered by a local patch beyond the buffer (Sec. 2.4.2). */
static int is_live(const orc_sim* s, int pi, int i, int j, int k) {
  const opatch* p = &s->p[pi];
  if (!in_interior(p, i, j, k)) return 0;
  if (pi != 0 || !s->flags_valid) return 1;
  int st = s->flags[gidx(p, i, j, k)] & 3;
  return st == ORC_LIVE || st == ORC_REVIVED;
}

/* ------------------------------------------------------------------------ */
/* Patch motion.  Local patches move rigidly: X_B = R(t) X' + X0(t).  Under
 * translation R = I and w = dX0/dt is the frame velocity entering the RHS.
 *   STATIC   : X0 = (p0, p1, p2)
 *   LINEAR   : X0 = (p0, p1, p2) + t (p3, p4, p5)
 *   CIRCULAR : X0 = (p0, p1, p2) + p3 (cos(p4 t + p5), sin(p4 t + p5), 0)
 *              (centre, radius, angular speed, phase; orbit in the z = p2 plane)
 *   ROTATING : X0 = (p0, p1, p2) + t (p3, p4, p5), and R(t) the rotation by
 *              theta = p9 t + p10 about the unit axis n = (p6, p7, p8), see
 *              orc_frame (the rotating local patch of Sec. 3.2, Test Two);
 *              orc_motion returns X0 and the frame velocity at X' = 0. */
void orc_motion(int motion, const double* mp, double t, double X0[3], double w[3]) {
  int a;
  if (motion == ORC_ROTATING) {
    const double zero[3] = {0.0, 0.0, 0.0};
    double R[9];
    orc_frame(motion, mp, t, R, X0);
    orc_frame_velocity(motion, mp, t, zero, w);
  } else if (motion == ORC_LINEAR) {
    for (a = 0; a < 3; ++a) {
      X0[a] = mp[a] + t * mp[3 + a];
      w[a] = mp[3 + a];
    }
  } else if (motion == ORC_CIRCULAR) {
    double ph = mp[4] * t + mp[5];
    double c = cos(ph), sn = sin(ph);
    X0[0] = mp[0] + mp[3] * c;
    X0[1] = mp[1] + mp[3] * sn;
    X0[2] = mp[2];
    w[0] = -(mp[3] * mp[4]) * sn;
    w[1] = (mp[3] * mp[4]) * c;
    w[2] = 0.0;
  } else {
    for (a = 0; a < 3; ++a) {
      X0[a] = mp[a];
      w[a] = 0.0;
    }
  }
}

/* Rotation about the unit axis n by theta, right-handed (counter-clockwise
 * seen from the tip of n), by Rodrigues' formula
 *   R = cos(theta) I + sin(theta) [n]_x + (1 - cos(theta)) n n^T,
 * [n]_x the cross-product matrix ([n]_x v = n x v).  For n = z this is the
 * rotation of the x-y plane by theta.  The entries are formed in a fixed
 * order: the cover flags depend on their last bit. */
void orc_frame(int motion, const double* mp, double t, double R[9], double X0[3]) {
  if (motion != ORC_ROTATING) {
    double w[3];
    orc_motion(motion, mp, t, X0, w);
    for (int e = 0; e < 9; ++e) R[e] = (e % 4 == 0) ? 1.0 : 0.0;
    return;
  }
  const double* n = mp + 6;
  const double th = mp[9] * t + mp[10];
  const double c = cos(th), sn = sin(th), omc = 1.0 - c;
  const double K[9] = {0.0, -n[2], n[1], n[2], 0.0, -n[0], -n[1], n[0], 0.0};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) R[3 * a + b] = ((a == b ? c : 0.0) + sn * K[3 * a + b]) + (omc * n[a]) * n[b];
  for (int a = 0; a < 3; ++a) X0[a] = mp[a] + t * mp[3 + a];
}

/* Frame velocity at the patch point X' in patch components: the background
 * velocity of the moving node, dX_B/dt = Omega n x (R X') + V, taken back to
 * the patch frame, w = R^T dX_B/dt = Omega n x X' + R^T V (R^T n = n). */
void orc_frame_velocity(int motion, const double* mp, double t, const double xl[3], double w[3]) {
  double R[9], X0[3];
  if (motion != ORC_ROTATING) {
    orc_motion(motion, mp, t, X0, w);
    return;
  }
  orc_frame(motion, mp, t, R, X0);
  const double* n = mp + 6;
  const double om = mp[9];
  const double cr[3] = {n[1] * xl[2] - n[2] * xl[1], n[2] * xl[0] - n[0] * xl[2], n[0] * xl[1] - n[1] * xl[0]};
  for (int a = 0; a < 3; ++a) w[a] = om * cr[a] + (R[a] * mp[3] + R[3 + a] * mp[4] + R[6 + a] * mp[5]);
}

/* The map of one patch at one time, and the two directions of it.  A
 * spherical shell's numeric coordinates (r, theta, phi) first go to the
 * Cartesian patch frame, X' = r (sin theta cos phi, sin theta sin phi,
 * cos theta); the rigid motion then acts on X'. */
typedef struct {
  int rot, sph;
  double R[9], X0[3];
} oframe;

static oframe frame_at(const opatch* p, double t) {
  oframe f;
  f.rot = p->d.motion == ORC_ROTATING;
  f.sph = p->d.topology == ORC_SPHERICAL;
  orc_frame(p->d.motion, p->d.motion_params, t, f.R, f.X0);
  return f;
}

static void sph_to_cart(const double q[3], double x[3]) {
  const double st = sin(q[1]);
  x[0] = q[0] * st * cos(q[2]);
  x[1] = q[0] * st * sin(q[2]);
  x[2] = q[0] * cos(q[1]);
}

/* X_B = R X' + X0 (translation: X' + X0) of the patch point with numeric
 * coordinates xl */
static void to_background(const oframe* f, const double xl[3], double xb[3]) {
  double x[3] = {xl[0], xl[1], xl[2]};
  if (f->sph) sph_to_cart(xl, x);
  for (int a = 0; a < 3; ++a)
    xb[a] = f->rot ? ((f->R[3 * a] * x[0] + f->R[3 * a + 1] * x[1]) + f->R[3 * a + 2] * x[2]) + f->X0[a]
                   : x[a] + f->X0[a];
}

/* X' = R^T (X_B - X0) (translation: X_B - X0), the Cartesian patch frame */
static void to_frame(const oframe* f, const double xb[3], double x[3]) {
  const double d[3] = {xb[0] - f->X0[0], xb[1] - f->X0[1], xb[2] - f->X0[2]};
  for (int a = 0; a < 3; ++a) x[a] = f->rot ? (f->R[a] * d[0] + f->R[3 + a] * d[1]) + f->R[6 + a] * d[2] : d[a];
}

/* numeric coordinates of the background point xb in the patch (a shell:
 * r = |X'|, theta = acos(z'/r), phi = atan2(y', x') in [0, 2 pi)) */
static void to_local(const oframe* f, const double xb[3], double xl[3]) {
  double x[3];
  to_frame(f, xb, x);
  if (!f->sph) {
    for (int a = 0; a < 3; ++a) xl[a] = x[a];
    return;
  }
  const double r = sqrt((x[0] * x[0] + x[1] * x[1]) + x[2] * x[2]);
  double c = r > 0.0 ? x[2] / r : 1.0;
  c = c > 1.0 ? 1.0 : (c < -1.0 ? -1.0 : c);
  double ph = atan2(x[1], x[0]);
  if (ph < 0.0) ph += 2.0 * ORC_PI;
  xl[0] = r;
  xl[1] = acos(c);
  xl[2] = ph;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.4, 1-D Lagrange interpolation and Eq. (Pijk).  s is the position in
 * index units of the donor grid (node q sits at s = q).  i_c = floor(s) is the
 * node closest to the point without exceeding it; the window starts at
 * i_c - 2 and holds P nodes (P = 6: i_c-2..i_c+3 as in the paper; P = 5:
 * i_c-2..i_c+2).  w[m] = prod_{q != m} (s - x_q) / (x_m - x_q). */
int orc_lagrange(int P, double s, double* w) {
  int start = (int)floor(s) - 2;
  for (int m = 0; m < P; ++m) {
    double xm = (double)(start + m), num = 1.0, den = 1.0;
    for (int q = 0; q < P; ++q) {
      if (q == m) continue;
      double xq = (double)(start + q);
      num *= (s - xq);
      den *= (xm - xq);
    }
    w[m] = num / den;
  }
  return start;
}

/* ------------------------------------------------------------------------ */
/* Closed-form solutions used as initial data and as analytic outer BCs.
 * GAUSS_SUM   params per pulse (A, width, cx, cy, cz): outgoing+incoming
 *             spherical wave with psi(0) = A exp(-r^2/width^2), Pi(0) = 0:
 *             psi = [g(t+r) - g(t-r)] / (2r), g(s) = A s exp(-s^2/width^2).
 * PLANE_SUM   params (C, then per wave A, kx, ky, kz, phase):
 *             psi = C + sum A sin(k.x - |k| t + phase)   (Sec. 3, Eq.
 *             wave_solution and the superposition of Sec. 3.4.2).
 * HARMONIC_POLY params: coefficients of the static harmonic basis
 *             1, x, y, z, xy, yz, zx, x^2-y^2, y^2-z^2, xyz, x^3-3xy^2,
 *             y^3-3yz^2, z^3-3zx^2, x^4-6x^2y^2+y^4;  Pi = 0.
 * PLANE_GAUSS params (C, A, kx, ky, kz, phase) of one plane wave, then
 *             count Gaussian pulses as in GAUSS_SUM: their sum.             */
static void gauss_derivs(double A, double a, double s, double g[5]) {
  double e = A * exp(-a * s * s), s2 = s * s;
  g[0] = e * s;
  g[1] = e * (1.0 - 2.0 * a * s2);
  g[2] = e * (4.0 * a * a * s2 * s - 6.0 * a * s);
  g[3] = e * (-6.0 * a + 24.0 * a * a * s2 - 8.0 * a * a * a * s2 * s2);
  g[4] = e * (60.0 * a * a * s - 80.0 * a * a * a * s2 * s + 16.0 * a * a * a * a * s2 * s2 * s);
}

void orc_closed_form(int kind, const double* prm, int count, double t, double x, double y, double z,
                     double* psi, double* pi) {
  double ps = 0.0, pv = 0.0;
  if (kind == ORC_GAUSS_SUM) {
    for (int q = 0; q < count; ++q) {
      const double* g = prm + 5 * q;
      double A = g[0], a = 1.0 / (g[1] * g[1]);
      double dx = x - g[2], dy = y - g[3], dz = z - g[4];
      double r = sqrt(dx * dx + dy * dy + dz * dz);
      if (r < 1e-5) { /* Taylor series in r of the same expression */
        double d[5];
        gauss_derivs(A, a, t, d);
        ps += d[1] + r * r * d[3] / 6.0;
        pv += d[2] + r * r * d[4] / 6.0;
      } else {
        double gp[5], gm[5];
        gauss_derivs(A, a, t + r, gp);
        gauss_derivs(A, a, t - r, gm);
        ps += (gp[0] - gm[0]) / (2.0 * r);
        pv += (gp[1] - gm[1]) / (2.0 * r);
      }
    }
  } else if (kind == ORC_PLANE_SUM) {
    ps = prm[0];
    for (int q = 0; q < count; ++q) {
      const double* wv = prm + 1 + 5 * q;
      double kk = sqrt(wv[1] * wv[1] + wv[2] * wv[2] + wv[3] * wv[3]);
      double th = wv[1] * x + wv[2] * y + wv[3] * z - kk * t + wv[4];
      ps += wv[0] * sin(th);
      pv -= wv[0] * kk * cos(th);
    }
  } else if (kind == ORC_PLANE_GAUSS) {
    /* one plane wave (C, A, kx, ky, kz, phase) plus count Gaussian pulses:
       the wave equation is linear, so the sum of the two solutions is one */
    double p1, v1, p2, v2;
    orc_closed_form(ORC_PLANE_SUM, prm, 1, t, x, y, z, &p1, &v1);
    orc_closed_form(ORC_GAUSS_SUM, prm + 6, count, t, x, y, z, &p2, &v2);
    ps = p1 + p2;
    pv = v1 + v2;
  } else if (kind == ORC_HARMONIC_POLY) {
    double b[14] = {1.0,
                    x,
                    y,
                    z,
                    x * y,
                    y * z,
                    z * x,
                    x * x - y * y,
                    y * y - z * z,
                    x * y * z,
                    x * x * x - 3.0 * x * y * y,
                    y * y * y - 3.0 * y * z * z,
                    z * z * z - 3.0 * z * x * x,
                    x * x * x * x - 6.0 * x * x * y * y + y * y * y * y};
    for (int q = 0; q < count && q < 14; ++q) ps += prm[q] * b[q];
  }
  *psi = ps;
  *pi = pv;
}

/* ------------------------------------------------------------------------ */
orc_sim* orc_create(int interp_points, double ko_eps, int buffer) {
  if (interp_points != 5 && interp_points != 6) return NULL;
  orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
  if (!s) return NULL;
  s->P = interp_points;
  s->eps = ko_eps;
  s->buffer = buffer > 0 ? buffer : NG + 1;
  s->nthreads = 1;
  s->l2g_first = 1;
  return s;
}

void orc_destroy(orc_sim* s) {
  if (!s) return;
  for (int q = 0; q < s->np; ++q) {
    for (int f = 0; f < 2; ++f) {
      free(s->p[q].U[f]);
      free(s->p[q].Y[f]);
      for (int l = 0; l < 4; ++l) free(s->p[q].K[l][f]);
    }
  }
  free(s->flags);
  free(s);
}

const char* orc_error(const orc_sim* s) { return s ? s->err : "null oracle"; }

int orc_set_threads(orc_sim* s, int nthreads) {
  s->nthreads = nthreads > 0 ? nthreads : 1;
  return 0;
}

int orc_set_fill_order(orc_sim* s, int l2g_first) {
  s->l2g_first = l2g_first ? 1 : 0;
  return 0;
}

static double* nan_array(long n) {
  double* a = (double*)malloc(sizeof(double) * (size_t)n);
  if (a)
    for (long i = 0; i < n; ++i) a[i] = NAN;
  return a;
}

int orc_add_patch(orc_sim* s, const orc_patch_desc* d) {
  if (s->np >= ORC_MAX_PATCHES) return fail(s, ORC_ERR_ARG, "too many patches");
  if ((s->np == 0) != (d->kind == ORC_GLOBAL))
    return fail(s, ORC_ERR_ARG, "patch 0 must be the single global patch");
  for (int a = 0; a < 3; ++a)
    if (d->n[a] < 2 * NG || !(d->hi[a] > d->lo[a])) return fail(s, ORC_ERR_ARG, "bad extent");
  if (d->motion < ORC_STATIC || d->motion > ORC_ROTATING) return fail(s, ORC_ERR_ARG, "bad motion law");
  if (d->topology == ORC_SPHERICAL) {
    /* a shell of full azimuth, its ghost nodes away from the origin and
     * from the poles */
    const double hr = (d->hi[0] - d->lo[0]) / d->n[0], ht = (d->hi[1] - d->lo[1]) / d->n[1];
    if (d->kind != ORC_LOCAL) return fail(s, ORC_ERR_ARG, "only local patches can be spherical shells");
    if (d->lo[0] - NG * hr <= 0.0 || d->lo[1] - NG * ht <= 0.0 || d->hi[1] + NG * ht >= ORC_PI)
      return fail(s, ORC_ERR_ARG, "shell ghost nodes must stay off the origin and the poles");
    if (d->lo[2] != 0.0 || fabs(d->hi[2] - 2.0 * ORC_PI) > 1e-12)
      return fail(s, ORC_ERR_ARG, "a shell spans the full azimuth [0, 2 pi)");
  } else if (d->topology != ORC_CARTESIAN) {
    return fail(s, ORC_ERR_ARG, "bad topology");
  }
  if (d->motion == ORC_ROTATING) {
    const double* n = d->motion_params + 6;
    if (fabs(n[0] * n[0] + n[1] * n[1] + n[2] * n[2] - 1.0) > 1e-12)
      return fail(s, ORC_ERR_ARG, "the rotation axis must be a unit vector");
  }
  opatch* p = &s->p[s->np];
  memset(p, 0, sizeof *p);
  p->d = *d;
  p->vol = 1;
  for (int a = 0; a < 3; ++a) {
    p->h[a] = (d->hi[a] - d->lo[a]) / d->n[a];
    p->m[a] = d->n[a] + 2 * NG;
    p->vol *= p->m[a];
  }
  for (int f = 0; f < 2; ++f) {
    p->U[f] = nan_array(p->vol);
    p->Y[f] = nan_array(p->vol);
    for (int l = 0; l < 4; ++l) p->K[l][f] = nan_array(p->vol);
    if (!p->U[f] || !p->Y[f]) return fail(s, ORC_ERR_ARG, "out of memory");
  }
  if (s->np == 0) {
    long n = (long)d->n[0] * d->n[1] * d->n[2];
    s->flags = (unsigned char*)calloc((size_t)n, 1);
  }
  s->flags_valid = 0;
  return s->np++;
}

int orc_set_analytic(orc_sim* s, int kind, const double* params, int count) {
  int need = kind == ORC_GAUSS_SUM     ? 5 * count
             : kind == ORC_PLANE_SUM   ? 1 + 5 * count
             : kind == ORC_PLANE_GAUSS ? 6 + 5 * count
                                       : count;
  if (need > ORC_MAX_APARAMS || count < 0) return fail(s, ORC_ERR_ARG, "too many analytic params");
  s->akind = kind;
  s->acount = count;
  memcpy(s->ap, params, sizeof(double) * (size_t)need);
  return 0;
}

void orc_set_time(orc_sim* s, double t) { s->t = t; }
double orc_time(const orc_sim* s) { return s->t; }

int orc_fill_analytic(orc_sim* s, double t) {
  for (int q = 0; q < s->np; ++q) {
    opatch* p = &s->p[q];
    oframe f = frame_at(p, t);
    for (int k = 0; k < p->d.n[2]; ++k)
      for (int j = 0; j < p->d.n[1]; ++j)
        for (int i = 0; i < p->d.n[0]; ++i) {
          long c = at(p, i, j, k);
          double xl[3] = {node(p, 0, i), node(p, 1, j), node(p, 2, k)}, xb[3];
          to_background(&f, xl, xb);
          orc_closed_form(s->akind, s->ap, s->acount, t, xb[0], xb[1], xb[2], &p->U[0][c], &p->U[1][c]);
        }
  }
  s->t = t;
  return 0;
}

int orc_set_fields(orc_sim* s, int q, const double* psi, const double* pi) {
  if (q < 0 || q >= s->np) return fail(s, ORC_ERR_ARG, "bad patch id");
  opatch* p = &s->p[q];
  long c = 0;
  for (int k = 0; k < p->d.n[2]; ++k)
    for (int j = 0; j < p->d.n[1]; ++j)
      for (int i = 0; i < p->d.n[0]; ++i, ++c) {
        p->U[0][at(p, i, j, k)] = psi[c];
        p->U[1][at(p, i, j, k)] = pi[c];
      }
  return 0;
}

int orc_get_fields(const orc_sim* s, int q, double* psi, double* pi) {
  if (q < 0 || q >= s->np) return ORC_ERR_ARG;
  const opatch* p = &s->p[q];
  long c = 0;
  for (int k = 0; k < p->d.n[2]; ++k)
    for (int j = 0; j < p->d.n[1]; ++j)
      for (int i = 0; i < p->d.n[0]; ++i, ++c) {
        int live = is_live(s, q, i, j, k);
        psi[c] = live ? p->U[0][at(p, i, j, k)] : NAN;
        pi[c] = live ? p->U[1][at(p, i, j, k)] : NAN;
      }
  return 0;
}

int orc_set_padded(orc_sim* s, int q, int which, const double* psi, const double* pi) {
  if (q < 0 || q >= s->np) return fail(s, ORC_ERR_ARG, "bad patch id");
  opatch* p = &s->p[q];
  double** dst = which ? p->Y : p->U;
  memcpy(dst[0], psi, sizeof(double) * (size_t)p->vol);
  memcpy(dst[1], pi, sizeof(double) * (size_t)p->vol);
  return 0;
}

int orc_get_padded(const orc_sim* s, int q, int which, double* psi, double* pi) {
  if (q < 0 || q >= s->np) return ORC_ERR_ARG;
  const opatch* p = &s->p[q];
  double* const* src = which ? p->Y : p->U;
  memcpy(psi, src[0], sizeof(double) * (size_t)p->vol);
  memcpy(pi, src[1], sizeof(double) * (size_t)p->vol);
  return 0;
}

long orc_live_points(const orc_sim* s) {
  long n = 0;
  for (int q = 0; q < s->np; ++q) {
    const opatch* p = &s->p[q];
    for (int k = 0; k < p->d.n[2]; ++k)
      for (int j = 0; j < p->d.n[1]; ++j)
        for (int i = 0; i < p->d.n[0]; ++i) n += is_live(s, q, i, j, k);
  }
  return n;
}

/* ------------------------------------------------------------------------ */
/* Tensor-product Lagrange interpolation, Eq. (Pijk), of both fields of the
 * donor patch q at numeric position x.  The whole window must lie in the
 * donor's interior and every donor cell must be live (the buffer guarantees
 * this: Sec. 2.4.2); otherwise the point is skipped and -1 is returned. */
static long wrap(int i, int n);

static int interp_point(const orc_sim* s, int q, double* const src[2], const double x[3], double out[2]) {
  const opatch* p = &s->p[q];
  const int sph = p->d.topology == ORC_SPHERICAL;
  double w[3][6];
  int st[3];
  for (int a = 0; a < 3; ++a) {
    double sidx = (x[a] - p->d.lo[a]) / p->h[a] - 0.5;
    st[a] = orc_lagrange(s->P, sidx, w[a]);
    /* the azimuth of a shell is periodic: its window wraps around */
    if (sph && a == 2) continue;
    if (st[a] < 0 || st[a] + s->P > p->d.n[a]) return -1;
  }
  double v0 = 0.0, v1 = 0.0;
  for (int c = 0; c < s->P; ++c)
    for (int b = 0; b < s->P; ++b)
      for (int a = 0; a < s->P; ++a) {
        int i = st[0] + a, j = st[1] + b, k = sph ? (int)wrap(st[2] + c, p->d.n[2]) : st[2] + c;
        if (!is_live(s, q, i, j, k)) return -2;
        long idx = at(p, i, j, k);
        double wt = w[0][a] * w[1][b] * w[2][c];
        v0 += wt * src[0][idx];
        v1 += wt * src[1][idx];
      }
  out[0] = v0;
  out[1] = v1;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Cover flags with buffer, Sec. 2.4.2 ("Find Covered Zones", "Calculate Cover
 * Flags with Buffer"), evaluated with the patch maps at the current time t_n
 * and then held for the whole step (Sec. 2.4.2, last paragraphs).
 *   covered : the global cell centre lies in a local patch's live box
 *             [lo, hi] (closed), tested in that patch's numeric coordinates;
 *   d       : L-infinity index distance to the nearest uncovered cell (cells
 *             outside the global interior count as uncovered);
 *   LIVE if d <= B (B = buffer, NG+1 by default), GHOST (effective ghost zone,
 *   filled by Local-to-Global) if B < d <= B+NG, DEAD (deactivated) beyond.
 * d <= r fails exactly when every cell within distance r is covered, so the
 * two thresholds are two erosions of the covered mask by cubes of half-width
 * B and B+NG; a cube erosion is the product of three 1-D erosions. */
static void erode_axis(const unsigned char* in, unsigned char* out, const int n[3], int axis, int r) {
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        int idx[3] = {i, j, k}, ok = 1;
        for (int dd = -r; dd <= r && ok; ++dd) {
          int v[3] = {i, j, k};
          v[axis] = idx[axis] + dd;
          if (v[axis] < 0 || v[axis] >= n[axis])
            ok = 0;
          else
            ok = in[((long)v[2] * n[1] + v[1]) * n[0] + v[0]] != 0;
        }
        out[((long)k * n[1] + j) * n[0] + i] = (unsigned char)ok;
      }
}

static void erode(const unsigned char* covered, unsigned char* out, unsigned char* tmp, const int n[3], int r) {
  erode_axis(covered, out, n, 0, r);
  erode_axis(out, tmp, n, 1, r);
  erode_axis(tmp, out, n, 2, r);
}

int orc_compute_flags(orc_sim* s) {
  if (s->np < 1) return fail(s, ORC_ERR_STATE, "no global patch");
  opatch* g = &s->p[0];
  long N = (long)g->d.n[0] * g->d.n[1] * g->d.n[2];
  unsigned char* owner = (unsigned char*)calloc((size_t)N, 1);
  unsigned char* cov = (unsigned char*)calloc((size_t)N, 1);
  unsigned char* e1 = (unsigned char*)calloc((size_t)N, 1);
  unsigned char* e2 = (unsigned char*)calloc((size_t)N, 1);
  unsigned char* tmp = (unsigned char*)calloc((size_t)N, 1);
  int rc = 0;
  if (!owner || !cov || !e1 || !e2 || !tmp) {
    rc = fail(s, ORC_ERR_ARG, "out of memory");
    goto done;
  }
  /* coverage test in each local patch's numeric coordinates */
  for (int q = 1; q < s->np && rc == 0; ++q) {
    opatch* p = &s->p[q];
    oframe f = frame_at(p, s->t);
    /* a shell covers r_lo <= r <= r_hi, theta_lo <= theta <= theta_hi, i.e.
     * r cos(theta_hi) <= z' <= r cos(theta_lo) (cos decreases on [0, pi]) */
    const double clo = cos(p->d.lo[1]), chi = cos(p->d.hi[1]);
    for (int k = 0; k < g->d.n[2] && rc == 0; ++k)
      for (int j = 0; j < g->d.n[1] && rc == 0; ++j)
        for (int i = 0; i < g->d.n[0]; ++i) {
          double xb[3] = {node(g, 0, i), node(g, 1, j), node(g, 2, k)}, xl[3];
          int inside = 1;
          if (f.sph) {
            to_frame(&f, xb, xl);
            const double r = sqrt((xl[0] * xl[0] + xl[1] * xl[1]) + xl[2] * xl[2]);
            inside = p->d.lo[0] <= r && r <= p->d.hi[0] && r * chi <= xl[2] && xl[2] <= r * clo;
          } else {
            to_local(&f, xb, xl);
            for (int a = 0; a < 3; ++a) inside = inside && (p->d.lo[a] <= xl[a]) && (xl[a] <= p->d.hi[a]);
          }
          if (!inside) continue;
          long c = gidx(g, i, j, k);
          if (owner[c]) {
            rc = fail(s, ORC_ERR_OVERLAP, "local patches %d and %d overlap", owner[c], q);
            break;
          }
          owner[c] = (unsigned char)q;
          cov[c] = 1;
        }
  }
  if (rc) goto done;
  erode(cov, e1, tmp, g->d.n, s->buffer);
  erode(cov, e2, tmp, g->d.n, s->buffer + NG);
  for (long c = 0; c < N; ++c) {
    int st = !e1[c] ? ORC_LIVE : (!e2[c] ? ORC_GHOST : ORC_DEAD);
    if (s->flags_valid && st == ORC_LIVE) {
      int old = s->flags[c] & 3;
      if (old == ORC_GHOST || old == ORC_DEAD) st = ORC_REVIVED;
    }
    s->flags[c] = (unsigned char)(st | (owner[c] << 2));
  }
  s->flags_valid = 1;
  /* poison deactivated cells (Sec. 2.4.2, "poisons the data of fully covered
   * cells"); revive cells that became live: they held interpolated data during
   * the previous step, so u_n there is taken from the local patch at t_n. */
  for (int k = 0; k < g->d.n[2]; ++k)
    for (int j = 0; j < g->d.n[1]; ++j)
      for (int i = 0; i < g->d.n[0]; ++i) {
        unsigned char f = s->flags[gidx(g, i, j, k)];
        long c = at(g, i, j, k);
        if ((f & 3) == ORC_DEAD) {
          g->U[0][c] = NAN;
          g->U[1][c] = NAN;
        } else if ((f & 3) == ORC_REVIVED) {
          int q = f >> 2;
          double xb[3] = {node(g, 0, i), node(g, 1, j), node(g, 2, k)}, x[3], v[2];
          if (q < 1 || q >= s->np) {
            rc = fail(s, ORC_ERR_UNFILLED, "revived cell without owner");
            continue;
          }
          oframe fq = frame_at(&s->p[q], s->t);
          to_local(&fq, xb, x);
          if (interp_point(s, q, s->p[q].U, x, v) != 0) {
            rc = fail(s, ORC_ERR_UNFILLED, "revived cell (%d,%d,%d) not interpolable", i, j, k);
            continue;
          }
          g->U[0][c] = v[0];
          g->U[1][c] = v[1];
        }
      }
done:
  free(owner);
  free(cov);
  free(e1);
  free(e2);
  free(tmp);
  return rc;
}

int orc_get_flags(const orc_sim* s, unsigned char* flags) {
  if (s->np < 1) return ORC_ERR_STATE;
  const opatch* g = &s->p[0];
  memcpy(flags, s->flags, (size_t)g->d.n[0] * g->d.n[1] * g->d.n[2]);
  return 0;
}

int orc_set_flags(orc_sim* s, const unsigned char* flags) {
  if (s->np < 1) return fail(s, ORC_ERR_STATE, "no global patch");
  const opatch* g = &s->p[0];
  memcpy(s->flags, flags, (size_t)g->d.n[0] * g->d.n[1] * g->d.n[2]);
  s->flags_valid = 1;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Stage state Y_l = u_n + dt a_{l,l-1} K_{l-1} on live points (Eqs. k1-k4);
 * every other entry (ghost zones, non-live global cells) is poisoned with NaN
 * so that any read of data not filled by a boundary condition this substage
 * shows up in the result. */
static void make_stage(orc_sim* s, int l, double dt) {
  for (int q = 0; q < s->np; ++q) {
    opatch* p = &s->p[q];
    double coef = dt * RK_A[l];
#pragma omp parallel for schedule(static) num_threads(s->nthreads)
    for (int k = -NG; k < p->d.n[2] + NG; ++k)
      for (int j = -NG; j < p->d.n[1] + NG; ++j)
        for (int i = -NG; i < p->d.n[0] + NG; ++i) {
          long c = at(p, i, j, k);
          for (int f = 0; f < 2; ++f) {
            if (!is_live(s, q, i, j, k))
              p->Y[f][c] = NAN;
            else if (l == 0)
              p->Y[f][c] = p->U[f][c];
            else
              p->Y[f][c] = p->U[f][c] + coef * p->K[l - 1][f][c];
          }
        }
  }
}

static long wrap(int i, int n) { return ((i % n) + n) % n; }

/* Local-to-Global (Sec. 2.4.2): each effective ghost cell of the global
 * patch is mapped into its owning local patch at time t and interpolated
 * there. */
static void fill_l2g(orc_sim* s, double t, const double Xg[3], long* unfilled_, long* bad_donor_) {
  opatch* g = &s->p[0];
  long unfilled = 0, bad_donor = 0;
#pragma omp parallel for schedule(dynamic) reduction(+ : unfilled, bad_donor) num_threads(s->nthreads)
  for (int k = 0; k < g->d.n[2]; ++k)
    for (int j = 0; j < g->d.n[1]; ++j)
      for (int i = 0; i < g->d.n[0]; ++i) {
        unsigned char f = s->flags[gidx(g, i, j, k)];
        if ((f & 3) != ORC_GHOST) continue;
        int q = f >> 2;
        double xb[3] = {node(g, 0, i) + Xg[0], node(g, 1, j) + Xg[1], node(g, 2, k) + Xg[2]}, x[3], v[2];
        oframe fq = frame_at(&s->p[q], t);
        to_local(&fq, xb, x);
        int r = interp_point(s, q, s->p[q].Y, x, v);
        if (r == -1) ++unfilled;
        if (r == -2) ++bad_donor;
        if (r) continue;
        long c = at(g, i, j, k);
        g->Y[0][c] = v[0];
        g->Y[1][c] = v[1];
      }
  *unfilled_ += unfilled;
  *bad_donor_ += bad_donor;
}

/* Global-to-Local (Sec. 2.4.1): each ghost point of a local patch is mapped
 * through the background frame into the global patch at time t and
 * interpolated there. */
static void fill_g2l(orc_sim* s, double t, const double Xg[3], long* unfilled_, long* bad_donor_) {
  opatch* g = &s->p[0];
  long unfilled = 0, bad_donor = 0;
  for (int q = 1; q < s->np; ++q) {
    opatch* p = &s->p[q];
    oframe f = frame_at(p, t);
#pragma omp parallel for schedule(dynamic) reduction(+ : unfilled, bad_donor) num_threads(s->nthreads)
    for (int k = -NG; k < p->d.n[2] + NG; ++k)
      for (int j = -NG; j < p->d.n[1] + NG; ++j)
        for (int i = -NG; i < p->d.n[0] + NG; ++i) {
          if (in_interior(p, i, j, k)) continue;
          if (f.sph && i >= 0 && i < p->d.n[0] && j >= 0 && j < p->d.n[1]) {
            /* azimuthal ghosts of a shell: the periodic image (an intrapatch
             * boundary, the same physical point) */
            long c = at(p, i, j, k), src = at(p, i, j, (int)wrap(k, p->d.n[2]));
            p->Y[0][c] = p->Y[0][src];
            p->Y[1][c] = p->Y[1][src];
            continue;
          }
          double xl[3] = {node(p, 0, i), node(p, 1, j), node(p, 2, k)}, xb[3], x[3], v[2];
          to_background(&f, xl, xb);
          x[0] = xb[0] - Xg[0];
          x[1] = xb[1] - Xg[1];
          x[2] = xb[2] - Xg[2];
          int r = interp_point(s, 0, g->Y, x, v);
          if (r == -1) ++unfilled;
          if (r == -2) ++bad_donor;
          if (r) continue;
          long c = at(p, i, j, k);
          p->Y[0][c] = v[0];
          p->Y[1][c] = v[1];
        }
  }
  *unfilled_ += unfilled;
  *bad_donor_ += bad_donor;
}

/* Boundary data in the paper's order (Sec. 2.4): physical (analytic or
 * periodic) -> interpatch, the interpatch part being Local-to-Global
 * (Sec. 2.4.2) then Global-to-Local (Sec. 2.4.1).  Maps at time t. */
static int fill_bc(orc_sim* s, double t) {
  opatch* g = &s->p[0];
  double Xg[3], wg[3];
  long unfilled = 0, bad_donor = 0;
  orc_motion(g->d.motion, g->d.motion_params, t, Xg, wg);
  /* 1. physical BC on the global outer ghost shell */
#pragma omp parallel for schedule(dynamic) num_threads(s->nthreads)
  for (int k = -NG; k < g->d.n[2] + NG; ++k)
    for (int j = -NG; j < g->d.n[1] + NG; ++j)
      for (int i = -NG; i < g->d.n[0] + NG; ++i) {
        if (in_interior(g, i, j, k)) continue;
        long c = at(g, i, j, k);
        if (g->d.outer_bc == ORC_BC_PERIODIC) {
          long src = at(g, (int)wrap(i, g->d.n[0]), (int)wrap(j, g->d.n[1]), (int)wrap(k, g->d.n[2]));
          g->Y[0][c] = g->Y[0][src];
          g->Y[1][c] = g->Y[1][src];
        } else {
          orc_closed_form(s->akind, s->ap, s->acount, t, node(g, 0, i) + Xg[0], node(g, 1, j) + Xg[1],
                          node(g, 2, k) + Xg[2], &g->Y[0][c], &g->Y[1][c]);
        }
      }
  /* 2./3. interpatch data: Local-to-Global and Global-to-Local */
  if (s->l2g_first) {
    fill_l2g(s, t, Xg, &unfilled, &bad_donor);
    fill_g2l(s, t, Xg, &unfilled, &bad_donor);
  } else {
    fill_g2l(s, t, Xg, &unfilled, &bad_donor);
    fill_l2g(s, t, Xg, &unfilled, &bad_donor);
  }
  if (bad_donor) return fail(s, ORC_ERR_DONOR, "%ld interpolation windows touched non-live cells", bad_donor);
  if (unfilled) return fail(s, ORC_ERR_UNFILLED, "%ld ghost points could not be interpolated", unfilled);
  return 0;
}

int orc_fill_ghosts(orc_sim* s, double t) {
  int rc;
  if (!s->flags_valid && (rc = orc_compute_flags(s)) != 0) return rc;
  make_stage(s, 0, 0.0);
  return fill_bc(s, t);
}

/* ------------------------------------------------------------------------ */
/* Right-hand side (Sec. 2.2, Eqs. eom1-eom3, in a rigidly moving frame with
 * Pi the background-frame time derivative of psi; w is the frame velocity at
 * the point, constant under translation, w(X') = Omega n x X' + R^T V in a
 * rotating frame, where the Laplacian keeps its form because R is
 * orthogonal):
 *   K_psi = Pi + w . D1 psi + KO(psi)
 *   K_Pi  = sum_a D2_a psi + w . D1 Pi + KO(Pi)
 * 4th-order centred differences along each axis with spacing h:
 *   D1 u = (u_{-2} - 8 u_{-1} + 8 u_{+1} - u_{+2}) / (12 h)
 *   D2 u = (-u_{-2} + 16 u_{-1} - 30 u_0 + 16 u_{+1} - u_{+2}) / (12 h^2)
 * Kreiss-Oliger dissipation with n = 5 (Sec. 2.3), per axis
 *   KO u = (eps / 64) (u_{-3} - 6 u_{-2} + 15 u_{-1} - 20 u_0 + 15 u_{+1}
 *                      - 6 u_{+2} + u_{+3}) / h.                           */
static double fd_d1(const double* u, long st, double h) {
  return (u[-2 * st] - 8.0 * u[-st] + 8.0 * u[st] - u[2 * st]) / (12.0 * h);
}
static double fd_d2(const double* u, long st, double h) {
  return (-u[-2 * st] + 16.0 * u[-st] - 30.0 * u[0] + 16.0 * u[st] - u[2 * st]) / (12.0 * h * h);
}
static double fd_ko(const double* u, long st, double h, double eps) {
  return (eps / 64.0) *
         (u[-3 * st] - 6.0 * u[-2 * st] + 15.0 * u[-st] - 20.0 * u[0] + 15.0 * u[st] - 6.0 * u[2 * st] +
          u[3 * st]) /
         h;
}

/* Right-hand side on a spherical shell (the paper's spherical local patch,
 * Sec. 3.3; the flat metric in spherical coordinates of the appendix, with
 * g_phiphi = r^2 sin^2 theta): the same two-field system with
 *   lap u   = u_rr + (2/r) u_r + (u_thth + cot(theta) u_th) / r^2
 *             + u_phph / (r^2 sin^2 theta),
 *   w . D u = w_r u_r + (w_th / r) u_th + (w_ph / (r sin theta)) u_ph,
 * w_r, w_th, w_ph the components of the frame velocity on the unit vectors
 * r^, theta^, phi^, each derivative the 4th-order centred difference along
 * its index axis, and KO per axis over the physical spacing of that axis
 * (h_r, r h_theta, r sin(theta) h_phi). */
static void rhs_shell(orc_sim* s, int q, double t, double* const Y[2], double* Kpsi, double* Kpi) {
  opatch* p = &s->p[q];
  long st[3] = {1, p->m[0], (long)p->m[0] * p->m[1]};
#pragma omp parallel for schedule(static) num_threads(s->nthreads)
  for (int k = 0; k < p->d.n[2]; ++k)
    for (int j = 0; j < p->d.n[1]; ++j)
      for (int i = 0; i < p->d.n[0]; ++i) {
        long c = at(p, i, j, k);
        const double r = node(p, 0, i), th = node(p, 1, j), ph = node(p, 2, k);
        const double sn = sin(th), cs = cos(th), sp = sin(ph), cp = cos(ph);
        const double q3[3] = {r, th, ph};
        double x[3], w[3];
        sph_to_cart(q3, x);
        orc_frame_velocity(p->d.motion, p->d.motion_params, t, x, w);
        const double wr = w[0] * sn * cp + w[1] * sn * sp + w[2] * cs;
        const double wt = w[0] * cs * cp + w[1] * cs * sp - w[2] * sn;
        const double wp = -w[0] * sp + w[1] * cp;
        double K[2];
        for (int f = 0; f < 2; ++f) {
          const double* u = Y[f] + c;
          const double ur = fd_d1(u, st[0], p->h[0]), ut = fd_d1(u, st[1], p->h[1]), up = fd_d1(u, st[2], p->h[2]);
          const double adv = wr * ur + (wt / r) * ut + (wp / (r * sn)) * up;
          const double ko = fd_ko(u, st[0], p->h[0], s->eps) + fd_ko(u, st[1], r * p->h[1], s->eps) +
                            fd_ko(u, st[2], r * sn * p->h[2], s->eps);
          K[f] = adv + ko;
        }
        const double* ps = Y[0] + c;
        const double lap = fd_d2(ps, st[0], p->h[0]) + (2.0 / r) * fd_d1(ps, st[0], p->h[0]) +
                           (fd_d2(ps, st[1], p->h[1]) + (cs / sn) * fd_d1(ps, st[1], p->h[1])) / (r * r) +
                           fd_d2(ps, st[2], p->h[2]) / (r * r * sn * sn);
        Kpsi[c] = Y[1][c] + K[0];
        Kpi[c] = lap + K[1];
      }
}

static void rhs(orc_sim* s, int q, double t, double* const Y[2], double* Kpsi, double* Kpi) {
  opatch* p = &s->p[q];
  if (p->d.topology == ORC_SPHERICAL) {
    rhs_shell(s, q, t, Y, Kpsi, Kpi);
    return;
  }
  double X0[3], w0[3];
  orc_motion(p->d.motion, p->d.motion_params, t, X0, w0);
  const int rot = p->d.motion == ORC_ROTATING;
  long st[3] = {1, p->m[0], (long)p->m[0] * p->m[1]};
#pragma omp parallel for schedule(static) num_threads(s->nthreads)
  for (int k = 0; k < p->d.n[2]; ++k)
    for (int j = 0; j < p->d.n[1]; ++j)
      for (int i = 0; i < p->d.n[0]; ++i) {
        long c = at(p, i, j, k);
        if (!is_live(s, q, i, j, k)) {
          Kpsi[c] = NAN;
          Kpi[c] = NAN;
          continue;
        }
        const double* ps = Y[0] + c;
        const double* pv = Y[1] + c;
        double w[3] = {w0[0], w0[1], w0[2]};
        if (rot) {
          const double xl[3] = {node(p, 0, i), node(p, 1, j), node(p, 2, k)};
          orc_frame_velocity(p->d.motion, p->d.motion_params, t, xl, w);
        }
        double kps = pv[0], kpi = 0.0;
        for (int a = 0; a < 3; ++a) {
          kps += w[a] * fd_d1(ps, st[a], p->h[a]) + fd_ko(ps, st[a], p->h[a], s->eps);
          kpi += fd_d2(ps, st[a], p->h[a]) + w[a] * fd_d1(pv, st[a], p->h[a]) + fd_ko(pv, st[a], p->h[a], s->eps);
        }
        Kpsi[c] = kps;
        Kpi[c] = kpi;
      }
}

int orc_eval_rhs(orc_sim* s, int q, double t, double* kpsi, double* kpi) {
  if (q < 0 || q >= s->np) return fail(s, ORC_ERR_ARG, "bad patch id");
  opatch* p = &s->p[q];
  rhs(s, q, t, p->U, p->K[0][0], p->K[0][1]);
  long c = 0;
  for (int k = 0; k < p->d.n[2]; ++k)
    for (int j = 0; j < p->d.n[1]; ++j)
      for (int i = 0; i < p->d.n[0]; ++i, ++c) {
        kpsi[c] = p->K[0][0][at(p, i, j, k)];
        kpi[c] = p->K[0][1][at(p, i, j, k)];
      }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* One full RK4 step per iteration (Sec. 2.3):
 *   flags at t_n (held for the step), then K_1..K_4 with boundary data laid
 *   down before each slope, then u_{n+1/2} = u_n + dt (b1 K1 + b2 K2 + b3 K3)
 *   and u_{n+1} = u_{n+1/2} + dt b4 K4 on live points. */
int orc_step(orc_sim* s, double dt, int nsteps) {
  if (s->np < 1) return fail(s, ORC_ERR_STATE, "no global patch");
  for (int n = 0; n < nsteps; ++n) {
    double tn = s->t;
    int rc = orc_compute_flags(s);
    if (rc) return rc;
    for (int l = 0; l < 4; ++l) {
      double tl = tn + RK_C[l] * dt;
      make_stage(s, l, dt);
      if ((rc = fill_bc(s, tl)) != 0) return rc;
      for (int q = 0; q < s->np; ++q) rhs(s, q, tl, s->p[q].Y, s->p[q].K[l][0], s->p[q].K[l][1]);
    }
    for (int q = 0; q < s->np; ++q) {
      opatch* p = &s->p[q];
#pragma omp parallel for schedule(static) num_threads(s->nthreads)
      for (int k = 0; k < p->d.n[2]; ++k)
        for (int j = 0; j < p->d.n[1]; ++j)
          for (int i = 0; i < p->d.n[0]; ++i) {
            if (!is_live(s, q, i, j, k)) continue;
            long c = at(p, i, j, k);
            for (int f = 0; f < 2; ++f) {
              double half = p->U[f][c] + dt * (RK_B[0] * p->K[0][f][c] + RK_B[1] * p->K[1][f][c] +
                                               RK_B[2] * p->K[2][f][c]);
              p->U[f][c] = half + dt * RK_B[3] * p->K[3][f][c];
            }
          }
    }
    s->t = tn + dt;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Pieces of a hybrid step, in which the global patch is advanced by other
 * means (a learned surrogate) and only the local patches take the method's
 * RK4 step.  Not part of the paper's method: the surrogate is an extension of
 * it, and these two functions lay out what that extension prescribes, so
 * that the library's hybrid path has an oracle. */

/* Every DEAD global cell (flags as last computed) of the stage state Y takes
 * the Lagrange interpolant, Eq. (Pijk), of the u of the local patch that
 * covers it, mapped at time t: a complete global field for the surrogate
 * (dead cells take no part in the method itself). */
int orc_fill_dead(orc_sim* s, double t) {
  if (s->np < 1 || !s->flags_valid) return fail(s, ORC_ERR_STATE, "no flags");
  opatch* g = &s->p[0];
  double Xg[3], wg[3];
  long unfilled = 0;
  orc_motion(g->d.motion, g->d.motion_params, t, Xg, wg);
#pragma omp parallel for schedule(dynamic) reduction(+ : unfilled) num_threads(s->nthreads)
  for (int k = 0; k < g->d.n[2]; ++k)
    for (int j = 0; j < g->d.n[1]; ++j)
      for (int i = 0; i < g->d.n[0]; ++i) {
        unsigned char f = s->flags[gidx(g, i, j, k)];
        if ((f & 3) != ORC_DEAD) continue;
        int q = f >> 2;
        double xb[3] = {node(g, 0, i) + Xg[0], node(g, 1, j) + Xg[1], node(g, 2, k) + Xg[2]}, x[3], v[2];
        oframe fq = frame_at(&s->p[q], t);
        to_local(&fq, xb, x);
        if (interp_point(s, q, s->p[q].U, x, v)) {
          ++unfilled;
          continue;
        }
        long c = at(g, i, j, k);
        g->Y[0][c] = v[0];
        g->Y[1][c] = v[1];
      }
  if (unfilled) return fail(s, ORC_ERR_UNFILLED, "%ld dead cells could not be interpolated", unfilled);
  return 0;
}

/* One RK4 step of the local patches only (Sec. 2.3, Table 1) while the global
 * patch holds, at substage l, the prescribed stage state gstage[2 l + f]
 * (field f, interior points in (k, j, i) order): flags at t_n, then per
 * substage the local stage states, the global's prescribed one (its outer
 * shell by periodic images), Global-to-Local ghost data (Sec. 2.4.1) at t_l
 * and the local slopes; then the local updates.  The global's u is left as
 * it was; t advances by dt. */
int orc_step_locals(orc_sim* s, double dt, const double* const* gstage) {
  if (s->np < 1) return fail(s, ORC_ERR_STATE, "no global patch");
  opatch* g = &s->p[0];
  if (g->d.outer_bc != ORC_BC_PERIODIC) return fail(s, ORC_ERR_ARG, "the global patch must be periodic");
  double tn = s->t;
  int rc = orc_compute_flags(s);
  if (rc) return rc;
  for (int l = 0; l < 4; ++l) {
    double tl = tn + RK_C[l] * dt, Xg[3], wg[3];
    long unfilled = 0, bad_donor = 0;
    make_stage(s, l, dt);
    long c = 0;
    for (int k = 0; k < g->d.n[2]; ++k)
      for (int j = 0; j < g->d.n[1]; ++j)
        for (int i = 0; i < g->d.n[0]; ++i, ++c) {
          g->Y[0][at(g, i, j, k)] = gstage[2 * l][c];
          g->Y[1][at(g, i, j, k)] = gstage[2 * l + 1][c];
        }
    for (int k = -NG; k < g->d.n[2] + NG; ++k)
      for (int j = -NG; j < g->d.n[1] + NG; ++j)
        for (int i = -NG; i < g->d.n[0] + NG; ++i) {
          if (in_interior(g, i, j, k)) continue;
          long d = at(g, i, j, k), src = at(g, (int)wrap(i, g->d.n[0]), (int)wrap(j, g->d.n[1]), (int)wrap(k, g->d.n[2]));
          g->Y[0][d] = g->Y[0][src];
          g->Y[1][d] = g->Y[1][src];
        }
    orc_motion(g->d.motion, g->d.motion_params, tl, Xg, wg);
    fill_g2l(s, tl, Xg, &unfilled, &bad_donor);
    if (bad_donor) return fail(s, ORC_ERR_DONOR, "%ld interpolation windows touched non-live cells", bad_donor);
    if (unfilled) return fail(s, ORC_ERR_UNFILLED, "%ld ghost points could not be interpolated", unfilled);
    for (int q = 1; q < s->np; ++q) rhs(s, q, tl, s->p[q].Y, s->p[q].K[l][0], s->p[q].K[l][1]);
  }
  for (int q = 1; q < s->np; ++q) {
    opatch* p = &s->p[q];
    for (int k = 0; k < p->d.n[2]; ++k)
      for (int j = 0; j < p->d.n[1]; ++j)
        for (int i = 0; i < p->d.n[0]; ++i) {
          long c = at(p, i, j, k);
          for (int f = 0; f < 2; ++f) {
            double half = p->U[f][c] + dt * (RK_B[0] * p->K[0][f][c] + RK_B[1] * p->K[1][f][c] +
                                             RK_B[2] * p->K[2][f][c]);
            p->U[f][c] = half + dt * RK_B[3] * p->K[3][f][c];
          }
        }
  }
  s->t = tn + dt;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Discrete energy of a periodic patch, E_h = 1/2 h^3 sum (Pi^2 - psi D2 psi),
 * with D2 the 3-axis operator above and periodic neighbours. */
double orc_energy(const orc_sim* s, int q) {
  const opatch* p = &s->p[q];
  const int* n = p->d.n;
  double e = 0.0;
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        double u0 = p->U[0][at(p, i, j, k)], pv = p->U[1][at(p, i, j, k)], lap = 0.0;
        for (int a = 0; a < 3; ++a) {
          double v[5];
          for (int o = -2; o <= 2; ++o) {
            int ii = i, jj = j, kk = k;
            if (a == 0) ii = (int)wrap(i + o, n[0]);
            if (a == 1) jj = (int)wrap(j + o, n[1]);
            if (a == 2) kk = (int)wrap(k + o, n[2]);
            v[o + 2] = p->U[0][at(p, ii, jj, kk)];
          }
          lap += (-v[0] + 16.0 * v[1] - 30.0 * v[2] + 16.0 * v[3] - v[4]) / (12.0 * p->h[a] * p->h[a]);
        }
        e += pv * pv - u0 * lap;
      }
  return 0.5 * p->h[0] * p->h[1] * p->h[2] * e;
}
