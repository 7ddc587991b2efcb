"""ctypes wrapper of the C oracle (test infrastructure only; see oracle/__init__.py)."""
import ctypes as C

import numpy as np

from . import LIB_PATH, build_oracle

GLOBAL, LOCAL = 0, 1
CARTESIAN, SPHERICAL = 0, 1
BC_ANALYTIC, BC_PERIODIC, BC_INTERPATCH = 0, 1, 2
STATIC, LINEAR, CIRCULAR, ROTATING = 0, 1, 2, 3
GAUSS_SUM, PLANE_SUM, HARMONIC_POLY, PLANE_GAUSS = 0, 1, 2, 3
LIVE, GHOST, DEAD, REVIVED = 0, 1, 2, 3
NG = 3


class PatchDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("outer_bc", C.c_int), ("motion", C.c_int), ("motion_params", C.c_double * 16),
                ("topology", C.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build_oracle()
        L = C.CDLL(LIB_PATH)
        dp = C.POINTER(C.c_double)
        vp = C.c_void_p
        L.orc_create.restype = vp
        L.orc_create.argtypes = [C.c_int, C.c_double, C.c_int]
        L.orc_destroy.argtypes = [vp]
        L.orc_error.restype = C.c_char_p
        L.orc_error.argtypes = [vp]
        L.orc_add_patch.argtypes = [vp, C.POINTER(PatchDesc)]
        L.orc_set_analytic.argtypes = [vp, C.c_int, dp, C.c_int]
        L.orc_fill_analytic.argtypes = [vp, C.c_double]
        L.orc_set_fields.argtypes = [vp, C.c_int, dp, dp]
        L.orc_get_fields.argtypes = [vp, C.c_int, dp, dp]
        L.orc_set_padded.argtypes = [vp, C.c_int, C.c_int, dp, dp]
        L.orc_get_padded.argtypes = [vp, C.c_int, C.c_int, dp, dp]
        L.orc_set_time.argtypes = [vp, C.c_double]
        L.orc_time.restype = C.c_double
        L.orc_time.argtypes = [vp]
        L.orc_set_threads.argtypes = [vp, C.c_int]
        L.orc_set_fill_order.argtypes = [vp, C.c_int]
        L.orc_compute_flags.argtypes = [vp]
        L.orc_get_flags.argtypes = [vp, C.POINTER(C.c_ubyte)]
        L.orc_set_flags.argtypes = [vp, C.POINTER(C.c_ubyte)]
        L.orc_fill_ghosts.argtypes = [vp, C.c_double]
        L.orc_eval_rhs.argtypes = [vp, C.c_int, C.c_double, dp, dp]
        L.orc_step.argtypes = [vp, C.c_double, C.c_int]
        L.orc_fill_dead.argtypes = [vp, C.c_double]
        L.orc_step_locals.argtypes = [vp, C.c_double, C.POINTER(dp)]
        L.orc_live_points.restype = C.c_long
        L.orc_live_points.argtypes = [vp]
        L.orc_energy.restype = C.c_double
        L.orc_energy.argtypes = [vp, C.c_int]
        L.orc_motion.argtypes = [C.c_int, dp, C.c_double, dp, dp]
        L.orc_frame.argtypes = [C.c_int, dp, C.c_double, dp, dp]
        L.orc_frame_velocity.argtypes = [C.c_int, dp, C.c_double, dp, dp]
        L.orc_lagrange.restype = C.c_int
        L.orc_lagrange.argtypes = [C.c_int, C.c_double, dp]
        L.orc_closed_form.argtypes = [C.c_int, dp, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, dp, dp]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_desc(kind, n, lo, hi, outer_bc, motion=STATIC, motion_params=(), topology=CARTESIAN):
    d = PatchDesc()
    d.topology = topology
    d.kind = kind
    for a in range(3):
        d.n[a] = int(n[a])
        d.lo[a] = float(lo[a])
        d.hi[a] = float(hi[a])
    d.outer_bc = outer_bc
    d.motion = motion
    for i, v in enumerate(motion_params):
        d.motion_params[i] = float(v)
    return d


def motion(kind, params, t):
    p = np.zeros(16)
    p[:len(params)] = params
    X0 = np.zeros(3)
    w = np.zeros(3)
    lib().orc_motion(kind, _dp(p), float(t), _dp(X0), _dp(w))
    return X0, w


def frame(kind, params, t):
    """(R, X0) of the patch map X_B = R X' + X0 at time t."""
    p = np.zeros(16)
    p[:len(params)] = params
    R = np.zeros(9)
    X0 = np.zeros(3)
    lib().orc_frame(kind, _dp(p), float(t), _dp(R), _dp(X0))
    return R.reshape(3, 3), X0


def frame_velocity(kind, params, t, xl):
    """Frame velocity (patch components) at the patch point xl."""
    p = np.zeros(16)
    p[:len(params)] = params
    x = np.ascontiguousarray(xl, dtype=np.float64)
    w = np.zeros(3)
    lib().orc_frame_velocity(kind, _dp(p), float(t), _dp(x), _dp(w))
    return w


def lagrange(P, s):
    w = np.zeros(P)
    start = lib().orc_lagrange(P, float(s), _dp(w))
    return start, w


def closed_form(kind, params, count, t, x, y, z):
    """Vectorised over x, y, z (broadcast); returns (psi, pi)."""
    prm = np.ascontiguousarray(params, dtype=np.float64)
    x, y, z = np.broadcast_arrays(np.asarray(x, float), np.asarray(y, float), np.asarray(z, float))
    ps = np.empty(x.shape)
    pv = np.empty(x.shape)
    a, b = C.c_double(), C.c_double()
    L = lib()
    for idx in np.ndindex(x.shape):
        L.orc_closed_form(kind, _dp(prm), count, float(t), float(x[idx]), float(y[idx]), float(z[idx]),
                          C.byref(a), C.byref(b))
        ps[idx] = a.value
        pv[idx] = b.value
    return ps, pv


class OracleError(RuntimeError):
    pass


class Oracle:
    """One multipatch simulation held by the C oracle."""

    def __init__(self, interp_points=6, ko_eps=0.005, buffer=NG + 1, threads=1):
        self.L = lib()
        self.h = self.L.orc_create(interp_points, ko_eps, buffer)
        if not self.h:
            raise OracleError("orc_create failed")
        self.L.orc_set_threads(self.h, threads)
        self.patches = []

    def close(self):
        if self.h:
            self.L.orc_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def _check(self, rc):
        if rc < 0:
            raise OracleError(f"oracle error {rc}: {self.L.orc_error(self.h).decode()}")
        return rc

    def add_patch(self, kind, n, lo, hi, outer_bc, motion=STATIC, motion_params=(), topology=CARTESIAN):
        d = make_desc(kind, n, lo, hi, outer_bc, motion, motion_params, topology)
        pid = self._check(self.L.orc_add_patch(self.h, C.byref(d)))
        self.patches.append(tuple(int(v) for v in n))
        return pid

    def set_analytic(self, kind, params, count):
        p = np.ascontiguousarray(params, dtype=np.float64)
        self._check(self.L.orc_set_analytic(self.h, kind, _dp(p), count))

    def fill_analytic(self, t):
        self._check(self.L.orc_fill_analytic(self.h, float(t)))

    def shape(self, pid):
        n = self.patches[pid]
        return (n[2], n[1], n[0])

    def padded_shape(self, pid):
        n = self.patches[pid]
        return (n[2] + 2 * NG, n[1] + 2 * NG, n[0] + 2 * NG)

    def set_fields(self, pid, psi, pi):
        psi = np.ascontiguousarray(psi, dtype=np.float64).reshape(self.shape(pid))
        pi = np.ascontiguousarray(pi, dtype=np.float64).reshape(self.shape(pid))
        self._check(self.L.orc_set_fields(self.h, pid, _dp(psi), _dp(pi)))

    def get_fields(self, pid):
        psi = np.empty(self.shape(pid))
        pi = np.empty(self.shape(pid))
        self._check(self.L.orc_get_fields(self.h, pid, _dp(psi), _dp(pi)))
        return psi, pi

    def set_padded(self, pid, psi, pi, which=0):
        psi = np.ascontiguousarray(psi, dtype=np.float64).reshape(self.padded_shape(pid))
        pi = np.ascontiguousarray(pi, dtype=np.float64).reshape(self.padded_shape(pid))
        self._check(self.L.orc_set_padded(self.h, pid, which, _dp(psi), _dp(pi)))

    def get_padded(self, pid, which=0):
        psi = np.empty(self.padded_shape(pid))
        pi = np.empty(self.padded_shape(pid))
        self._check(self.L.orc_get_padded(self.h, pid, which, _dp(psi), _dp(pi)))
        return psi, pi

    @property
    def time(self):
        return self.L.orc_time(self.h)

    @time.setter
    def time(self, t):
        self.L.orc_set_time(self.h, float(t))

    def set_fill_order(self, l2g_first):
        self.L.orc_set_fill_order(self.h, 1 if l2g_first else 0)

    def compute_flags(self):
        self._check(self.L.orc_compute_flags(self.h))

    def get_flags(self):
        f = np.empty(self.shape(0), dtype=np.uint8)
        self._check(self.L.orc_get_flags(self.h, f.ctypes.data_as(C.POINTER(C.c_ubyte))))
        return f

    def set_flags(self, flags):
        f = np.ascontiguousarray(flags, dtype=np.uint8).reshape(self.shape(0))
        self._check(self.L.orc_set_flags(self.h, f.ctypes.data_as(C.POINTER(C.c_ubyte))))

    def fill_ghosts(self, t):
        self._check(self.L.orc_fill_ghosts(self.h, float(t)))

    def eval_rhs(self, pid, t):
        kps = np.empty(self.shape(pid))
        kpi = np.empty(self.shape(pid))
        self._check(self.L.orc_eval_rhs(self.h, pid, float(t), _dp(kps), _dp(kpi)))
        return kps, kpi

    def step(self, dt, nsteps=1):
        self._check(self.L.orc_step(self.h, float(dt), int(nsteps)))

    def fill_dead(self, t):
        """Dead global cells of the stage state from their local patch (the
        complete field a learned surrogate reads)."""
        self._check(self.L.orc_fill_dead(self.h, float(t)))

    def step_locals(self, dt, gstage):
        """One RK4 step of the local patches, the global's stage states
        prescribed: gstage[l] = (psi, pi) interior arrays of substage l."""
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for l in range(4) for a in gstage[l]]
        n = self.shape(0)
        for a in arrs:
            if a.shape != tuple(n):
                raise ValueError("stage arrays must have the global patch's interior shape")
        ptrs = (C.POINTER(C.c_double) * 8)(*[_dp(a) for a in arrs])
        self._check(self.L.orc_step_locals(self.h, float(dt), ptrs))

    def live_points(self):
        return self.L.orc_live_points(self.h)

    def energy(self, pid=0):
        return self.L.orc_energy(self.h, pid)
