"""Thin ctypes binding of libmpw (include/mpw.h, include/mpw_surrogate.h).

Argument marshalling only: every step of the method runs in the CUDA kernels
of libmpw.so.  PyTorch supplies device memory (through the allocator hook
bound to its caching allocator), the stream and, for the tests and the
benchmark, device tensors.  There is no CPU fallback: if libmpw.so is missing
or cannot be loaded, importing this module raises.
"""
import ctypes as C
import os

import numpy as np

from .build import LIB_PATH

# enums of include/mpw.h
MPW_OK = 0
STATUS_NAMES = {0: "MPW_OK", 1: "MPW_ERR_ARG", 2: "MPW_ERR_OVERLAP", 3: "MPW_ERR_CFL", 4: "MPW_ERR_TRAVERSAL",
                5: "MPW_ERR_OUTSIDE", 6: "MPW_ERR_GHOST_UNFILLED", 8: "MPW_ERR_TIMEOUT", 9: "MPW_ERR_CUDA",
                10: "MPW_ERR_STATE"}
ERR_ARG, ERR_CFL, ERR_GHOST_UNFILLED, ERR_TIMEOUT, ERR_CUDA = 1, 3, 6, 8, 9
PATCH_GLOBAL, PATCH_LOCAL = 0, 1
BC_ANALYTIC, BC_PERIODIC, BC_INTERPATCH = 0, 1, 2
MOTION_STATIC, MOTION_LINEAR, MOTION_CIRCULAR, MOTION_ROTATING = 0, 1, 2, 3
TOPOLOGY_CARTESIAN, TOPOLOGY_SPHERICAL = 0, 1
ANALYTIC_GAUSS_SUM, ANALYTIC_PLANE_SUM, ANALYTIC_HARMONIC_POLY, ANALYTIC_PLANE_GAUSS = 0, 1, 2, 3
FLAG_LIVE, FLAG_GHOST, FLAG_DEAD, FLAG_REVIVED = 0, 1, 2, 3
NG = 3

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class mpw_config(C.Structure):
    _fields_ = [("precision", C.c_int), ("ghost", C.c_int), ("interp_points", C.c_int), ("ko_eps", C.c_double),
                ("buffer", C.c_int), ("device", C.c_int), ("stream", C.c_void_p), ("alloc", ALLOC_FN),
                ("free", FREE_FN), ("alloc_user", C.c_void_p), ("arith", C.c_int)]


class mpw_patch_desc(C.Structure):
    _fields_ = [("kind", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("outer_bc", C.c_int), ("motion", C.c_int), ("motion_params", C.c_double * 16),
                ("topology", C.c_int)]


# Every symbol that include/mpw.h declares, with its ctypes signature.
_dp = C.POINTER(C.c_double)
_vp = C.c_void_p
SIGNATURES = {
    "mpw_create": (C.c_int, [C.POINTER(mpw_config), C.POINTER(C.c_void_p)]),
    "mpw_create_patch": (C.c_int, [_vp, C.POINTER(mpw_patch_desc), C.POINTER(C.c_int)]),
    "mpw_set_analytic": (C.c_int, [_vp, C.c_int, _dp, C.c_int]),
    "mpw_fill_analytic": (C.c_int, [_vp, C.c_double]),
    "mpw_set_fields": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_int]),
    "mpw_get_fields": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_int]),
    "mpw_get_padded": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_int]),
    "mpw_set_time": (C.c_int, [_vp, C.c_double]),
    "mpw_time": (C.c_double, [_vp]),
    "mpw_compute_flags": (C.c_int, [_vp]),
    "mpw_get_flags": (C.c_int, [_vp, _vp]),
    "mpw_set_flags": (C.c_int, [_vp, _vp]),
    "mpw_fill_ghosts": (C.c_int, [_vp, C.c_double]),
    "mpw_set_wait_limit": (C.c_int, [_vp, C.c_uint]),
    "mpw_step": (C.c_int, [_vp, C.c_double, C.c_int]),
    "mpw_live_points": (C.c_int, [_vp, C.POINTER(C.c_longlong)]),
    "mpw_profile_enable": (C.c_int, [_vp, C.c_int]),
    "mpw_profile_read": (C.c_int, [_vp, _dp, C.POINTER(C.c_longlong), C.c_int]),
    "mpw_step_periodic_noalloc": (C.c_int, [C.POINTER(C.c_int), _dp, _dp, C.c_double, C.c_double, C.c_int, _vp, _vp,
                                            _vp]),
    "mpw_step_async": (C.c_int, [_vp, C.c_double, C.c_int]),
    "mpw_set_fields_async": (C.c_int, [_vp, C.c_int, _vp, _vp]),
    "mpw_get_fields_async": (C.c_int, [_vp, C.c_int, _vp, _vp]),
    "mpw_sync": (C.c_int, [_vp]),
    "mpw_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_void_p)]),
    "mpw_batch_step": (C.c_int, [_vp, _dp, C.c_int]),
    "mpw_batch_tuning": (C.c_int, [_vp, C.POINTER(C.c_int), _dp, C.POINTER(C.c_longlong),
                                   C.POINTER(C.c_longlong)]),
    "mpw_batch_destroy": (None, [_vp]),
    "mpw_last_error": (C.c_char_p, []),
    # include/mpw_surrogate.h
    "mpw_conv3_forward": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_int, C.c_int, C.POINTER(C.c_int), C.c_int, _vp, _vp,
                                    _vp, _vp]),
    "mpw_conv3_backward_data": (C.c_int, [_vp, C.c_int, _vp, C.c_int, C.c_int, C.POINTER(C.c_int), _vp, _vp, _vp,
                                          _vp]),
    "mpw_conv3_wgrad_scratch_bytes": (C.c_size_t, [C.c_int, C.c_int]),
    "mpw_conv3_select": (C.c_int, [C.c_int]),
    "mpw_conv3_backward_weights": (C.c_int, [_vp, C.c_int, _vp, C.c_int, C.c_int, C.POINTER(C.c_int), _vp, _vp, _vp,
                                             C.c_size_t, _vp]),
    "mpw_adam_step": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.c_longlong, C.c_float, C.c_float, C.c_float, C.c_float,
                                C.c_int, _vp]),
    "mpw_mse_grad": (C.c_int, [_vp, C.c_int, _vp, C.c_int, C.c_longlong, _vp, _vp, _vp]),
    "mpw_sur_param_count": (C.c_longlong, []),
    "mpw_sur_create": (C.c_int, [C.c_int, _vp, C.c_double, C.c_double, C.c_double, C.POINTER(C.c_void_p)]),
    "mpw_sur_destroy": (None, [_vp]),
    "mpw_sur_set_params": (C.c_int, [_vp, _vp, C.c_longlong]),
    "mpw_sur_get_params": (C.c_int, [_vp, _vp, C.c_longlong]),
    "mpw_sur_get_grads": (C.c_int, [_vp, _vp, C.c_longlong]),
    "mpw_sur_features": (C.c_int, [_vp, _vp, _vp, C.c_int, C.POINTER(C.c_int), _vp, _vp]),
    "mpw_sur_targets": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.c_int, C.POINTER(C.c_int), _vp, _vp]),
    "mpw_sur_train_step": (C.c_int, [_vp, _vp, _vp, C.c_int, C.POINTER(C.c_int), C.c_float, _dp]),
    "mpw_sur_forward": (C.c_int, [_vp, _vp, C.c_int, C.POINTER(C.c_int), _vp]),
    "mpw_sur_predict": (C.c_int, [_vp, _vp, _vp, C.c_int, C.POINTER(C.c_int), _vp, _vp]),
    "mpw_sur_check": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.c_int, C.POINTER(C.c_int), _vp, _vp]),
    "mpw_step_surrogate": (C.c_int, [_vp, _vp, C.c_double, C.c_int, C.c_double, C.POINTER(C.c_int), _dp]),
    "mpw_sur_stage_weights": (C.c_int, [C.c_int, C.c_int, C.c_double, _dp]),
    "mpw_destroy": (None, [_vp]),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_2002_00088_gb300.build.build_library() "
                          "(or __graft_entry__.build()) first; there is no fallback path")
    L = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


lib = _load()


NOALLOC_MAX_N = 48


def check_noalloc_fields(n, psi, pi):
    """Raise ValueError unless psi and pi are C-contiguous float64 CUDA tensors
    of shape (n2, n1, n0) on the current device: the kernels read and write
    exactly that many values through the raw pointers."""
    torch = _torch()
    want = (int(n[2]), int(n[1]), int(n[0]))
    for name, a in (("psi", psi), ("pi", pi)):
        if not isinstance(a, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor")
        if tuple(a.shape) != want:
            raise ValueError(f"{name} has shape {tuple(a.shape)}, expected (n2, n1, n0) = {want}")
        if a.dtype != torch.float64:
            raise ValueError(f"{name} must be float64, not {a.dtype}")
        if not a.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    for name, a in (("psi", psi), ("pi", pi)):
        if not a.is_cuda or a.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} must live on the current CUDA device")


def step_periodic_noalloc(n, lo, hi, ko_eps, dt, nsteps, psi, pi, stream=None):
    """mpw_step_periodic_noalloc on two CUDA float64 tensors of shape (n2, n1, n0),
    advanced in place; nothing is allocated by the library.  Returns once the
    work has finished on the stream."""
    check_noalloc_fields(n, psi, pi)
    nn = (C.c_int * 3)(*[int(v) for v in n])
    lo_ = (C.c_double * 3)(*[float(v) for v in lo])
    hi_ = (C.c_double * 3)(*[float(v) for v in hi])
    s = None if stream is None else C.c_void_p(stream.cuda_stream)
    check(lib.mpw_step_periodic_noalloc(nn, lo_, hi_, float(ko_eps), float(dt), int(nsteps),
                                        C.c_void_p(psi.data_ptr()), C.c_void_p(pi.data_ptr()), s))


class MpwError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status):
    if status != MPW_OK:
        raise MpwError(status, lib.mpw_last_error().decode())
    return status


def _torch():
    import torch
    return torch


class Multipatch:
    """One multipatch simulation on one GPU (owns an mpw_ctx).

    Device storage comes from PyTorch's caching allocator through the
    mpw_config allocator hook; work is enqueued on the current torch stream.
    """

    def __init__(self, interp_points=6, ko_eps=0.005, buffer=0, device=0, stream=None, arith=0, precision=64):
        torch = _torch()
        self.device = device
        self._torch = torch
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream

        def _alloc(nbytes, user):
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, self.stream)

        def _free(ptr, user):
            torch.cuda.caching_allocator_delete(ptr)

        self._alloc_cb = ALLOC_FN(_alloc)
        self._free_cb = FREE_FN(_free)
        self.precision = precision
        cfg = mpw_config(precision=precision, ghost=NG, interp_points=interp_points, ko_eps=ko_eps, buffer=buffer,
                         device=device, stream=C.c_void_p(stream.cuda_stream), alloc=self._alloc_cb,
                         free=self._free_cb, alloc_user=None, arith=arith)
        self.h = C.c_void_p()
        check(lib.mpw_create(C.byref(cfg), C.byref(self.h)))
        self.shapes = []

    def close(self):
        if self.h:
            lib.mpw_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- setup --------------------------------------------------------------
    def create_patch(self, kind, n, lo, hi, outer_bc, motion=MOTION_STATIC, motion_params=(),
                     topology=TOPOLOGY_CARTESIAN):
        d = mpw_patch_desc()
        d.kind = kind
        d.topology = topology
        for a in range(3):
            d.n[a] = int(n[a])
            d.lo[a] = float(lo[a])
            d.hi[a] = float(hi[a])
        d.outer_bc = outer_bc
        d.motion = motion
        for i, v in enumerate(motion_params):
            d.motion_params[i] = float(v)
        pid = C.c_int()
        check(lib.mpw_create_patch(self.h, C.byref(d), C.byref(pid)))
        self.shapes.append((int(n[2]), int(n[1]), int(n[0])))
        return pid.value

    def set_analytic(self, kind, params, count):
        p = np.ascontiguousarray(params, dtype=np.float64)
        check(lib.mpw_set_analytic(self.h, kind, p.ctypes.data_as(_dp), count))

    def fill_analytic(self, t):
        check(lib.mpw_fill_analytic(self.h, float(t)))

    # -- fields -------------------------------------------------------------
    def set_fields(self, pid, psi, pi):
        """psi, pi: numpy arrays (host) or torch CUDA tensors, shape (n2, n1, n0) float64."""
        torch = self._torch
        if isinstance(psi, torch.Tensor) and psi.is_cuda:
            psi = psi.contiguous()
            pi = pi.contiguous()
            assert psi.dtype == torch.float64 and pi.dtype == torch.float64
            check(lib.mpw_set_fields(self.h, pid, C.c_void_p(psi.data_ptr()), C.c_void_p(pi.data_ptr()), 1))
        else:
            psi = np.ascontiguousarray(psi, dtype=np.float64)
            pi = np.ascontiguousarray(pi, dtype=np.float64)
            check(lib.mpw_set_fields(self.h, pid, psi.ctypes.data_as(_vp), pi.ctypes.data_as(_vp), 0))

    def get_fields(self, pid, out=None):
        """Returns host numpy arrays, or fills the given pair of CUDA tensors or
        C-contiguous float64 host arrays (page-locked ones are written in place
        by the pack kernel)."""
        if out is not None:
            psi, pi = out
            if isinstance(psi, self._torch.Tensor) and psi.is_cuda:
                check(lib.mpw_get_fields(self.h, pid, C.c_void_p(psi.data_ptr()), C.c_void_p(pi.data_ptr()), 1))
                return psi, pi
            for a in (psi, pi):
                if a.dtype != np.float64 or not a.flags.c_contiguous or a.shape != tuple(self.shapes[pid]):
                    raise ValueError("host output arrays must be C-contiguous float64 of the patch shape")
            check(lib.mpw_get_fields(self.h, pid, psi.ctypes.data_as(_vp), pi.ctypes.data_as(_vp), 0))
            return psi, pi
        psi = np.empty(self.shapes[pid])
        pi = np.empty(self.shapes[pid])
        check(lib.mpw_get_fields(self.h, pid, psi.ctypes.data_as(_vp), pi.ctypes.data_as(_vp), 0))
        return psi, pi

    def set_fields_async(self, pid, psi, pi):
        """Queue page-locked host arrays (C-contiguous float64, patch shape) as the
        new interior; they enter u at the next call that uses u.  Keep them
        unchanged until sync()."""
        self._check_host(pid, psi, pi)
        check(lib.mpw_set_fields_async(self.h, pid, psi.ctypes.data_as(_vp), pi.ctypes.data_as(_vp)))

    def get_fields_async(self, pid, psi, pi):
        """Copy the interior into page-locked host arrays; valid after sync()."""
        self._check_host(pid, psi, pi)
        check(lib.mpw_get_fields_async(self.h, pid, psi.ctypes.data_as(_vp), pi.ctypes.data_as(_vp)))

    def step_async(self, dt, nsteps=1):
        """Enqueue the steps and return; device errors surface at sync()."""
        check(lib.mpw_step_async(self.h, float(dt), int(nsteps)))

    def sync(self):
        check(lib.mpw_sync(self.h))

    def _check_host(self, pid, *arrays):
        for a in arrays:
            if a.dtype != np.float64 or not a.flags.c_contiguous or a.shape != tuple(self.shapes[pid]):
                raise ValueError("host arrays must be C-contiguous float64 of the patch shape")

    def get_padded(self, pid):
        s = tuple(v + 2 * NG for v in self.shapes[pid])
        psi = np.empty(s)
        pi = np.empty(s)
        check(lib.mpw_get_padded(self.h, pid, psi.ctypes.data_as(_vp), pi.ctypes.data_as(_vp), 0))
        return psi, pi

    # -- time, flags, stepping ----------------------------------------------
    @property
    def time(self):
        return lib.mpw_time(self.h)

    @time.setter
    def time(self, t):
        check(lib.mpw_set_time(self.h, float(t)))

    def compute_flags(self):
        check(lib.mpw_compute_flags(self.h))

    def get_flags(self):
        f = np.empty(self.shapes[0], dtype=np.uint8)
        check(lib.mpw_get_flags(self.h, f.ctypes.data_as(_vp)))
        return f

    def set_flags(self, flags):
        f = np.ascontiguousarray(flags, dtype=np.uint8)
        check(lib.mpw_set_flags(self.h, f.ctypes.data_as(_vp)))

    def fill_ghosts(self, t):
        check(lib.mpw_fill_ghosts(self.h, float(t)))

    def set_wait_limit(self, limit):
        """Try-waits allowed to the RHS kernels' pipeline waits (0: give up at once)."""
        check(lib.mpw_set_wait_limit(self.h, int(limit)))

    def step(self, dt, nsteps=1):
        check(lib.mpw_step(self.h, float(dt), int(nsteps)))

    def profile(self, enable=True):
        check(lib.mpw_profile_enable(self.h, 1 if enable else 0))

    def profile_read(self):
        """{family: (device ms, launches)} since the last read; families rhs, fill, flags."""
        ms = (C.c_double * 3)()
        n = (C.c_longlong * 3)()
        check(lib.mpw_profile_read(self.h, ms, n, 3))
        return {name: (ms[i], n[i]) for i, name in enumerate(("rhs", "fill", "flags"))}

    def live_points(self):
        n = C.c_longlong()
        check(lib.mpw_live_points(self.h, C.byref(n)))
        return n.value


class Batch:
    """Independent Multipatch instances advanced together: one ghost-fill and
    one RHS launch per substage over all of them (mpw_batch_*)."""

    def __init__(self, sims):
        self.sims = list(sims)  # keeps the contexts alive as long as the batch
        arr = (C.c_void_p * len(self.sims))(*[s.h.value for s in self.sims])
        self.h = C.c_void_p()
        check(lib.mpw_batch_create(arr, len(self.sims), C.byref(self.h)))

    def step(self, dt, nsteps=1):
        """dt: one step size for all instances, or one per instance."""
        d = np.broadcast_to(np.asarray(dt, dtype=np.float64), (len(self.sims),)).copy()
        check(lib.mpw_batch_step(self.h, d.ctypes.data_as(_dp), int(nsteps)))

    def tuning(self):
        """(chosen RHS chunk depth or 0 while tuning, its RHS ms per step,
        batched launches, steps replayed from a captured CUDA graph)."""
        zc, ms, n, g = C.c_int(), C.c_double(), C.c_longlong(), C.c_longlong()
        check(lib.mpw_batch_tuning(self.h, C.byref(zc), C.byref(ms), C.byref(n), C.byref(g)))
        return zc.value, ms.value, n.value, g.value

    def __del__(self):
        if getattr(self, "h", None) and self.h.value:
            lib.mpw_batch_destroy(self.h)
            self.h = C.c_void_p()
