"""Binding of the learned surrogate (include/mpw_surrogate.h): its layer
primitives, the network handle (features, targets, training step, forward,
call, residual check), hybrid stepping of a multipatch simulation, and the
training driver that feeds the network the method's own trajectories.

Argument marshalling only: every layer, gradient, optimizer update and step
of the method runs in the CUDA kernels of libmpw.so.  Tensors are torch CUDA
tensors, channels-last volumes (batch, n2, n1, n0, C); BF16 tensors are
torch.bfloat16.
"""
import ctypes as C

from .mpw import check, lib


def _torch():
    import torch
    return torch


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dims(x):
    B, n2, n1, n0, _ = x.shape
    return int(B), (C.c_int * 3)(int(n0), int(n1), int(n2))


def conv3_forward(x, w, bias=None, relu=False, mask=None, out_bf16=True, out_f32=False, stream=None):
    """y = act(conv3(x, w) + bias); returns (y_bf16 or None, y_f32 or None)."""
    torch = _torch()
    B, n = _dims(x)
    cout, cin = int(w.shape[0]), int(x.shape[4])
    shape = tuple(x.shape[:4]) + (cout,)
    y = torch.empty(shape, dtype=torch.bfloat16, device=x.device) if out_bf16 else None
    y32 = torch.empty(shape, dtype=torch.float32, device=x.device) if out_f32 else None
    check(lib.mpw_conv3_forward(_p(x), cin, _p(w), _p(bias), cout, B, n, int(bool(relu)), _p(mask), _p(y), _p(y32),
                                _stream(stream)))
    return y, y32


def conv3_backward_data(gy, w, mask=None, out_bf16=True, out_f32=False, stream=None):
    """Gradient at the input of a layer with weights w[cout][27][cin]."""
    torch = _torch()
    B, n = _dims(gy)
    cout, cin = int(w.shape[0]), int(w.shape[2])
    shape = tuple(gy.shape[:4]) + (cin,)
    gx = torch.empty(shape, dtype=torch.bfloat16, device=gy.device) if out_bf16 else None
    gx32 = torch.empty(shape, dtype=torch.float32, device=gy.device) if out_f32 else None
    check(lib.mpw_conv3_backward_data(_p(gy), cout, _p(w), cin, B, n, _p(mask), _p(gx), _p(gx32), _stream(stream)))
    return gx, gx32


class WeightGrad:
    """Workspace of mpw_conv3_backward_weights for one (cin, cout) layer."""

    def __init__(self, cin, cout, device):
        torch = _torch()
        self.cin, self.cout = cin, cout
        nbytes = int(lib.mpw_conv3_wgrad_scratch_bytes(cin, cout))
        self.scratch = torch.empty(max(nbytes, 16) // 4, dtype=torch.float32, device=device)

    def __call__(self, x, gy, gw, gb, stream=None):
        B, n = _dims(x)
        check(lib.mpw_conv3_backward_weights(_p(x), self.cin, _p(gy), self.cout, B, n, _p(gw), _p(gb),
                                             _p(self.scratch), self.scratch.numel() * 4, _stream(stream)))


def adam_step(w, g, m, v, lr, t, b1=0.9, b2=0.999, eps=1e-8, w16=None, stream=None):
    check(lib.mpw_adam_step(_p(w), _p(w16), _p(g), _p(m), _p(v), w.numel(), float(lr), float(b1), float(b2),
                            float(eps), int(t), _stream(stream)))


def mse_grad(y, t, gy, loss=None, stream=None):
    """y (points, cy) FP32, t (points, used) FP32 -> gy (points, cy) BF16, loss (1,) FP64."""
    points, cy = int(y.shape[0]), int(y.shape[1])
    check(lib.mpw_mse_grad(_p(y), cy, _p(t), int(t.shape[1]), points, _p(gy), _p(loss), _stream(stream)))


class Surrogate:
    """The learned surrogate (mpw_sur): one call advances a periodic global
    patch by four RK4 steps of the method (Delta = 4 dt)."""

    def __init__(self, dt, h, sigma=1e-3, device=0, stream=None, params=None):
        torch = _torch()
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self.dt, self.h, self.sigma = float(dt), float(h), float(sigma)
        self.count = int(lib.mpw_sur_param_count())
        self.handle = C.c_void_p()
        check(lib.mpw_sur_create(int(device), C.c_void_p(self.stream.cuda_stream), self.dt, self.h, self.sigma,
                                 C.byref(self.handle)))
        if params is not None:
            self.set_params(params)

    def close(self):
        if self.handle:
            lib.mpw_sur_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        check(lib.mpw_sur_set_params(self.handle, C.c_void_p(p.ctypes.data), p.size))

    def _host(self, fn):
        import numpy as np
        out = np.empty(self.count, dtype=np.float32)
        check(fn(self.handle, C.c_void_p(out.ctypes.data), out.size))
        return out

    def params(self):
        return self._host(lib.mpw_sur_get_params)

    def grads(self):
        return self._host(lib.mpw_sur_get_grads)

    @staticmethod
    def _dims(u):
        if u.dim() == 3:
            u = u.unsqueeze(0)
        B, n2, n1, n0 = u.shape
        return u, int(B), (C.c_int * 3)(int(n0), int(n1), int(n2))

    def features(self, psi, pi):
        """(x BF16 (B, n2, n1, n0, 8), scale FP32 (B,)) of FP64 fields (B, n2, n1, n0)."""
        torch = _torch()
        psi, B, n = self._dims(psi)
        pi = pi.reshape(psi.shape)
        x = torch.empty(tuple(psi.shape) + (8,), dtype=torch.bfloat16, device=psi.device)
        s = torch.empty(B, dtype=torch.float32, device=psi.device)
        check(lib.mpw_sur_features(self.handle, _p(psi), _p(pi), B, n, _p(x), _p(s)))
        return x, s

    def targets(self, psi0, pi0, psi1, pi1, scale):
        torch = _torch()
        psi0, B, n = self._dims(psi0)
        t = torch.empty(tuple(psi0.shape) + (2,), dtype=torch.float32, device=psi0.device)
        check(lib.mpw_sur_targets(self.handle, _p(psi0), _p(pi0), _p(psi1), _p(pi1), B, n, _p(scale), _p(t)))
        return t

    def forward(self, x):
        torch = _torch()
        B, n2, n1, n0, _ = x.shape
        y = torch.empty((B, n2, n1, n0, 8), dtype=torch.float32, device=x.device)
        check(lib.mpw_sur_forward(self.handle, _p(x), int(B), (C.c_int * 3)(int(n0), int(n1), int(n2)), _p(y)))
        return y

    def train_step(self, x, t, lr, want_loss=True):
        B, n2, n1, n0, _ = x.shape
        loss = C.c_double(0.0)
        check(lib.mpw_sur_train_step(self.handle, _p(x), _p(t), int(B), (C.c_int * 3)(int(n0), int(n1), int(n2)),
                                     float(lr), C.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def check(self, psi0, pi0, psi1, pi1, want_laplacians=False):
        """(max residual, max state) per sample (FP32 (B, 2)) and optionally the
        Laplacians (4, B, n2, n1, n0) of mpw_sur_check."""
        torch = _torch()
        psi0_, B, n = self._dims(psi0)
        out = torch.empty((B, 2), dtype=torch.float32, device=psi0.device)
        lap = torch.empty((4,) + tuple(psi0_.shape), dtype=torch.float64, device=psi0.device) if want_laplacians else None
        check(lib.mpw_sur_check(self.handle, _p(psi0_), _p(pi0), _p(psi1), _p(pi1), B, n, _p(lap), _p(out)))
        return out, lap

    def predict(self, psi0, pi0, out=None):
        torch = _torch()
        psi0_, B, n = self._dims(psi0)
        if out is None:
            out = (torch.empty_like(psi0), torch.empty_like(pi0))
        check(lib.mpw_sur_predict(self.handle, _p(psi0_), _p(pi0), B, n, _p(out[0]), _p(out[1])))
        return out


# ---------------------------------------------------------------- training on the method's trajectories

class Trajectories:
    """Training pairs from the plain method: each trajectory starts from a
    seeded superposition of eight Gaussians (``workloads.surrogate_pulses``)
    on the periodic global patch [-1,1]^3 of n^3 cells, runs 4 m steps (m
    seeded in 0..max_skip) and yields the state then and four steps later.
    Every step is the method's own (libmpw, FP64)."""

    def __init__(self, n, dt, interp_points=6, ko_eps=0.005, device=0, max_skip=3):
        from . import mpw
        from . import workloads as wl
        self.wl = wl
        self.n, self.dt, self.max_skip = n, dt, max_skip
        self.sim = mpw.Multipatch(interp_points, ko_eps, device=device)
        self.sim.create_patch(mpw.PATCH_GLOBAL, (n, n, n), (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0), mpw.BC_PERIODIC)

    def pair(self, index, out0, out1):
        """Trajectory `index` into the device tensor pairs out0 = (psi0, Pi0), out1."""
        wl = self.wl
        self.sim.set_analytic(wl.GAUSS_SUM, wl.surrogate_pulses(1000 + index), 8)
        self.sim.fill_analytic(0.0)
        skip = int(wl.rng(50000 + index).integers(0, self.max_skip + 1))
        if skip:
            self.sim.step(self.dt, 4 * skip)
        self.sim.get_fields(0, out=out0)
        self.sim.step(self.dt, 4)
        self.sim.get_fields(0, out=out1)


def train(sur, source, trajectories, batch=2, lr=2e-3, lr_end=1e-4, first=0, log_every=0):
    """Train `sur` on `trajectories` pairs of `source` in batches; the learning
    rate decays geometrically from lr to lr_end.  Returns the loss of every
    step.  All arithmetic runs in libmpw (the method's steps, the features,
    targets, forward, backward and Adam)."""
    torch = _torch()
    n = source.n
    shape = (batch, n, n, n)
    dev = torch.device("cuda", sur.device)
    u0 = [torch.empty(shape, dtype=torch.float64, device=dev) for _ in range(2)]
    u1 = [torch.empty(shape, dtype=torch.float64, device=dev) for _ in range(2)]
    steps = max(trajectories // batch, 1)
    losses = []
    for k in range(steps):
        for b in range(batch):
            source.pair(first + k * batch + b, (u0[0][b], u0[1][b]), (u1[0][b], u1[1][b]))
        x, s = sur.features(u0[0], u0[1])
        t = sur.targets(u0[0], u0[1], u1[0], u1[1], s)
        rate = lr * (lr_end / lr) ** (k / max(steps - 1, 1))
        losses.append(sur.train_step(x, t, rate))
        if log_every and k % log_every == 0:
            print(f"step {k} loss {losses[-1]:.4e} lr {rate:.2e}", flush=True)
    return losses


def step_hybrid(sim, sur, dt, calls, tol):
    """mpw_step_surrogate: `calls` surrogate calls of four steps each on the
    multipatch simulation `sim`; returns (accepted calls, largest residual)."""
    acc = C.c_int(0)
    res = C.c_double(0.0)
    check(lib.mpw_step_surrogate(sim.h, sur.handle, float(dt), int(calls), float(tol), C.byref(acc), C.byref(res)))
    return acc.value, res.value
