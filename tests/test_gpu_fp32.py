"""The binary32 precision (mpw_config.precision = 32) against the FP64 oracle
and the closed form.

Tolerance, derived from the arithmetic.  Notation:
- u = 2^-24 is the binary32 unit roundoff;
- M_f is the largest |value| of field f over the domain;
- errors are measured relative to M_f.

Error sources per RK4 step:
- set_fields rounds each value once: u/2.
- Every substage rounds its stored outputs (ACC, the next stage state) once
  each.  This adds at most ~3u per step through ACC and u_{n+1}.
- A ghost fill adds at most (1 + L + L^2 + L^3) u/2 < 3u, with L = 1.39 the
  Lebesgue constant of the windows.
- The stencils are built from exact differences to the centre value, so
  their own rounding is small.  But the stored psi carries its rounding of
  u/2 M_psi, and the Laplacian weighs that by 3 x 64 / (12 h^2).  K_Pi is
  therefore off by up to 8 u M_psi / h^2.  Over a step (sum of b_l dt = dt =
  h_min / 4) that adds 2 u M_psi / h_min to Pi.

At CFL 0.25 with KO dissipation, errors carry over from step to step without
growing.  After n steps:
    err_psi <= (3 n + 1) u
    err_Pi  <= (n (3 + 2 (M_psi / M_Pi) / h_min) + 1) u
The tests take twice these bounds.
"""
import os

import numpy as np
import pytest

from paper_2002_00088_gb300 import workloads as wl
from tests.helpers import gpu_from, oracle_from

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1
U32 = 2.0 ** -24


def tol(steps, h_min=None, ratio=0.0):
    """2x the bound of the module docstring; ratio = M_psi / M_Pi (0 for psi)."""
    amp = 2.0 * ratio / h_min if h_min else 0.0
    return 2.0 * (steps * (3.0 + amp) + 1.0) * U32


def field_tols(w, want, steps):
    h_min = min(min((p.hi[a] - p.lo[a]) / p.n[a] for a in range(3)) for p in w.patches)
    m = [max(np.nanmax(np.abs(x[f])) for x in want) for f in range(2)]
    return [tol(steps), tol(steps, h_min, m[0] / m[1])]


def seed(o, g, npatch):
    o.fill_analytic(0.0)
    for q in range(npatch):
        g.set_fields(q, *o.get_fields(q))
    g.time = 0.0


def domain_errors(got, want):
    """max |got - want| per field over all patches / max |want| of the field."""
    out = []
    for f in range(2):
        scale = max(np.nanmax(np.abs(w[f])) for w in want)
        e = 0.0
        for a, b in zip(got, want):
            m = np.isfinite(b[f])
            assert np.array_equal(np.isfinite(a[f]), m), "live masks differ"
            e = max(e, float(np.abs(a[f][m] - b[f][m]).max()) / scale)
        out.append(e)
    return out


@pytest.mark.parametrize("make", [lambda: wl.plane_gauss(scale=8), lambda: wl.orbiting_gauss(scale=4)])
def test_fp32_ghost_fill_matches_oracle(mpw_lib, make):
    w = make()
    o = oracle_from(w, THREADS)
    g = gpu_from(mpw_lib, w, precision=32)
    seed(o, g, len(w.patches))
    o.compute_flags()
    g.compute_flags()
    o.fill_ghosts(0.004)
    g.fill_ghosts(0.004)
    got = [g.get_padded(q) for q in range(len(w.patches))]
    want = [o.get_padded(q, which=1) for q in range(len(w.patches))]
    scale = max(np.nanmax(np.abs(b[f])) for b in want for f in range(2))
    for a, b in zip(got, want):
        for f in range(2):
            m = np.isfinite(b[f])
            # set_fields rounding (u/2) plus one fill (< 3u), doubled
            assert np.abs(a[f][m] - b[f][m]).max() <= 7 * U32 * scale


@pytest.mark.parametrize("steps", [1, 20])
def test_fp32_plane_gauss_matches_oracle(mpw_lib, steps):
    """Periodic 64^3 + static 32^3 at 2x: the precision configuration at 1/8 size."""
    w = wl.plane_gauss(scale=8)
    o = oracle_from(w, THREADS)
    g = gpu_from(mpw_lib, w, precision=32)
    seed(o, g, 2)
    o.step(w.dt, steps)
    g.step(w.dt, steps)
    want = [o.get_fields(q) for q in range(2)]
    errs = domain_errors([g.get_fields(q) for q in range(2)], want)
    tols = field_tols(w, want, steps)
    print(f"plane_gauss_64+32, {steps} steps, FP32 vs FP64 oracle: psi {errs[0]:.2e} (bound {tols[0]:.1e}), "
          f"Pi {errs[1]:.2e} (bound {tols[1]:.1e})")
    assert errs[0] <= tols[0] and errs[1] <= tols[1], (errs, tols)


def test_fp32_orbiting_matches_oracle(mpw_lib):
    """Moving patches (maps, cover flags, revival) in binary32."""
    w = wl.orbiting_gauss(scale=4)
    o = oracle_from(w, THREADS)
    g = gpu_from(mpw_lib, w, precision=32)
    seed(o, g, len(w.patches))
    o.step(w.dt, 10)
    g.step(w.dt, 10)
    assert np.array_equal(g.get_flags(), o.get_flags())
    want = [o.get_fields(q) for q in range(len(w.patches))]
    errs = domain_errors([g.get_fields(q) for q in range(len(w.patches))], want)
    tols = field_tols(w, want, 10)
    assert errs[0] <= tols[0] and errs[1] <= tols[1], (errs, tols)


def test_fp32_error_against_closed_form(mpw_lib):
    """At 128^3 + 64^3 the truncation error dominates: the binary32 run stays
    within 1 % (plus the binary32 floor) of the FP64 run's error against the
    closed form."""
    w = wl.plane_gauss(scale=4, steps=40)
    o = oracle_from(w, THREADS)
    runs = {}
    for prec in (64, 32):
        g = gpu_from(mpw_lib, w, precision=prec)
        seed(o, g, 2)
        g.step(w.dt, w.steps)
        runs[prec] = [g.get_fields(q) for q in range(2)]
    t = w.steps * w.dt
    o.fill_analytic(t)
    exact = [o.get_fields(q) for q in range(2)]

    def errors(run):  # over the live cells of the run (non-live global cells read as NaN)
        out = []
        for f in range(2):
            scale = max(np.abs(x[f]).max() for x in exact)
            out.append(max(float(np.nanmax(np.abs(a[f] - b[f]))) for a, b in zip(run, exact)) / scale)
        return out

    e64 = errors(runs[64])
    e32 = errors(runs[32])
    print(f"plane_gauss_128+64, {w.steps} steps, error vs closed form: FP64 psi {e64[0]:.3e} Pi {e64[1]:.3e}; "
          f"FP32 psi {e32[0]:.3e} Pi {e32[1]:.3e}")
    tols = field_tols(w, runs[64], w.steps)
    for a, b, t in zip(e32, e64, tols):
        assert a <= 1.01 * b + t
