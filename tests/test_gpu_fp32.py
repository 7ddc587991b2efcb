"""The binary32 precision (mpw_config.precision = 32) against the FP64 oracle
and the closed form.

Tolerance (derived from the arithmetic, u = 2^-24 the binary32 unit roundoff,
all errors relative to the largest |value| of the field over the domain):
- set_fields rounds each value once, u/2;
- every substage rounds its stored outputs once each.  K itself, built from
  exact differences to the centre value, is off by a few roundings of its own
  terms, which are dt-times smaller than the field.  A step therefore adds at
  most ~3u through ACC and u_{n+1};
- a ghost fill adds at most (1 + L + L^2 + L^3) u/2 < 3u, with L = 1.39 the
  Lebesgue constant of the windows;
- at CFL 0.25 with KO dissipation, errors carry over from step to step without
  growing.
After n steps the difference to the FP64 oracle is then below 6 (n + 1) u;
the tests take 8 (n + 1) u.
"""
import os

import numpy as np
import pytest

from paper_2002_00088_gb300 import workloads as wl
from tests.helpers import gpu_from, oracle_from

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1
U32 = 2.0 ** -24


def tol(steps):
    return 8.0 * (steps + 1) * U32


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
            assert np.abs(a[f][m] - b[f][m]).max() <= 6 * U32 * scale


@pytest.mark.parametrize("steps", [1, 20])
def test_fp32_plane_gauss_matches_oracle(mpw_lib, steps):
    """Periodic 64^3 + static 32^3 at 2x: the precision configuration at 1/8 size."""
    w = wl.plane_gauss(scale=8)
    o = oracle_from(w, THREADS)
    g = gpu_from(mpw_lib, w, precision=32)
    seed(o, g, 2)
    o.step(w.dt, steps)
    g.step(w.dt, steps)
    errs = domain_errors([g.get_fields(q) for q in range(2)], [o.get_fields(q) for q in range(2)])
    print(f"plane_gauss_64+32, {steps} steps, FP32 vs FP64 oracle: psi {errs[0]:.2e}, Pi {errs[1]:.2e}")
    assert max(errs) <= tol(steps), errs


def test_fp32_orbiting_matches_oracle(mpw_lib):
    """Moving patches (maps, cover flags, revival) in binary32."""
    w = wl.orbiting_gauss(scale=4)
    o = oracle_from(w, THREADS)
    g = gpu_from(mpw_lib, w, precision=32)
    seed(o, g, len(w.patches))
    o.step(w.dt, 10)
    g.step(w.dt, 10)
    assert np.array_equal(g.get_flags(), o.get_flags())
    errs = domain_errors([g.get_fields(q) for q in range(len(w.patches))],
                         [o.get_fields(q) for q in range(len(w.patches))])
    assert max(errs) <= tol(10), errs


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
    for a, b in zip(e32, e64):
        assert a <= 1.01 * b + tol(w.steps)
