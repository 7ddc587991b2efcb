"""Spherical-shell local patches (the paper's spherical local patch, Sec. 3.3)
on the GPU against the CPU oracle, element by element.

The parity bar of the Cartesian path: cover flags byte for byte (the covered
set has a hole, so the GPU uses its separable distance transform), ghost fills
to 1e-13 of the state maximum, 1e-12 after one step and 1e-10 after many.
Layouts: a static shell, a thicker shell spinning about its local z axis as in
the paper's Test Three, and a translating shell.
"""
import os

import numpy as np
import pytest

from paper_2002_00088_gb300 import workloads as wl
from tests.helpers import gpu_from, oracle_from
from tests.test_gpu_parity import ARITH, compare_fields, seed_both

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1
CENTRE = (0.013, -0.021, 0.017)

LAYOUTS = [
    pytest.param(lambda: wl.shell_plane(scale=2), id="static"),
    pytest.param(lambda: wl.shell_plane(scale=2, r=(0.25, 0.75), n=(16, 24, 96), motion=wl.ROTATING,
                                        motion_params=CENTRE + (0.0, 0.0, 0.0, 0.0, 0.0, 1.0, np.pi, 0.3)),
                 id="spinning"),
    pytest.param(lambda: wl.shell_plane(scale=2, motion=wl.LINEAR, motion_params=CENTRE + (0.2, -0.1, 0.1)),
                 id="translating"),
]


@pytest.mark.parametrize("make", LAYOUTS)
def test_shell_analytic_fill_matches_oracle(mpw_lib, make):
    w = make()
    o = oracle_from(w, THREADS)
    g = gpu_from(mpw_lib, w)
    o.fill_analytic(0.071)
    g.fill_analytic(0.071)
    got = [g.get_fields(q) for q in range(len(w.patches))]
    want = [o.get_fields(q) for q in range(len(w.patches))]
    for f in range(2):
        scale = max(np.abs(b[f]).max() for b in want)
        err = max(np.abs(a[f] - b[f]).max() for a, b in zip(got, want)) / scale
        assert err < 1e-13, (f, err)


@pytest.mark.parametrize("make", LAYOUTS)
def test_shell_flags_match_oracle_every_step(mpw_lib, make):
    w = make()
    o = oracle_from(w, THREADS)
    g = gpu_from(mpw_lib, w)
    seed_both(o, g, len(w.patches))
    for _ in range(3):
        o.step(w.dt, 1)
        g.step(w.dt, 1)
        fo = o.get_flags()
        np.testing.assert_array_equal(g.get_flags(), fo)
    assert ((fo & 3) == mpw_lib.FLAG_GHOST).sum() > 0
    assert g.live_points() == o.live_points()


@pytest.mark.parametrize("arith", ARITH)
@pytest.mark.parametrize("data", ["closed_form", "random"])
@pytest.mark.parametrize("make", LAYOUTS)
def test_shell_ghost_fill_matches_oracle(mpw_lib, make, data, arith):
    w = make()
    o = oracle_from(w, THREADS)
    g = gpu_from(mpw_lib, w, arith=arith)
    seed_both(o, g, len(w.patches))
    if data == "random":
        for q, p in enumerate(w.patches):
            shape = (p.n[2], p.n[1], p.n[0])
            ps, pi = wl.random_fields(shape, 110 + q)
            mag = 10.0 ** np.random.default_rng(130 + q).uniform(-3.0, 3.0, shape)
            o.set_fields(q, ps * mag, pi * mag)
            g.set_fields(q, ps * mag, pi * mag)
    o.compute_flags()
    g.compute_flags()
    t = 0.013
    o.fill_ghosts(t)
    g.fill_ghosts(t)
    got = [g.get_padded(q) for q in range(len(w.patches))]
    want = [o.get_padded(q, which=1) for q in range(len(w.patches))]
    scale = max(np.nanmax(np.abs(b[f])) for b in want for f in range(2))
    for f in range(2):
        for q in range(len(w.patches)):
            a, b = got[q][f], want[q][f]
            m = np.isfinite(b)
            assert m.sum() > 0
            err = np.abs(a[m] - b[m]).max() / scale
            assert err <= 1e-13, f"patch {q} field {f}: {err:.3e}"


@pytest.mark.parametrize("arith", ARITH)
@pytest.mark.parametrize("make", LAYOUTS)
def test_shell_one_and_thirty_steps(mpw_lib, make, arith):
    w = make()
    o = oracle_from(w, THREADS)
    g = gpu_from(mpw_lib, w, arith=arith)
    n = len(w.patches)
    seed_both(o, g, n)
    o.step(w.dt, 1)
    g.step(w.dt, 1)
    compare_fields(o, g, n, 1e-12)
    o.step(w.dt, 29)
    g.step(w.dt, 29)
    compare_fields(o, g, n, 1e-10)
    np.testing.assert_array_equal(g.get_flags(), o.get_flags())
    assert abs(g.time - o.time) == 0.0


def test_shell_validation(mpw_lib):
    w = wl.shell_plane(scale=2)
    p = w.patches[1]
    g = gpu_from(mpw_lib, wl.shell_plane(scale=2))
    cases = [
        dict(lo=(p.lo[0], 0.02, 0.0)),                       # ghost nodes reach the pole
        dict(hi=(p.hi[0], p.hi[1], np.pi)),                  # not the full azimuth
        dict(n=(4, p.n[1], p.n[2])),                         # radial spacing above the global one
    ]
    for c in cases:
        lo, hi, n = c.get("lo", p.lo), c.get("hi", p.hi), c.get("n", p.n)
        with pytest.raises(mpw_lib.MpwError):
            g.create_patch(p.kind, n, lo, hi, p.outer_bc, p.motion, p.motion_params, p.topology)
    s32 = mpw_lib.Multipatch(interp_points=6, precision=32)
    s32.create_patch(*_args(w.patches[0]))
    with pytest.raises(mpw_lib.MpwError):
        s32.create_patch(*_args(p))


def _args(p):
    return (p.kind, p.n, p.lo, p.hi, p.outer_bc, p.motion, p.motion_params, p.topology)


def test_batch_with_a_shell_matches_individual_steps(mpw_lib):
    ws = wl.batch_instances(count=2, steps=12, seed_index=14, max_global=96)
    ws += [wl.shell_plane(scale=2), LAYOUTS[1].values[0]()]
    sims = []
    for rep in range(2):
        out = []
        for w in ws:
            g = gpu_from(mpw_lib, w)
            g.fill_analytic(0.0)
            out.append(g)
        sims.append(out)
    alone, together = sims
    steps = 5
    for g, w in zip(alone, ws):
        g.step(w.dt, steps)
    b = mpw_lib.Batch(together)
    b.step([w.dt for w in ws], steps)
    for g, h, w in zip(alone, together, ws):
        assert g.time == h.time
        np.testing.assert_array_equal(g.get_flags(), h.get_flags())
        for q in range(len(w.patches)):
            a, c = g.get_fields(q), h.get_fields(q)
            np.testing.assert_array_equal(a[0], c[0])
            np.testing.assert_array_equal(a[1], c[1])
