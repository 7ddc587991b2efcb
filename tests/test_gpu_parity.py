"""GPU (libmpw, sm_103a) against the CPU oracle, element by element.

Every case feeds both sides the same seeded inputs (closed-form initial data
evaluated by the oracle, or random arrays from the workload generators) and
compares through the C ABI.  Tolerances are the parity bar of the project:
1e-12 relative to max|field| after one step, 1e-10 relative to max|psi| after
100 steps; cover flags must match byte for byte.
"""
import os

import numpy as np
import pytest

from oracle import pyoracle as po
from paper_2002_00088_gb300 import workloads as wl
from tests.helpers import gpu_from, interior, oracle_from, rel_err

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1


def seed_both(o, g, npatch):
    """Closed-form initial data at t = 0 from the oracle, copied into the GPU."""
    o.fill_analytic(0.0)
    for q in range(npatch):
        ps, pi = o.get_fields(q)
        g.set_fields(q, ps, pi)
    g.time = 0.0


def compare_fields(o, g, npatch, tol):
    """max |gpu - oracle| of each field over every patch, relative to the
    largest |value| of that field over the whole domain (all patches)."""
    got = [g.get_fields(q) for q in range(npatch)]
    want = [o.get_fields(q) for q in range(npatch)]
    worst = 0.0
    for f in range(2):
        scale = max(np.nanmax(np.abs(w[f])) for w in want)
        for q in range(npatch):
            a, b = got[q][f], want[q][f]
            np.testing.assert_array_equal(np.isnan(a), np.isnan(b))
            m = np.isfinite(b)
            e = float(np.abs(a[m] - b[m]).max() / scale)
            worst = max(worst, e)
            assert e <= tol, f"patch {q} field {f}: relative error {e:.3e} > {tol:.1e}"
    return worst


ARITH = [pytest.param(0, id="fixed"), pytest.param(1, id="fp64")]


@pytest.mark.parametrize("arith", ARITH)
@pytest.mark.parametrize("w", [(0.0, 0.0, 0.0), (0.7, -0.4, 1.3)])
@pytest.mark.parametrize("n,lo,hi", [((40, 24, 20), (-0.5, -0.3, -0.2), (0.5, 0.4, 0.3)),
                                     ((67, 29, 33), (-0.5, -0.3, -0.2), (0.5, 0.4, 0.3)),
                                     ((48, 48, 48), (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0))])
def test_periodic_patch_random_fields(mpw_lib, w, n, lo, hi, arith):
    """Fused RHS + RK4 stage kernel alone: one periodic patch (several tiles and
    ragged tails, anisotropic and isotropic spacing), random data, with and
    without frame velocity, in both arithmetic modes."""
    motion = po.LINEAR if any(w) else po.STATIC
    mp = (0.0, 0.0, 0.0) + tuple(w)
    o = po.Oracle(6, 0.005, threads=THREADS)
    o.add_patch(po.GLOBAL, n, lo, hi, po.BC_PERIODIC, motion, mp)
    g = mpw_lib.Multipatch(6, 0.005, arith=arith)
    g.create_patch(mpw_lib.PATCH_GLOBAL, n, lo, hi, mpw_lib.BC_PERIODIC, motion, mp)
    ps, pi = wl.random_fields((n[2], n[1], n[0]), 3)
    o.set_fields(0, ps, pi)
    g.set_fields(0, ps, pi)
    h = min((hi[a] - lo[a]) / n[a] for a in range(3))
    dt = 0.1 * h
    o.step(dt, 1)
    g.step(dt, 1)
    compare_fields(o, g, 1, 1e-12)
    o.step(dt, 4)
    g.step(dt, 4)
    compare_fields(o, g, 1, 5e-12)
    assert g.time == o.time


def test_non_finite_values_propagate_like_ieee(mpw_lib):
    """A NaN in live data spreads through the stencil exactly as in the oracle's
    FP64 arithmetic (the fixed-point kernel falls back per CTA)."""
    n, lo, hi = (40, 24, 20), (-0.5, -0.3, -0.2), (0.5, 0.4, 0.3)
    ps, pi = wl.random_fields((n[2], n[1], n[0]), 4)
    ps[7, 11, 13] = np.nan
    o = po.Oracle(6, 0.005)
    o.add_patch(po.GLOBAL, n, lo, hi, po.BC_PERIODIC)
    g = mpw_lib.Multipatch(6, 0.005)
    g.create_patch(mpw_lib.PATCH_GLOBAL, n, lo, hi, mpw_lib.BC_PERIODIC)
    o.set_fields(0, ps, pi)
    g.set_fields(0, ps, pi)
    o.step(0.002, 1)
    g.step(0.002, 1)
    a, b = g.get_fields(0), o.get_fields(0)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(np.isnan(x), np.isnan(y))
        assert np.isnan(y).any()
        m = np.isfinite(y)
        assert np.abs(x[m] - y[m]).max() <= 1e-12 * np.abs(y[m]).max()


def test_analytic_fill_matches_oracle(mpw_lib):
    for w in (wl.static_gauss(), wl.orbiting_gauss(scale=4), wl.translating_plane()):
        o = oracle_from(w, THREADS)
        g = gpu_from(mpw_lib, w)
        o.fill_analytic(0.071)
        g.fill_analytic(0.071)
        for q in range(len(w.patches)):
            a, b = g.get_fields(q), o.get_fields(q)
            assert rel_err(a[0], b[0]) < 1e-13 and rel_err(a[1], b[1]) < 1e-13


@pytest.mark.parametrize("scale", [4, 2])
def test_flags_match_oracle_every_step(mpw_lib, scale):
    w = wl.orbiting_gauss(scale=scale)
    o = oracle_from(w, THREADS)
    g = gpu_from(mpw_lib, w)
    seed_both(o, g, len(w.patches))
    for s in range(4):
        o.step(w.dt, 1)
        g.step(w.dt, 1)
        np.testing.assert_array_equal(g.get_flags(), o.get_flags())


def test_static_flags_counts(mpw_lib):
    w = wl.static_gauss()
    g = gpu_from(mpw_lib, w)
    g.fill_analytic(0.0)
    g.compute_flags()
    f = g.get_flags() & 3
    assert (f == mpw_lib.FLAG_GHOST).sum() == 504 and (f == mpw_lib.FLAG_DEAD).sum() == 8
    assert g.live_points() == 48 ** 3 - 512 + 32 ** 3


@pytest.mark.parametrize("arith", ARITH)
@pytest.mark.parametrize("data", ["closed_form", "random"])
@pytest.mark.parametrize("make", [lambda: wl.static_gauss(), lambda: wl.orbiting_gauss(scale=4)])
def test_ghost_fill_matches_oracle(mpw_lib, make, data, arith):
    """Outer BC + Local-to-Global + Global-to-Local on identical data: the
    closed form, or random fields whose magnitude varies over six decades."""
    w = make()
    o = oracle_from(w, THREADS)
    g = gpu_from(mpw_lib, w, arith=arith)
    seed_both(o, g, len(w.patches))
    if data == "random":
        for q, p in enumerate(w.patches):
            shape = (p.n[2], p.n[1], p.n[0])
            ps, pi = wl.random_fields(shape, 40 + q)
            mag = 10.0 ** np.random.default_rng(60 + q).uniform(-3.0, 3.0, shape)
            o.set_fields(q, ps * mag, pi * mag)
            g.set_fields(q, ps * mag, pi * mag)
    o.compute_flags()
    g.compute_flags()
    t = 0.013
    o.fill_ghosts(t)
    g.fill_ghosts(t)
    got = [g.get_padded(q) for q in range(len(w.patches))]
    want = [o.get_padded(q, which=1) for q in range(len(w.patches))]
    # max |difference| over every patch relative to the largest |value| of the
    # state over the whole domain (both fields: at t = 0.013 the closed-form
    # Pi is near zero and cancels, so its own maximum is rounding noise)
    scale = max(np.nanmax(np.abs(b[f])) for b in want for f in range(2))
    for f in range(2):
        for q in range(len(w.patches)):
            a, b = got[q][f], want[q][f]
            m = np.isfinite(b)
            assert m.sum() > 0
            err = np.abs(a[m] - b[m]).max() / scale
            assert err <= 1e-13, f"patch {q} field {f}: {err:.3e}"


@pytest.mark.parametrize("arith", ARITH)
def test_static_gauss_one_and_hundred_steps(mpw_lib, arith):
    """48^3 global + 32^3 local, static, 5-point Lagrange, 100 steps."""
    w = wl.static_gauss()
    o = oracle_from(w, THREADS)
    g = gpu_from(mpw_lib, w, arith=arith)
    seed_both(o, g, 2)
    o.step(w.dt, 1)
    g.step(w.dt, 1)
    compare_fields(o, g, 2, 1e-12)
    o.step(w.dt, w.steps - 1)
    g.step(w.dt, w.steps - 1)
    for q in range(2):
        a_ps, _ = g.get_fields(q)
        b_ps, _ = o.get_fields(q)
        m = np.isfinite(b_ps)
        assert np.abs(a_ps[m] - b_ps[m]).max() <= 1e-10 * np.abs(b_ps[m]).max()
    assert abs(g.time - o.time) == 0.0


@pytest.mark.parametrize("arith", ARITH)
def test_orbiting_downscaled_many_steps(mpw_lib, arith):
    """64^3 global + four orbiting 32^3 locals, 6-point Lagrange, 40 steps:
    flags change, cells are revived and poisoned along the way."""
    w = wl.orbiting_gauss(scale=4)
    o = oracle_from(w, THREADS)
    g = gpu_from(mpw_lib, w, arith=arith)
    seed_both(o, g, 5)
    o.step(w.dt, 1)
    g.step(w.dt, 1)
    compare_fields(o, g, 5, 1e-12)
    o.step(w.dt, 39)
    g.step(w.dt, 39)
    compare_fields(o, g, 5, 1e-10)
    np.testing.assert_array_equal(g.get_flags(), o.get_flags())


def test_orbiting_half_size_hundred_steps(mpw_lib):
    """128^3 global + four orbiting 64^3 locals (the throughput workload at
    half resolution), 100 steps: the parity bar of 1e-10 after 100 steps on a
    moving layout, with the flags recomputed, cells revived and poisoned at
    every step."""
    w = wl.orbiting_gauss(scale=2)
    o = oracle_from(w, THREADS)
    g = gpu_from(mpw_lib, w)
    seed_both(o, g, 5)
    o.step(w.dt, 1)
    g.step(w.dt, 1)
    compare_fields(o, g, 5, 1e-12)
    o.step(w.dt, 99)
    g.step(w.dt, 99)
    compare_fields(o, g, 5, 1e-10)
    np.testing.assert_array_equal(g.get_flags(), o.get_flags())
    assert g.time == o.time


def test_orbiting_full_size_one_step(mpw_lib):
    """256^3 global + four 128^3 locals (the throughput workload), one step."""
    w = wl.orbiting_gauss()
    o = oracle_from(w, THREADS)
    g = gpu_from(mpw_lib, w)
    seed_both(o, g, 5)
    o.step(w.dt, 1)
    g.step(w.dt, 1)
    compare_fields(o, g, 5, 1e-12)
    np.testing.assert_array_equal(g.get_flags(), o.get_flags())


@pytest.mark.parametrize("P", [5, 6])
def test_harmonic_fixed_point(mpw_lib, P):
    o = po.Oracle(P, 0.005)
    g = mpw_lib.Multipatch(P, 0.005)
    coef = np.random.default_rng(9).normal(size=14)
    for sim, kind in ((o, "o"), (g, "g")):
        sim_add = sim.add_patch if kind == "o" else sim.create_patch
        sim_add(0, (36, 36, 36), (-1, -1, -1), (1, 1, 1), 0)
        sim_add(1, (24, 24, 24), (-1 / 3,) * 3, (1 / 3,) * 3, 2, 0, (0.013, -0.021, 0.007))
        sim.set_analytic(po.HARMONIC_POLY, coef, 14)
        sim.fill_analytic(0.0)
    before = [g.get_fields(q) for q in range(2)]
    g.step(0.25 / 36, 4)
    for q in range(2):
        ps, pi = g.get_fields(q)
        m = np.isfinite(ps)
        assert np.abs(ps[m] - before[q][0][m]).max() < 1e-12 * np.abs(before[q][0][m]).max()


def test_checkpoint_restart_is_bitwise(mpw_lib):
    w = wl.orbiting_gauss(scale=4)
    a = gpu_from(mpw_lib, w)
    a.fill_analytic(0.0)
    a.step(w.dt, 6)
    ref = [a.get_fields(q) for q in range(5)]
    b = gpu_from(mpw_lib, w)
    b.fill_analytic(0.0)
    b.step(w.dt, 3)
    state = [b.get_fields(q) for q in range(5)], b.get_flags(), b.time
    c = gpu_from(mpw_lib, w)
    for q in range(5):
        c.set_fields(q, *state[0][q])
    c.set_flags(state[1])
    c.time = state[2]
    c.step(w.dt, 3)
    for q in range(5):
        x, y = c.get_fields(q), ref[q]
        np.testing.assert_array_equal(x[0], y[0])
        np.testing.assert_array_equal(x[1], y[1])


def test_device_pointer_fields(mpw_lib):
    import torch
    w = wl.static_gauss()
    g = gpu_from(mpw_lib, w)
    g.fill_analytic(0.0)
    ps = torch.empty((32, 32, 32), dtype=torch.float64, device="cuda")
    pi = torch.empty_like(ps)
    g.get_fields(1, out=(ps, pi))
    hp, hq = g.get_fields(1)
    np.testing.assert_array_equal(ps.cpu().numpy(), hp)
    g.set_fields(1, ps * 2, pi)
    np.testing.assert_array_equal(g.get_fields(1)[0], 2 * hp)


def test_pinned_host_fields_match_pageable(mpw_lib):
    """Page-locked host arrays take the in-place kernel path, pageable ones the
    staging copy: both must move the same bits, in and out, and a step run
    from pinned input must equal one run from pageable input."""
    import torch
    w = wl.orbiting_gauss(scale=4)
    rng = np.random.default_rng(11)
    a = gpu_from(mpw_lib, w)
    b = gpu_from(mpw_lib, w)
    a.fill_analytic(0.0)
    b.fill_analytic(0.0)
    for q in range(len(w.patches)):
        shape = a.shapes[q]
        pin = [torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy() for _ in range(2)]
        src = [rng.standard_normal(shape) * 1e-3 + a.get_fields(q)[f] for f in range(2)]
        src = [np.nan_to_num(x) for x in src]
        pin[0][...] = src[0]
        pin[1][...] = src[1]
        a.set_fields(q, pin[0], pin[1])
        b.set_fields(q, src[0].copy(), src[1].copy())
        out = [torch.zeros(shape, dtype=torch.float64, pin_memory=True).numpy() for _ in range(2)]
        a.get_fields(q, out=out)
        ref = b.get_fields(q)
        np.testing.assert_array_equal(out[0], ref[0])
        np.testing.assert_array_equal(out[1], ref[1])
    a.step(w.dt, 2)
    b.step(w.dt, 2)
    for q in range(len(w.patches)):
        out = [torch.zeros(a.shapes[q], dtype=torch.float64, pin_memory=True).numpy() for _ in range(2)]
        a.get_fields(q, out=out)
        ref = b.get_fields(q)
        np.testing.assert_array_equal(out[0], ref[0])
        np.testing.assert_array_equal(out[1], ref[1])


def test_async_host_io_matches_synchronous(mpw_lib):
    """Pipelined use of the asynchronous transfers: each step takes a fresh
    input and returns its result; the bits must equal the synchronous calls."""
    import torch
    w = wl.orbiting_gauss(scale=4)
    rng = np.random.default_rng(5)
    a = gpu_from(mpw_lib, w)
    b = gpu_from(mpw_lib, w)
    a.fill_analytic(0.0)
    b.fill_analytic(0.0)
    npatch = len(w.patches)
    pinned = lambda s: torch.zeros(s, dtype=torch.float64, pin_memory=True).numpy()
    base = [a.get_fields(q) for q in range(npatch)]
    inputs = []
    for k in range(3):
        step_in = []
        for q in range(npatch):
            ps, pi = (np.nan_to_num(x) * (1.0 + 1e-3 * rng.standard_normal(x.shape)) for x in base[q])
            hp, hq = pinned(ps.shape), pinned(pi.shape)
            hp[...] = ps
            hq[...] = pi
            step_in.append((hp, hq))
        inputs.append(step_in)
    outs = [[(pinned(a.shapes[q]), pinned(a.shapes[q])) for q in range(npatch)] for _ in range(3)]
    for k in range(3):
        for q in range(npatch):
            a.set_fields_async(q, *inputs[k][q])
        a.step_async(w.dt, 1)
        for q in range(npatch):
            a.get_fields_async(q, *outs[k][q])
    a.sync()
    for k in range(3):
        for q in range(npatch):
            b.set_fields(q, *inputs[k][q])
        b.step(w.dt, 1)
        for q in range(npatch):
            ref = b.get_fields(q)
            np.testing.assert_array_equal(outs[k][q][0], ref[0])
            np.testing.assert_array_equal(outs[k][q][1], ref[1])
    with pytest.raises(mpw_lib.MpwError) as e:
        a.set_fields_async(0, np.zeros(a.shapes[0]), np.zeros(a.shapes[0]))  # pageable
    assert e.value.status == 1


def test_validation_errors(mpw_lib):
    M = mpw_lib
    w = wl.static_gauss()
    g = gpu_from(M, w)
    g.fill_analytic(0.0)
    with pytest.raises(M.MpwError) as e:
        g.step(1.0 / 48, 1)  # far beyond the RK4 stability estimate
    assert e.value.status == 3
    with pytest.raises(M.MpwError):
        g.step(-1.0, 1)
    # a patch that leaves the global interior
    g2 = M.Multipatch(6, 0.005)
    g2.create_patch(M.PATCH_GLOBAL, (32, 32, 32), (-1, -1, -1), (1, 1, 1), M.BC_ANALYTIC)
    g2.create_patch(M.PATCH_LOCAL, (16, 16, 16), (-0.25,) * 3, (0.25,) * 3, M.BC_INTERPATCH, M.MOTION_STATIC,
                    (0.7, 0.0, 0.0))
    g2.set_analytic(M.ANALYTIC_GAUSS_SUM, [1, 0.2, 0, 0, 0], 1)
    with pytest.raises(M.MpwError) as e:
        g2.step(0.25 / 32, 1)
    assert e.value.status == 5
    # two patches closer than the separation rule
    g3 = M.Multipatch(6, 0.005)
    g3.create_patch(M.PATCH_GLOBAL, (32, 32, 32), (-1, -1, -1), (1, 1, 1), M.BC_ANALYTIC)
    for x in (-0.15, 0.15):
        g3.create_patch(M.PATCH_LOCAL, (16, 16, 16), (-0.125,) * 3, (0.125,) * 3, M.BC_INTERPATCH,
                        M.MOTION_STATIC, (x, 0.0, 0.0))
    g3.set_analytic(M.ANALYTIC_GAUSS_SUM, [1, 0.2, 0, 0, 0], 1)
    with pytest.raises(M.MpwError) as e:
        g3.step(0.25 / 64, 1)
    assert e.value.status == 2
    # a patch faster than one global cell per step (1:1 resolution, so the
    # stability estimate still admits the step)
    g4 = M.Multipatch(6, 0.005)
    g4.create_patch(M.PATCH_GLOBAL, (32, 32, 32), (-1, -1, -1), (1, 1, 1), M.BC_ANALYTIC)
    g4.create_patch(M.PATCH_LOCAL, (8, 8, 8), (-0.25,) * 3, (0.25,) * 3, M.BC_INTERPATCH,
                    M.MOTION_LINEAR, (0.0, 0.0, 0.0, 5.0, 0.0, 0.0))
    g4.set_analytic(M.ANALYTIC_GAUSS_SUM, [1, 0.2, 0, 0, 0], 1)
    with pytest.raises(M.MpwError) as e:
        g4.step(0.25 / 16, 1)
    assert e.value.status == 4
    # configuration errors
    with pytest.raises(M.MpwError):
        M.Multipatch(interp_points=4)
    g5 = M.Multipatch(6, 0.005)
    with pytest.raises(M.MpwError):
        g5.create_patch(M.PATCH_LOCAL, (16, 16, 16), (-1,) * 3, (1,) * 3, M.BC_INTERPATCH)
