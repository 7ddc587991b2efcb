"""Pins of the oracle's multipatch plumbing (Sec. 2.4: flags, Local-to-Global,
Global-to-Local, buffer, one-way data flow) and of its motion handling.

* A static harmonic polynomial of degree <= P-1 is a fixed point of the whole
  discrete scheme: the RHS is exactly zero and every interpolation is exact,
  so a multipatch run must leave it unchanged up to rounding.
* Poisoning: every non-live or ghost entry of a stage state is NaN until a
  boundary condition fills it; a finite result proves every read was filled.
* A planted mistake (buffer narrower than the interpolation stencil) makes the
  oracle's own donor check fire: windows would read effective-ghost data
  (interpolation of interpolated data, which the buffer exists to prevent).
* L2G and G2L commute (Sec. 2.4.1) bit for bit.
* A patch translating with zero velocity is bitwise the static patch.
"""
import numpy as np
import pytest

from oracle import pyoracle as po
from paper_2002_00088_gb300 import workloads as wl
from tests.helpers import oracle_from


def harmonic_layout(P, motion=po.STATIC, mparams=()):
    o = po.Oracle(interp_points=P, ko_eps=0.005, threads=4)
    o.add_patch(po.GLOBAL, (36, 36, 36), (-1, -1, -1), (1, 1, 1), po.BC_ANALYTIC)
    o.add_patch(po.LOCAL, (24, 24, 24), (-1 / 3,) * 3, (1 / 3,) * 3, po.BC_INTERPATCH, motion,
                mparams or (0.013, -0.021, 0.007))
    rng = np.random.default_rng(9)
    coef = rng.normal(size=14)
    o.set_analytic(po.HARMONIC_POLY, coef, 14)
    o.fill_analytic(0.0)
    return o


@pytest.mark.parametrize("P", [5, 6])
def test_harmonic_polynomial_is_a_fixed_point(P):
    o = harmonic_layout(P)
    before = [o.get_fields(q) for q in range(2)]
    h = 2.0 / 36 / 2
    o.step(0.25 * h, 4)
    for q in range(2):
        ps, pi = o.get_fields(q)
        ref = before[q][0]
        m = np.isfinite(ps)
        assert m.sum() > 0.9 * ps.size
        scale = np.abs(ref[m]).max()
        assert np.abs(ps[m] - ref[m]).max() < 1e-12 * scale
        assert np.abs(pi[m]).max() < 1e-10 * scale


def test_no_nan_reaches_live_data():
    w = wl.orbiting_gauss(scale=4, steps=3)
    o = oracle_from(w)
    o.fill_analytic(0.0)
    o.step(w.dt, 3)
    f = o.get_flags() & 3
    ps, pi = o.get_fields(0)
    live = (f == po.LIVE) | (f == po.REVIVED)
    assert np.isfinite(ps[live]).all() and np.isfinite(pi[live]).all()
    assert np.isnan(ps[~live]).all()
    for q in range(1, 5):
        a, b = o.get_fields(q)
        assert np.isfinite(a).all() and np.isfinite(b).all()


def test_planted_narrow_buffer_is_caught():
    """Buffer 1 < NG+1: Global-to-Local windows reach effective ghost cells."""
    w = wl.static_gauss(steps=1)
    o = oracle_from(w, buffer=1)
    o.fill_analytic(0.0)
    with pytest.raises(po.OracleError, match="non-live"):
        o.step(w.dt, 1)


def test_l2g_g2l_order_is_irrelevant():
    w = wl.orbiting_gauss(scale=4, steps=2)
    res = []
    for first in (True, False):
        o = oracle_from(w)
        o.set_fill_order(first)
        o.fill_analytic(0.0)
        o.step(w.dt, 2)
        res.append([o.get_fields(q) for q in range(5)])
    for a, b in zip(*res):
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])


def test_zero_velocity_translation_is_static():
    w = wl.static_gauss(steps=3)
    outs = []
    for motion, mp in ((po.STATIC, (0.0, 0.0, 0.0)), (po.LINEAR, (0.0, 0.0, 0.0, 0.0, 0.0, 0.0))):
        w.patches[1].motion = motion
        w.patches[1].motion_params = mp
        o = oracle_from(w)
        o.fill_analytic(0.0)
        o.step(w.dt, 3)
        outs.append([o.get_fields(q) for q in range(2)])
    for a, b in zip(*outs):
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])
