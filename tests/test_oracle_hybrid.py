"""Pins of the oracle's hybrid-call pieces (oracle/oracle.c orc_fill_dead and
orc_step_locals, oracle/surrogate.py hermite_stage_weights): the parts of the
learned surrogate's hybrid call with local patches, an extension of the
paper's method (RK4, Table 1; Global-to-Local and Local-to-Global, Sec. 2.4).

* ψ = t² + (x² + y² + z²)/3, Π = 2t solves the wave equation, and every
  operator of the method is exact on it: 4th-order differences on quadratics,
  KO on quadratics (zero), 6-point Lagrange windows on quadratics, RK4 on a
  quadratic in time.  So one locals-only step whose global stage states are
  the RK4 stage states the method forms on the global must reproduce the exact
  solution at t + dt on the local patch, to rounding; a wrong stage weight,
  a wrong stage-to-substage mapping or a wrong Global-to-Local donor fails it.
* The dead-cell fill of that field is exact too (cells deep under the local
  patch, interpolated from it).
* The Hermite stage weights, fed with the exact data of y' = λ y, reproduce
  the stage inputs RK4 forms from the exact state, to the quintic
  interpolant's O((λΔ)^6): the error falls 2^6-fold when Δ halves.
"""
import numpy as np
import pytest

from oracle import pyoracle as po
from oracle import surrogate as so

X0 = (0.06, -0.04, 0.02)


def quad(x, y, z, t):
    return t * t + (x * x + y * y + z * z) / 3.0, 2.0 * t + 0.0 * x


def nodes(n, lo, hi, shift=(0.0, 0.0, 0.0)):
    """Background positions of the cell centres, arrays in (k, j, i) order."""
    ax = [lo[a] + (np.arange(n[a]) + 0.5) * (hi[a] - lo[a]) / n[a] + shift[a] for a in range(3)]
    z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return x, y, z


def layout(t0):
    o = po.Oracle(interp_points=6, ko_eps=0.005, threads=4)
    ng, nl = (48, 48, 48), (48, 48, 48)
    o.add_patch(po.GLOBAL, ng, (-1, -1, -1), (1, 1, 1), po.BC_PERIODIC)
    o.add_patch(po.LOCAL, nl, (-0.5,) * 3, (0.5,) * 3, po.BC_INTERPATCH, po.STATIC, X0)
    o.time = t0
    xg = nodes(ng, (-1, -1, -1), (1, 1, 1))
    xl = nodes(nl, (-0.5,) * 3, (0.5,) * 3, X0)
    o.set_fields(0, *quad(*xg, t0))
    o.set_fields(1, *quad(*xl, t0))
    return o, xg, xl


def test_locals_step_with_the_methods_global_stage_states_is_exact():
    t0, dt = 0.3, 0.02
    o, xg, xl = layout(t0)
    psi, pi = quad(*xg, t0)
    # the global's RK4 stage states for K(psi, Pi) = (Pi, lap psi) = (Pi, 2)
    k = lambda s: (s[1], 2.0 + 0.0 * s[0])
    y1 = (psi, pi)
    k1 = k(y1)
    y2 = (psi + 0.5 * dt * k1[0], pi + 0.5 * dt * k1[1])
    k2 = k(y2)
    y3 = (psi + 0.5 * dt * k2[0], pi + 0.5 * dt * k2[1])
    k3 = k(y3)
    y4 = (psi + dt * k3[0], pi + dt * k3[1])
    o.step_locals(dt, [y1, y2, y3, y4])
    got = o.get_fields(1)
    want = quad(*xl, t0 + dt)
    # rounding only: the second differences divide values of order 0.4 by h^2
    scale = max(np.abs(want[0]).max(), np.abs(want[1]).max())
    for f in range(2):
        assert np.abs(got[f] - want[f]).max() < 1e-12 * scale
    assert o.time == t0 + dt
    # the global's own u is left as it was on its live cells (the flags poison
    # the dead ones, as in a step of the method)
    live = (o.get_flags() & 3) == po.LIVE
    np.testing.assert_array_equal(o.get_fields(0)[0][live], psi[live])


def test_locals_step_rejects_a_planted_stage_swap():
    """The same step with substages 1 and 2 of the global swapped is not exact
    (the Global-to-Local data then lag the interior stage states)."""
    t0, dt = 0.3, 0.02
    o, xg, xl = layout(t0)
    psi, pi = quad(*xg, t0)
    y1 = (psi, pi)
    y2 = (psi + 0.5 * dt * pi, pi + dt)
    y3 = (psi + 0.5 * dt * (pi + dt), pi + dt)
    y4 = (psi + dt * (pi + dt), pi + 2 * dt)
    o.step_locals(dt, [y1, y3, y2, y4])
    got = o.get_fields(1)
    want = quad(*xl, t0 + dt)
    assert np.abs(got[0] - want[0]).max() > 1e-9


def test_dead_cells_take_the_local_interpolant():
    t0 = 0.3
    o, xg, _ = layout(t0)
    o.compute_flags()
    o.fill_ghosts(t0)
    o.fill_dead(t0)
    ps, pq = o.get_padded(0, which=1)
    inner = (slice(po.NG, -po.NG),) * 3
    f = o.get_flags() & 3
    assert (f == po.DEAD).sum() > 100 and (f == po.GHOST).sum() > 100
    want = quad(*xg, t0)
    scale = np.abs(want[0]).max()
    for got, w in ((ps[inner], want[0]), (pq[inner], want[1])):
        assert np.isfinite(got).all()
        assert np.abs(got - w).max() < 1e-13 * scale


@pytest.mark.parametrize("lam", [1.0, -1.0, 1j])
def test_hermite_stage_weights_reproduce_rk4_stage_inputs(lam):
    errs = []
    for D in (0.2, 0.1):
        dt = D / 4.0
        y0, y1 = 1.0, np.exp(lam * D)
        data = (y0, lam * D * y0, (lam * D) ** 2 * y0, y1, lam * D * y1, (lam * D) ** 2 * y1)
        e = 0.0
        for m in range(4):
            u = np.exp(lam * m * dt)
            z = lam * dt
            exact = [u, u * (1 + z / 2), u * (1 + z / 2 + z * z / 4), u * (1 + z + z * z / 2 + z ** 3 / 4)]
            for l in range(4):
                w = so.hermite_stage_weights(m, l)
                e = max(e, abs(sum(wj * v for wj, v in zip(w, data)) - exact[l]))
        errs.append(e)
    assert errs[0] < 1e-6
    assert 40.0 < errs[0] / errs[1] < 90.0   # 2^6 = 64
