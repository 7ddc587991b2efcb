"""Pins of the oracle's rotating patches (the rotating local patch of Sec. 3.2,
Test Two; map chain numeric -> background of Sec. 2.4).

A rotating patch maps X_B = R(t) X' + X0(t), R the rotation by
theta = Omega t + phase about a unit axis n.  What fixes each part, without
trusting the oracle's own formulas:

* R: scipy's rotation-vector routine, and for n = z the counter-clockwise
  plane rotation written out;
* the frame velocity w(X'): the time derivative of the map itself, taken by
  central differences and brought back to the patch frame (w = R^T dX_B/dt);
* the RHS in the rotating frame: on polynomial fields of degree <= 4 the
  stencils are exact, so K_psi and K_Pi must equal the background-frame
  chain rule  d/dt psi(X_B(X', t)) = Pi + grad psi . dX_B/dt  (and the same
  for Pi with the Laplacian), evaluated analytically with scipy's R;
* the interpolation through a rotated map: a polynomial of total degree <= 4
  stays one in rotated coordinates, so every ghost value filled by
  Global-to-Local and Local-to-Global equals the closed form at its
  background position (computed here with scipy's R);
* the cover flags: the covered set equals scipy's point-in-rotated-box test,
  a rotation by a quarter turn of a cube about its centre covers what the
  unrotated cube covers, zero angular speed is bitwise the translating
  patch, and the LIVE / GHOST / DEAD states match a brute-force distance;
* global accuracy: 4th-order convergence with the slope the paper reports
  for its rotating patch (tests/golden/convergence_slopes.txt).
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import pyoracle as po
from paper_2002_00088_gb300 import workloads as wl
from tests.golden_fixtures import key_values
from tests.helpers import oracle_from
from tests.test_oracle_flags import brute_force_states

NG = 3


def scipy_R(axis, theta):
    n = np.asarray(axis, float)
    return Rotation.from_rotvec(theta * n / np.linalg.norm(n)).as_matrix()


def rot_params(centre, velocity, axis, omega, phase):
    n = np.asarray(axis, float)
    n = n / np.linalg.norm(n)
    return tuple(centre) + tuple(velocity) + tuple(n) + (omega, phase)


def test_rotation_matches_scipy_and_the_plane_rotation():
    rng = np.random.default_rng(11)
    for _ in range(5):
        axis = rng.normal(size=3)
        mp = rot_params(rng.normal(size=3), rng.normal(size=3), axis, rng.normal(), rng.uniform(0, 6))
        t = rng.uniform(-2, 2)
        R, X0 = po.frame(po.ROTATING, mp, t)
        np.testing.assert_allclose(R, scipy_R(axis, mp[9] * t + mp[10]), atol=1e-15)
        np.testing.assert_allclose(X0, np.array(mp[:3]) + t * np.array(mp[3:6]), atol=1e-15)
    th = 0.7
    R, _ = po.frame(po.ROTATING, rot_params((0, 0, 0), (0, 0, 0), (0, 0, 1), 1.0, 0.0), th)
    want = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    np.testing.assert_allclose(R, want, atol=1e-16)
    # every other motion law has R = I
    R, X0 = po.frame(po.CIRCULAR, (0.1, 0.2, 0.3, 0.4, 2.0, 0.5), 0.3)
    np.testing.assert_array_equal(R, np.eye(3))


def test_frame_velocity_is_the_time_derivative_of_the_map():
    rng = np.random.default_rng(12)
    mp = rot_params((0.1, -0.2, 0.05), (0.3, -0.1, 0.2), (1.0, 2.0, -2.0), 2.5, 0.4)
    t, dt = 0.37, 1e-5
    for _ in range(5):
        xl = rng.uniform(-0.5, 0.5, 3)
        Rp, Xp = po.frame(po.ROTATING, mp, t + dt)
        Rm, Xm = po.frame(po.ROTATING, mp, t - dt)
        R, _ = po.frame(po.ROTATING, mp, t)
        xdot = ((Rp @ xl + Xp) - (Rm @ xl + Xm)) / (2 * dt)
        np.testing.assert_allclose(po.frame_velocity(po.ROTATING, mp, t, xl), R.T @ xdot, atol=1e-8)


def poly(c, X, Y, Z):
    """psi = c0 x^2 y + c1 y z^3 + c2 x z + c3 x^4 + c4, its gradient and Laplacian."""
    v = c[0] * X ** 2 * Y + c[1] * Y * Z ** 3 + c[2] * X * Z + c[3] * X ** 4 + c[4]
    g = (2 * c[0] * X * Y + c[2] * Z + 4 * c[3] * X ** 3,
         c[0] * X ** 2 + c[1] * Z ** 3,
         3 * c[1] * Y * Z ** 2 + c[2] * X)
    lap = 2 * c[0] * Y + 6 * c[1] * Y * Z + 12 * c[3] * X ** 2
    return v, g, lap


def test_rhs_in_a_rotating_frame_is_the_chain_rule():
    """K on a rotating patch equals d/dt of the background fields sampled at
    the moving nodes: K_psi = Pi + grad psi . Xdot, K_Pi = lap psi + grad Pi . Xdot."""
    axis, omega, phase, t = (0.3, -0.5, 0.8), 1.7, 0.2, 0.45
    mp = rot_params((0.05, -0.04, 0.02), (0.2, 0.1, -0.3), axis, omega, phase)
    o = po.Oracle(interp_points=6, ko_eps=0.005)
    o.add_patch(po.GLOBAL, (12, 12, 12), (-1, -1, -1), (1, 1, 1), po.BC_PERIODIC)
    n, lo, hi = (10, 11, 12), (-0.3, -0.25, -0.35), (0.3, 0.3, 0.25)
    o.add_patch(po.LOCAL, n, lo, hi, po.BC_INTERPATCH, po.ROTATING, mp)
    h = [(hi[a] - lo[a]) / n[a] for a in range(3)]
    ax = [lo[a] + (np.arange(-NG, n[a] + NG) + 0.5) * h[a] for a in range(3)]
    z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    R = scipy_R(axis, omega * t + phase)
    X0 = np.array(mp[:3]) + t * np.array(mp[3:6])
    xb = [R[a, 0] * x + R[a, 1] * y + R[a, 2] * z + X0[a] for a in range(3)]
    cps, cpi = (0.7, -0.4, 1.1, 0.3, 0.5), (-0.2, 0.6, 0.9, -0.5, 1.3)
    o.set_padded(1, poly(cps, *xb)[0], poly(cpi, *xb)[0])
    kps, kpi = o.eval_rhs(1, t)
    sl = (slice(NG, -NG),) * 3
    XB = [c[sl] for c in xb]
    om = omega * np.asarray(axis) / np.linalg.norm(axis)
    d = [XB[a] - X0[a] for a in range(3)]
    xdot = [om[1] * d[2] - om[2] * d[1] + mp[3], om[2] * d[0] - om[0] * d[2] + mp[4],
            om[0] * d[1] - om[1] * d[0] + mp[5]]
    ps, gps, lap = poly(cps, *XB)
    pi, gpi, _ = poly(cpi, *XB)
    want_ps = pi + sum(gps[a] * xdot[a] for a in range(3))
    want_pi = lap + sum(gpi[a] * xdot[a] for a in range(3))
    scale = max(np.abs(want_ps).max(), np.abs(want_pi).max())
    assert np.abs(kps - want_ps).max() < 1e-10 * scale
    assert np.abs(kpi - want_pi).max() < 1e-10 * scale


NGL, NLOC, HALF = 64, 40, 0.35


def harmonic_rotating(P, axis=(1.0, 2.0, 2.0), omega=1.3, phase=0.4, centre=(0.021, -0.017, 0.012)):
    o = po.Oracle(interp_points=P, ko_eps=0.005, threads=4)
    o.add_patch(po.GLOBAL, (NGL,) * 3, (-1, -1, -1), (1, 1, 1), po.BC_ANALYTIC)
    mp = rot_params(centre, (0.0, 0.0, 0.0), axis, omega, phase)
    o.add_patch(po.LOCAL, (NLOC,) * 3, (-HALF,) * 3, (HALF,) * 3, po.BC_INTERPATCH, po.ROTATING, mp)
    coef = np.random.default_rng(13).normal(size=14)
    o.set_analytic(po.HARMONIC_POLY, coef, 14)
    return o, mp, coef


@pytest.mark.parametrize("P", [5, 6])
def test_rotated_interpolation_is_exact_on_polynomials(P):
    o, mp, coef = harmonic_rotating(P)
    t = 0.6
    o.fill_analytic(t)
    o.compute_flags()
    o.fill_ghosts(t)
    R = scipy_R(mp[6:9], mp[9] * t + mp[10])
    X0 = np.array(mp[:3])
    # Global-to-Local: every ghost of the local patch
    ps, pi = o.get_padded(1, which=1)
    h = 2 * HALF / NLOC
    ax = -HALF + (np.arange(-NG, NLOC + NG) + 0.5) * h
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    xb = [R[a, 0] * x + R[a, 1] * y + R[a, 2] * z + X0[a] for a in range(3)]
    ex, _ = po.closed_form(po.HARMONIC_POLY, coef, 14, t, *xb)
    assert np.isfinite(ps).all()
    assert np.abs(ps - ex).max() < 1e-11 * np.abs(ex).max()
    assert np.abs(pi).max() < 1e-12 * np.abs(ex).max()
    # Local-to-Global: the effective ghost cells of the global patch
    gps, _ = o.get_padded(0, which=1)
    f = o.get_flags()
    ghost = (f & 3) == po.GHOST
    assert ghost.sum() > 100
    axg = -1 + (np.arange(NGL) + 0.5) * (2 / NGL)
    Z, Y, X = np.meshgrid(axg, axg, axg, indexing="ij")
    exg, _ = po.closed_form(po.HARMONIC_POLY, coef, 14, t, X[ghost], Y[ghost], Z[ghost])
    got = gps[NG:-NG, NG:-NG, NG:-NG][ghost]
    assert np.abs(got - exg).max() < 1e-11 * np.abs(ex).max()


def covered_by_scipy(mp, t, n_g, half, margin=1e-12):
    """Covered mask (global centres in the rotated closed box) and the cells
    within `margin` of a face, by scipy's R."""
    R = scipy_R(mp[6:9], mp[9] * t + mp[10])
    X0 = np.array(mp[:3]) + t * np.array(mp[3:6])
    ax = -1 + (np.arange(n_g) + 0.5) * (2 / n_g)
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    d = np.stack([X - X0[0], Y - X0[1], Z - X0[2]], -1)
    xl = d @ R  # R^T d
    inside = np.all(np.abs(xl) <= half, -1)
    near = np.any(np.abs(np.abs(xl) - half) < margin, -1)
    return inside, near


@pytest.mark.parametrize("axis,phase", [((0, 0, 1), 0.3), ((1.0, 2.0, 2.0), 1.1), ((-0.3, 0.1, 0.9), 2.0)])
def test_rotated_cover_flags(axis, phase):
    mp = rot_params((0.031, -0.042, 0.017), (0.0, 0.0, 0.0), axis, 0.8, phase)
    o = po.Oracle(interp_points=6)
    o.add_patch(po.GLOBAL, (64, 64, 64), (-1, -1, -1), (1, 1, 1), po.BC_ANALYTIC)
    o.add_patch(po.LOCAL, (36, 36, 36), (-0.3,) * 3, (0.3,) * 3, po.BC_INTERPATCH, po.ROTATING, mp)
    o.compute_flags()
    f = o.get_flags()
    cov = (f >> 2) == 1
    want, near = covered_by_scipy(mp, 0.0, 64, 0.3)
    assert not near.any()
    np.testing.assert_array_equal(cov, want)
    # brute-force distances inside the covered box widened by 9 cells (the
    # states only distinguish distances up to buffer + NG + 1 = 8)
    lo = np.maximum(np.argwhere(cov).min(0) - 9, 0)
    hi = np.minimum(np.argwhere(cov).max(0) + 10, 64)
    crop = tuple(slice(lo[a], hi[a]) for a in range(3))
    np.testing.assert_array_equal((f & 3)[crop], brute_force_states(cov[crop]))
    assert not cov[tuple(slice(None) for _ in range(3))].sum() - cov[crop].sum()
    assert ((f & 3) == po.GHOST).sum() > 0
    if axis == (0, 0, 1):  # a tilted cube of this size holds no cell at distance 8
        assert ((f & 3) == po.DEAD).sum() > 0


def test_quarter_turn_of_a_cube_covers_the_same_cells():
    centre = (0.0213, -0.0347, 0.0119)
    outs = []
    for motion, mp in ((po.STATIC, centre), (po.ROTATING, rot_params(centre, (0, 0, 0), (0, 0, 1), 0.0, np.pi / 2))):
        o = po.Oracle(interp_points=6)
        o.add_patch(po.GLOBAL, (32, 32, 32), (-1, -1, -1), (1, 1, 1), po.BC_ANALYTIC)
        o.add_patch(po.LOCAL, (16, 16, 16), (-0.25,) * 3, (0.25,) * 3, po.BC_INTERPATCH, motion, mp)
        o.compute_flags()
        outs.append(o.get_flags())
    np.testing.assert_array_equal(outs[0], outs[1])


def test_zero_angular_speed_is_the_translating_patch():
    w = wl.static_gauss(steps=2)
    c, v = (0.011, -0.013, 0.007), (0.2, -0.1, 0.15)
    outs = []
    for motion, mp in ((po.LINEAR, c + v), (po.ROTATING, rot_params(c, v, (0, 0, 1), 0.0, 0.0))):
        w.patches[1].motion = motion
        w.patches[1].motion_params = mp
        o = oracle_from(w)
        o.fill_analytic(0.0)
        o.step(w.dt, 2)
        outs.append((o.get_flags(), [o.get_fields(q) for q in range(2)]))
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    for a, b in zip(outs[0][1], outs[1][1]):
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])


def test_harmonic_polynomial_is_a_fixed_point_under_rotation():
    """Static harmonic field, rotating local patch: the local values are the
    field at moving nodes, so they change, but the global live data and the
    local data, compared with the closed form at the current map, stay exact
    up to the RK4 error of d/dt psi(X_B(X', t)) along the nodes."""
    o, mp, coef = harmonic_rotating(6, omega=0.5)
    o.fill_analytic(0.0)
    dt = 0.25 * 2 * HALF / NLOC
    o.step(dt, 4)
    t = o.time
    ps, _ = o.get_fields(0)
    f = o.get_flags() & 3
    live = (f == po.LIVE) | (f == po.REVIVED)
    axg = -1 + (np.arange(NGL) + 0.5) * (2 / NGL)
    Z, Y, X = np.meshgrid(axg, axg, axg, indexing="ij")
    ex, _ = po.closed_form(po.HARMONIC_POLY, coef, 14, t, X[live], Y[live], Z[live])
    assert np.abs(ps[live] - ex).max() < 1e-9 * np.abs(ex).max()
    lp, _ = o.get_fields(1)
    R = scipy_R(mp[6:9], mp[9] * t + mp[10])
    ax = -HALF + (np.arange(NLOC) + 0.5) * (2 * HALF / NLOC)
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    xb = [R[a, 0] * x + R[a, 1] * y + R[a, 2] * z + mp[a] for a in range(3)]
    exl, _ = po.closed_form(po.HARMONIC_POLY, coef, 14, t, *xb)
    assert np.abs(lp - exl).max() < 1e-7 * np.abs(exl).max()


def integrated_relative_error(w):
    o = oracle_from(w, threads=8)
    o.fill_analytic(0.0)
    o.step(w.dt, w.steps)
    total = 0.0
    for q, p in enumerate(w.patches):
        ps, _ = o.get_fields(q)
        h = [(p.hi[a] - p.lo[a]) / p.n[a] for a in range(3)]
        ax = [p.lo[a] + (np.arange(p.n[a]) + 0.5) * h[a] for a in range(3)]
        z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        if p.motion == po.ROTATING:
            mp = p.motion_params
            R = scipy_R(mp[6:9], mp[9] * o.time + mp[10])
            X0 = np.array(mp[:3]) + o.time * np.array(mp[3:6])
        else:
            R, X0 = np.eye(3), np.zeros(3)
        xb = [R[a, 0] * x + R[a, 1] * y + R[a, 2] * z + X0[a] for a in range(3)]
        ex, _ = po.closed_form(w.analytic_kind, w.analytic_params, w.analytic_count, o.time, *xb)
        live = np.isfinite(ps)
        total += np.sum(np.abs(ps[live] - ex[live]) / np.abs(ex[live])) * h[0] * h[1] * h[2]
    return total


def test_fourth_order_convergence_of_a_rotating_patch():
    """Sec. 3.2, Test Two, rotating local patch (reduced size, one revolution
    per unit time about z): the error must drop by ~16 per halving, slope
    within 0.3 of the paper's -4.05."""
    e1 = integrated_relative_error(wl.rotating_plane(scale=1))
    e2 = integrated_relative_error(wl.rotating_plane(scale=2))
    slope = -np.log2(e1 / e2)
    assert 11.0 < e1 / e2 < 22.0
    assert abs(slope - key_values("convergence_slopes.txt")["rotating"]) < 0.3
