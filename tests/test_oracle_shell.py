"""Pins of the oracle's spherical-shell local patches (the paper's spherical
local patch, Sec. 3.3: theta in [pi/4, 3 pi/4], full azimuth; flat metric in
spherical coordinates, appendix, with g_phiphi = r^2 sin^2 theta).

What fixes each part, without trusting the oracle's own formulas:

* the map (r, theta, phi) -> X_B and the node positions: the closed form
  written into the shell equals the closed form at positions computed here;
* coverage: numpy's test of r and theta on every global cell centre, and the
  LIVE / GHOST / DEAD states against scipy's chessboard distance transform
  (the covered set has a hole, so it is not convex);
* the RHS: exact on fields polynomial in r (the r stencils are exact there and
  the angular ones see constants), with the frame advection along r^; the
  Kreiss-Oliger terms on u = r^6, theta^6 and phi^6, whose sixth differences
  are exactly 720 h^6 (so the physical spacing of each axis shows); 4th-order
  convergence of the Laplacian and of the advection term on Cartesian
  polynomials, which are not polynomial in the angles;
* the fills: Global-to-Local ghosts (interpolation on the Cartesian global
  grid) exact for polynomials, azimuthal ghosts the periodic image;
  Local-to-Global (interpolation in (r, theta, phi)) converging at 6th order;
* global accuracy: 4th-order convergence of a multipatch run with a shell.
"""
import numpy as np
import pytest
from scipy.ndimage import distance_transform_cdt

from oracle import pyoracle as po
from paper_2002_00088_gb300 import workloads as wl
from tests.helpers import oracle_from

NG = 3
TH = (np.pi / 4, 3 * np.pi / 4)


def shell_nodes(n, r, th, padded=True):
    e = NG if padded else 0
    h = ((r[1] - r[0]) / n[0], (th[1] - th[0]) / n[1], 2 * np.pi / n[2])
    ax = [lo + (np.arange(-e, m + e) + 0.5) * hh for lo, m, hh in zip((r[0], th[0], 0.0), n, h)]
    P, T, R = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return R, T, P, h


def cart(R, T, P, X0=(0.0, 0.0, 0.0)):
    return (R * np.sin(T) * np.cos(P) + X0[0], R * np.sin(T) * np.sin(P) + X0[1], R * np.cos(T) + X0[2])


def one_shell(n=(10, 12, 40), r=(0.3, 0.6), centre=(0.011, -0.007, 0.013), motion=po.STATIC, mp=None, eps=0.005,
              global_n=32, P=6):
    o = po.Oracle(interp_points=P, ko_eps=eps, threads=4)
    o.add_patch(po.GLOBAL, (global_n,) * 3, (-1, -1, -1), (1, 1, 1), po.BC_ANALYTIC)
    o.add_patch(po.LOCAL, n, (r[0], TH[0], 0.0), (r[1], TH[1], 2 * np.pi), po.BC_INTERPATCH, motion,
                mp if mp is not None else centre, po.SPHERICAL)
    return o


def test_shell_initial_data_is_the_closed_form_at_the_mapped_nodes():
    n, r, X0 = (10, 12, 40), (0.3, 0.6), (0.011, -0.007, 0.013)
    o = one_shell(n, r, X0)
    coef = np.random.default_rng(21).normal(size=14)
    o.set_analytic(po.HARMONIC_POLY, coef, 14)
    o.fill_analytic(0.0)
    R, T, P, _ = shell_nodes(n, r, TH, padded=False)
    ex, _ = po.closed_form(po.HARMONIC_POLY, coef, 14, 0.0, *cart(R, T, P, X0))
    ps, _ = o.get_fields(1)
    np.testing.assert_allclose(ps, ex, rtol=0, atol=1e-14 * np.abs(ex).max())


def test_shell_validation():
    o = po.Oracle(interp_points=6)
    o.add_patch(po.GLOBAL, (16,) * 3, (-1, -1, -1), (1, 1, 1), po.BC_ANALYTIC)
    for lo, hi in (((0.3, 0.05, 0.0), (0.6, 2.0, 2 * np.pi)),   # ghosts reach the pole
                   ((0.3, 0.5, 0.0), (0.6, 2.0, np.pi)),        # not the full azimuth
                   ((0.01, 0.5, 0.0), (0.6, 2.0, 2 * np.pi))):  # ghosts reach the origin
        with pytest.raises(po.OracleError):
            o.add_patch(po.LOCAL, (10, 10, 20), lo, hi, po.BC_INTERPATCH, po.STATIC, (0, 0, 0), po.SPHERICAL)


@pytest.mark.parametrize("centre", [(0.011, -0.007, 0.013), (0.2, 0.1, -0.15)])
def test_shell_cover_flags(centre):
    ng, r = 64, (0.25, 0.7)
    o = one_shell((16, 24, 64), r, centre, global_n=ng)
    o.compute_flags()
    f = o.get_flags()
    cov = (f >> 2) == 1
    ax = -1 + (np.arange(ng) + 0.5) * (2 / ng)
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    x, y, z = X - centre[0], Y - centre[1], Z - centre[2]
    rr = np.sqrt(x * x + y * y + z * z)
    th = np.arccos(np.clip(z / rr, -1, 1))
    want = (rr >= r[0]) & (rr <= r[1]) & (th >= TH[0]) & (th <= TH[1])
    near = (np.minimum(np.abs(rr - r[0]), np.abs(rr - r[1])) < 1e-12) | (
        np.minimum(np.abs(th - TH[0]), np.abs(th - TH[1])) < 1e-12)
    assert not near.any()
    np.testing.assert_array_equal(cov, want)
    # L-infinity distance to the nearest uncovered cell by scipy's chessboard
    # transform (a border of uncovered cells: outside the grid is uncovered)
    d = distance_transform_cdt(np.pad(cov, 1), metric="chessboard")[1:-1, 1:-1, 1:-1]
    want_states = np.where(d <= 4, po.LIVE, np.where(d <= 7, po.GHOST, po.DEAD))
    np.testing.assert_array_equal(f & 3, want_states)
    assert ((f & 3) == po.GHOST).sum() > 0


def radial(c, R):
    """u = c0 + c1 r^2 + c2 r^4, u_r, u_rr."""
    return c[0] + c[1] * R ** 2 + c[2] * R ** 4, 2 * c[1] * R + 4 * c[2] * R ** 3, 2 * c[1] + 12 * c[2] * R ** 2


@pytest.mark.parametrize("velocity", [(0.0, 0.0, 0.0), (0.3, -0.2, 0.4)])
def test_shell_rhs_exact_on_radial_polynomials(velocity):
    n, r, X0 = (10, 12, 40), (0.3, 0.6), (0.011, -0.007, 0.013)
    mp = tuple(X0) + tuple(velocity)
    o = one_shell(n, r, motion=po.LINEAR, mp=mp)
    R, T, P, _ = shell_nodes(n, r, TH)
    cps, cpi = (0.4, -1.3, 2.1), (0.7, 0.9, -0.6)
    o.set_padded(1, radial(cps, R)[0], radial(cpi, R)[0])
    kps, kpi = o.eval_rhs(1, 0.0)
    sl = (slice(NG, -NG),) * 3
    Rr, Tt, Pp = R[sl], T[sl], P[sl]
    rhat = np.stack([np.sin(Tt) * np.cos(Pp), np.sin(Tt) * np.sin(Pp), np.cos(Tt)])
    wr = np.tensordot(np.asarray(velocity), rhat, 1)
    ps, ps_r, ps_rr = radial(cps, Rr)
    pi, pi_r, _ = radial(cpi, Rr)
    want_ps = pi + wr * ps_r
    want_pi = ps_rr + 2 * ps_r / Rr + wr * pi_r
    scale = max(np.abs(want_ps).max(), np.abs(want_pi).max())
    assert np.abs(kps - want_ps).max() < 1e-11 * scale
    assert np.abs(kpi - want_pi).max() < 1e-11 * scale


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_shell_ko_over_the_physical_spacing(axis):
    """u = q^6 along one numeric axis q: the sixth difference is 720 h^6, so
    KO adds (eps/64) 720 h^6 / L with L = h_r, r h_theta or r sin(theta) h_phi."""
    eps = 0.005
    n, r = (10, 12, 40), (0.3, 0.6)
    o = one_shell(n, r, eps=eps)
    R, T, P, h = shell_nodes(n, r, TH)
    q = (R, T, P)[axis]
    o.set_padded(1, q ** 6, 0.25 * np.ones_like(R))
    kps, _ = o.eval_rhs(1, 0.0)
    sl = (slice(NG, -NG),) * 3
    L = (h[0] * np.ones_like(R), R * h[1], R * np.sin(T) * h[2])[axis][sl]
    np.testing.assert_allclose(kps, 0.25 + eps / 64 * 720 * h[axis] ** 6 / L, rtol=1e-9, atol=0)


def cart_poly(X, Y, Z):
    """psi = x^2 y + y z^2 - 0.5 x z + 0.3 x^3: value, gradient, Laplacian."""
    v = X ** 2 * Y + Y * Z ** 2 - 0.5 * X * Z + 0.3 * X ** 3
    g = (2 * X * Y - 0.5 * Z + 0.9 * X ** 2, X ** 2 + Z ** 2, 2 * Y * Z - 0.5 * X)
    lap = 2 * Y + 2 * Y + 1.8 * X
    return v, g, lap


def shell_rhs_error(scale):
    """Max errors of K_Pi (Laplacian) and K_psi (frame advection) on a
    Cartesian polynomial, rotating shell, eps = 0."""
    n, r = (10 * scale, 12 * scale, 40 * scale), (0.3, 0.6)
    axis = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    mp = (0.01, -0.02, 0.015, 0.1, 0.2, -0.1) + tuple(axis) + (1.7, 0.4)
    o = one_shell(n, r, motion=po.ROTATING, mp=mp, eps=0.0)
    R, T, P, _ = shell_nodes(n, r, TH)
    x = cart(R, T, P)
    o.set_padded(1, cart_poly(*x)[0], np.zeros_like(R))
    t = 0.3
    kps, kpi = o.eval_rhs(1, t)
    sl = (slice(NG, -NG),) * 3
    xs = [c[sl] for c in x]
    _, g, lap = cart_poly(*xs)
    w = np.stack([po.frame_velocity(po.ROTATING, mp, t, p) for p in np.stack(xs, -1).reshape(-1, 3)])
    w = w.reshape(xs[0].shape + (3,))
    adv = sum(w[..., a] * g[a] for a in range(3))
    return np.abs(kpi - lap).max() / np.abs(lap).max(), np.abs(kps - adv).max() / np.abs(adv).max()


def test_shell_rhs_converges_at_fourth_order():
    e1 = shell_rhs_error(1)
    e2 = shell_rhs_error(2)
    for a, b in zip(e1, e2):
        assert 11.0 < a / b < 22.0, (e1, e2)


def test_shell_fills():
    """G2L (Cartesian donors) exact on a harmonic polynomial; azimuthal ghosts
    the periodic image; L2G (donors on the shell) converging at 6th order."""
    errs = []
    for scale in (1, 2):
        n, r, X0 = (12 * scale, 16 * scale, 48 * scale), (0.25, 0.7), (0.011, -0.007, 0.013)
        o = one_shell(n, r, X0, global_n=64)
        coef = np.random.default_rng(22).normal(size=14)
        o.set_analytic(po.HARMONIC_POLY, coef, 14)
        o.fill_analytic(0.0)
        o.compute_flags()
        o.fill_ghosts(0.0)
        ps, _ = o.get_padded(1, which=1)
        R, T, P, _ = shell_nodes(n, r, TH)
        ex, _ = po.closed_form(po.HARMONIC_POLY, coef, 14, 0.0, *cart(R, T, P, X0))
        assert np.isfinite(ps).all()
        assert np.abs(ps - ex).max() < 1e-12 * np.abs(ex).max()
        gps, _ = o.get_padded(0, which=1)
        f = o.get_flags()
        ghost = (f & 3) == po.GHOST
        assert ghost.sum() > 0
        ax = -1 + (np.arange(64) + 0.5) * (2 / 64)
        Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
        exg, _ = po.closed_form(po.HARMONIC_POLY, coef, 14, 0.0, X[ghost], Y[ghost], Z[ghost])
        errs.append(np.abs(gps[NG:-NG, NG:-NG, NG:-NG][ghost] - exg).max() / np.abs(ex).max())
    assert errs[0] / errs[1] > 30.0, errs


def integrated_relative_error(w):
    o = oracle_from(w, threads=8)
    o.fill_analytic(0.0)
    o.step(w.dt, w.steps)
    total = 0.0
    for q, p in enumerate(w.patches):
        ps, _ = o.get_fields(q)
        if p.topology == po.SPHERICAL:
            R, T, P, h = shell_nodes(p.n, (p.lo[0], p.hi[0]), (p.lo[1], p.hi[1]), padded=False)
            x = cart(R, T, P, p.motion_params[:3])
            vol = R ** 2 * np.sin(T) * h[0] * h[1] * h[2]
        else:
            h = [(p.hi[a] - p.lo[a]) / p.n[a] for a in range(3)]
            ax = [p.lo[a] + (np.arange(p.n[a]) + 0.5) * h[a] for a in range(3)]
            z, y, xx = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
            x = (xx, y, z)
            vol = h[0] * h[1] * h[2]
        ex, _ = po.closed_form(w.analytic_kind, w.analytic_params, w.analytic_count, o.time, *x)
        live = np.isfinite(ps)
        total += np.sum((np.abs(ps - ex) / np.abs(ex) * vol)[live])
    return total


def test_fourth_order_convergence_with_a_shell():
    e1 = integrated_relative_error(wl.shell_plane(scale=1))
    e2 = integrated_relative_error(wl.shell_plane(scale=2))
    assert 11.0 < e1 / e2 < 22.0, (e1, e2)
