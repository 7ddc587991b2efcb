"""Pins of the oracle's closed-form solutions (initial data and analytic BCs).

The plane-wave forms are the paper's own (Sec. 3, Eq. wave_solution; Sec.
3.4.2 superposition); the Gaussian pulse pair is checked against the wave
equation itself by finite differences of the closed form, and against its
initial data.
"""
import numpy as np
import pytest

from oracle import pyoracle as po


def cf(kind, params, count, t, x, y, z):
    return po.closed_form(kind, params, count, t, x, y, z)


def test_gauss_initial_data():
    prm = [1.3, 0.2, 0.1, -0.2, 0.05]
    pts = np.array([[0.1, -0.2, 0.05], [0.1 + 3e-6, -0.2, 0.05], [0.3, 0.0, 0.0], [-0.5, 0.4, 0.2]])
    ps, pv = cf(po.GAUSS_SUM, prm, 1, 0.0, pts[:, 0], pts[:, 1], pts[:, 2])
    r2 = ((pts - np.array(prm[2:])) ** 2).sum(1)
    np.testing.assert_allclose(ps, 1.3 * np.exp(-r2 / 0.04), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(pv, 0.0, atol=1e-13)


def test_gauss_series_branch_is_continuous():
    prm = [0.7, 0.15, 0.0, 0.0, 0.0]
    for t in [0.0, 0.05, 0.2]:
        a = cf(po.GAUSS_SUM, prm, 1, t, 0.99e-5, 0.0, 0.0)
        b = cf(po.GAUSS_SUM, prm, 1, t, 1.01e-5, 0.0, 0.0)
        assert abs(a[0] - b[0]) < 1e-9
        assert abs(a[1] - b[1]) < 1e-8


@pytest.mark.parametrize("t", [0.03, 0.11, 0.3])
def test_gauss_solves_wave_equation(t):
    """Pi = d psi/dt and dPi/dt = laplacian(psi), by 4th-order differences."""
    prm = [0.8, 0.3, 0.05, -0.1, 0.2, -0.4, 0.25, -0.3, 0.1, 0.0]
    x0 = np.array([0.31, 0.12, -0.07])
    d = 2e-3

    def psi(tt, x):
        return cf(po.GAUSS_SUM, prm, 2, tt, x[0], x[1], x[2])[0]

    def pi(tt, x):
        return cf(po.GAUSS_SUM, prm, 2, tt, x[0], x[1], x[2])[1]

    def d1(f, a, b):  # 4th-order first derivative from samples f(a +- k b)
        return (-f(a + 2 * b) + 8 * f(a + b) - 8 * f(a - b) + f(a - 2 * b)) / (12 * d)

    dpsi_dt = d1(lambda tt: float(psi(tt, x0)), t, d)
    assert abs(dpsi_dt - float(pi(t, x0))) < 1e-7
    dpi_dt = d1(lambda tt: float(pi(tt, x0)), t, d)
    lap = 0.0
    for a in range(3):
        e = np.zeros(3)
        e[a] = d
        f = [float(psi(t, x0 + k * e)) for k in (-2, -1, 0, 1, 2)]
        lap += (-f[0] + 16 * f[1] - 30 * f[2] + 16 * f[3] - f[4]) / (12 * d * d)
    assert abs(dpi_dt - lap) < 1e-5 * max(1.0, abs(lap))


def test_plane_wave_of_the_paper():
    """Sec. 3, Eq. wave_solution: phi = sin(2 pi (x - t) / L) + 2, L = 20."""
    L = 20.0
    prm = [2.0, 1.0, 2 * np.pi / L, 0.0, 0.0, 0.0]
    rng = np.random.default_rng(3)
    for _ in range(10):
        x, y, z, t = rng.uniform(-20, 20, 4)
        ps, pv = cf(po.PLANE_SUM, prm, 1, t, x, y, z)
        assert abs(ps - (np.sin(2 * np.pi / L * (x - t)) + 2.0)) < 1e-13
        assert abs(pv - (-2 * np.pi / L * np.cos(2 * np.pi / L * (x - t)))) < 1e-13


def test_superposition_of_the_paper():
    """Sec. 3.4.2: sin(2 pi (x - t)/L1) + cos(2 pi (x - y + z - sqrt(3) t)/L2) + 3."""
    L1, L2 = 20.0, 30.0
    k2 = 2 * np.pi / L2
    prm = [3.0, 1.0, 2 * np.pi / L1, 0.0, 0.0, 0.0, 1.0, k2, -k2, k2, np.pi / 2]
    rng = np.random.default_rng(4)
    for _ in range(10):
        x, y, z, t = rng.uniform(-20, 20, 4)
        ps, _ = cf(po.PLANE_SUM, prm, 2, t, x, y, z)
        want = np.sin(2 * np.pi / L1 * (x - t)) + np.cos(2 * np.pi / L2 * (x - y + z - np.sqrt(3) * t)) + 3
        assert abs(ps - want) < 1e-12


def test_harmonic_basis_is_harmonic_and_static():
    rng = np.random.default_rng(5)
    coef = rng.normal(size=14)
    x0 = rng.uniform(-1, 1, 3)
    d = 1e-2
    lap = 0.0
    for a in range(3):
        e = np.zeros(3)
        e[a] = d
        f = [float(cf(po.HARMONIC_POLY, coef, 14, 0.0, *(x0 + k * e))[0]) for k in (-2, -1, 0, 1, 2)]
        lap += (-f[0] + 16 * f[1] - 30 * f[2] + 16 * f[3] - f[4]) / (12 * d * d)
    assert abs(lap) < 1e-9  # the 5-point D2 is exact on quartics
    a = cf(po.HARMONIC_POLY, coef, 14, 0.0, *x0)
    b = cf(po.HARMONIC_POLY, coef, 14, 5.0, *x0)
    assert a[0] == b[0] and a[1] == 0.0
    # the basis as listed: 1, x, y, z, xy, yz, zx, x^2-y^2, y^2-z^2, xyz, x^3-3xy^2, ...
    x, y, z = x0
    basis = [1, x, y, z, x * y, y * z, z * x, x * x - y * y, y * y - z * z, x * y * z, x ** 3 - 3 * x * y * y,
             y ** 3 - 3 * y * z * z, z ** 3 - 3 * z * x * x, x ** 4 - 6 * x * x * y * y + y ** 4]
    assert abs(a[0] - np.dot(coef, basis)) < 1e-13


def test_circular_and_linear_motion():
    X0, w = po.motion(po.CIRCULAR, [0.1, -0.2, 0.3, 0.4, 2 * np.pi, 0.5], 0.125)
    ph = 2 * np.pi * 0.125 + 0.5
    np.testing.assert_allclose(X0, [0.1 + 0.4 * np.cos(ph), -0.2 + 0.4 * np.sin(ph), 0.3], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, [-0.8 * np.pi * np.sin(ph), 0.8 * np.pi * np.cos(ph), 0.0], atol=1e-14)
    X0, w = po.motion(po.LINEAR, [-5, -5, 0, 0.1, 0.1, 0], 20.0)  # Sec. 3.2 translating patch
    np.testing.assert_allclose(X0, [-3.0, -3.0, 0.0], atol=1e-14)
    np.testing.assert_array_equal(w, [0.1, 0.1, 0.0])


PLANE_GAUSS_PRM = [0.5, 0.7, 2 * np.pi, 3 * np.pi, 5 * np.pi, 0.3,   # plane wave k = (2, 3, 5) pi
                   1.1, 0.12, 0.05, -0.02, 0.01]                      # one Gaussian pulse


def test_plane_gauss_initial_data():
    """At t = 0: psi = C + A sin(k.x + phase) + A_g exp(-r^2/w^2); Pi = -A |k| cos(k.x + phase)."""
    p = PLANE_GAUSS_PRM
    rng = np.random.default_rng(7)
    k = np.array(p[2:5])
    for _ in range(8):
        x = rng.uniform(-1, 1, 3)
        ps, pv = cf(po.PLANE_GAUSS, p, 1, 0.0, *x)
        th = k @ x + p[5]
        r2 = ((x - np.array(p[8:11])) ** 2).sum()
        assert abs(ps - (p[0] + p[1] * np.sin(th) + p[6] * np.exp(-r2 / p[7] ** 2))) < 1e-13
        assert abs(pv - (-p[1] * np.linalg.norm(k) * np.cos(th))) < 1e-12


@pytest.mark.parametrize("t", [0.02, 0.07])
def test_plane_gauss_solves_wave_equation(t):
    """Pi = d psi/dt and dPi/dt = laplacian(psi), by 4th-order differences."""
    p = PLANE_GAUSS_PRM
    x0 = np.array([0.11, -0.07, 0.04])
    d = 1e-3

    def f(tt, x, which):
        return float(cf(po.PLANE_GAUSS, p, 1, tt, *x)[which])

    def d1(g, a):
        return (-g(a + 2 * d) + 8 * g(a + d) - 8 * g(a - d) + g(a - 2 * d)) / (12 * d)

    assert abs(d1(lambda tt: f(tt, x0, 0), t) - f(t, x0, 1)) < 1e-6
    lap = 0.0
    for a in range(3):
        e = np.zeros(3)
        e[a] = d
        v = [f(t, x0 + k * e, 0) for k in (-2, -1, 0, 1, 2)]
        lap += (-v[0] + 16 * v[1] - 30 * v[2] + 16 * v[3] - v[4]) / (12 * d * d)
    dpi = d1(lambda tt: f(tt, x0, 1), t)
    assert abs(dpi - lap) < 2e-4 * max(1.0, abs(lap))


def test_plane_gauss_plane_part_has_period_two():
    """k = (2, 3, 5) pi: the plane wave repeats with period 2 on every axis, so a
    periodic box [-1, 1]^3 holds it exactly (the Gaussian is switched off here)."""
    p = PLANE_GAUSS_PRM[:6] + [0.0, 0.12, 0.0, 0.0, 0.0]
    rng = np.random.default_rng(9)
    for _ in range(5):
        x = rng.uniform(-1, 1, 3)
        t = rng.uniform(0, 0.2)
        a = cf(po.PLANE_GAUSS, p, 1, t, *x)
        for ax in range(3):
            y = x.copy()
            y[ax] += 2.0
            b = cf(po.PLANE_GAUSS, p, 1, t, *y)
            assert abs(a[0] - b[0]) < 1e-12 and abs(a[1] - b[1]) < 1e-11
