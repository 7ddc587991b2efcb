"""Exact discrete evolution of one Fourier mode on a periodic box.

For psi = Re(a e^{ik.x}), Pi = Re(b e^{ik.x}) the semi-discrete system of the
oracle (Sec. 2.2 RHS with 4th-order stencils, Sec. 2.3 KO) is the 2x2 linear
ODE d/dt (a, b) = A (a, b) with, per axis and theta = k_a h_a,
  D2 symbol  sigma = sum (-2 cos 2theta + 32 cos theta - 30) / (12 h^2)
  D1 symbol  i s,  s = (8 sin theta - sin 2 theta) / (6 h)
  KO symbol  kappa = -sum (eps/h) sin^6(theta/2)
  A = [[kappa + i w.s, 1], [sigma, kappa + i w.s]],
and one step of the printed Butcher tableau (Table 1, read from
tests/golden/rk4_tableau.txt) applied to that ODE is a 2x2 matrix M.  The
oracle must reproduce M^n to rounding.  This pins the stencil coefficients, the KO
sign and normalisation, the advection term, the Butcher tableau and the
periodic boundary fill at once.
"""
import numpy as np
import pytest

from oracle import pyoracle as po
from tests.golden_fixtures import rk4_tableau

N = (8, 10, 12)
LO = (-0.5, 0.0, 0.2)
HI = (0.5, 1.3, 0.9)
MODE = (1, 2, 3)
NG = 3


def rk4_matrix(A, dt):
    """One step of the explicit RK method of the printed tableau (Sec. 2.3,
    Table 1, tests/golden/rk4_tableau.txt) applied to the linear ODE v' = A v."""
    c, a, b = rk4_tableau()
    I = np.eye(2, dtype=complex)
    K = []
    for l in range(4):
        Y = I + dt * sum(a[l, m] * K[m] for m in range(l)) if l else I
        K.append(A @ Y)
    M = I + dt * sum(b[l] * K[l] for l in range(4))
    return M


def symbol(eps, w):
    h = np.array([(HI[a] - LO[a]) / N[a] for a in range(3)])
    L = np.array(HI) - np.array(LO)
    k = 2 * np.pi * np.array(MODE) / L
    th = k * h
    sigma = np.sum((-2 * np.cos(2 * th) + 32 * np.cos(th) - 30) / (12 * h * h))
    s = (8 * np.sin(th) - np.sin(2 * th)) / (6 * h)
    kappa = -np.sum(eps / h * np.sin(th / 2) ** 6)
    lam = kappa + 1j * np.dot(w, s)
    return np.array([[lam, 1.0], [sigma, lam]]), k, h


@pytest.mark.parametrize("eps,w", [(0.0, (0, 0, 0)), (0.005, (0, 0, 0)), (0.005, (0.7, -0.4, 1.3)),
                                   (0.3, (0.2, 0.0, -0.5))])
def test_single_mode_matches_rk4_matrix_power(eps, w):
    A, k, h = symbol(eps, np.array(w, float))
    ax = [LO[a] + (np.arange(N[a]) + 0.5) * h[a] for a in range(3)]
    z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    phase = np.exp(1j * (k[0] * x + k[1] * y + k[2] * z))
    v0 = np.array([0.8 - 0.3j, 0.2 + 1.1j])
    o = po.Oracle(interp_points=6, ko_eps=eps)
    motion = po.LINEAR if any(w) else po.STATIC
    o.add_patch(po.GLOBAL, N, LO, HI, po.BC_PERIODIC, motion, (0, 0, 0) + tuple(w))
    o.set_fields(0, (v0[0] * phase).real, (v0[1] * phase).real)
    dt = 0.2 * h.min()
    steps = 25
    o.step(dt, steps)
    vn = np.linalg.matrix_power(rk4_matrix(A, dt), steps) @ v0
    ps, pi = o.get_fields(0)
    want_ps = (vn[0] * phase).real
    want_pi = (vn[1] * phase).real
    assert np.abs(ps - want_ps).max() <= 1e-13 * np.abs(want_ps).max() + 1e-15
    assert np.abs(pi - want_pi).max() <= 1e-13 * np.abs(want_pi).max() + 1e-15
    assert abs(o.time - steps * dt) < 1e-15


def test_energy_of_a_mode_follows_rk4_amplification():
    """With eps = 0, w = 0 the discrete energy E_h = 1/2 h^3 sum(Pi^2 - psi D2 psi)
    of one mode is multiplied per step by |R(i y)|^2 = 1 - y^6/72 + y^8/576,
    y = omega_h dt, omega_h^2 = -sigma."""
    A, k, h = symbol(0.0, np.zeros(3))
    omega = np.sqrt(-A[1, 0].real)
    ax = [LO[a] + (np.arange(N[a]) + 0.5) * h[a] for a in range(3)]
    z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    phase = np.exp(1j * (k[0] * x + k[1] * y + k[2] * z))
    o = po.Oracle(interp_points=6, ko_eps=0.0)
    o.add_patch(po.GLOBAL, N, LO, HI, po.BC_PERIODIC)
    o.set_fields(0, (0.9 * phase).real, (0.4j * phase).real)
    dt = 0.35 * h.min()
    yv = omega * dt
    amp = 1 - yv ** 6 / 72 + yv ** 8 / 576
    e0 = o.energy(0)
    steps = 40
    o.step(dt, steps)
    assert abs(o.energy(0) / e0 - amp ** steps) < 1e-12
    assert amp < 1.0


def test_energy_decreases_with_dissipation():
    rng = np.random.default_rng(11)
    o = po.Oracle(interp_points=6, ko_eps=0.05)
    o.add_patch(po.GLOBAL, N, LO, HI, po.BC_PERIODIC)
    o.set_fields(0, rng.normal(size=(N[2], N[1], N[0])), rng.normal(size=(N[2], N[1], N[0])))
    h = min((HI[a] - LO[a]) / N[a] for a in range(3))
    e = [o.energy(0)]
    for _ in range(15):
        o.step(0.2 * h, 1)
        e.append(o.energy(0))
    assert all(b < a for a, b in zip(e, e[1:]))
