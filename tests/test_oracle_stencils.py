"""Pins of the oracle's right-hand side (Sec. 2.2 Eqs. eom1-eom3 with the 4th-order
centred stencils; Sec. 2.3 Kreiss-Oliger dissipation, n = 5).

Polynomial exactness: D1 is exact through degree 4, D2 through degree 5 and
the KO sixth difference annihilates degree <= 5, so on such fields the RHS
must equal the analytic  K_psi = Pi + w.grad psi,  K_Pi = lap psi + w.grad Pi.
On x^6 the truncation terms are exact constants derived by hand below, which
fixes the KO sign and the 1/64 normalisation.
"""
import numpy as np
import pytest

from oracle import pyoracle as po

N = (8, 9, 10)
LO = (-0.3, 0.1, -1.0)
HI = (0.5, 0.7, 0.2)
NG = 3


def grids():
    h = [(HI[a] - LO[a]) / N[a] for a in range(3)]
    ax = [LO[a] + (np.arange(-NG, N[a] + NG) + 0.5) * h[a] for a in range(3)]
    z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return h, x, y, z


def make(w, eps):
    o = po.Oracle(interp_points=6, ko_eps=eps)
    motion = po.LINEAR if any(w) else po.STATIC
    o.add_patch(po.GLOBAL, N, LO, HI, po.BC_PERIODIC, motion, (0, 0, 0) + tuple(w))
    return o


def poly_terms(rng, degree):
    terms = []
    for _ in range(12):
        e = rng.integers(0, degree + 1, 3)
        while e.sum() > degree:
            e = rng.integers(0, degree + 1, 3)
        terms.append((rng.normal(), tuple(int(v) for v in e)))
    return terms


def ev(terms, x, y, z, d=(0, 0, 0)):
    """Value of sum c x^a y^b z^c, or of its derivative of orders d."""
    out = np.zeros_like(x)
    for c, e in terms:
        coef = c
        pw = []
        for k in range(3):
            p = e[k]
            for _ in range(d[k]):
                coef *= p
                p -= 1
            if p < 0:
                coef = 0.0
            pw.append(max(p, 0))
        out = out + coef * x ** pw[0] * y ** pw[1] * z ** pw[2]
    return out


@pytest.mark.parametrize("w", [(0.0, 0.0, 0.0), (0.3, -0.7, 1.1)])
def test_rhs_exact_on_polynomials(w):
    rng = np.random.default_rng(7)
    h, x, y, z = grids()
    ps_t = poly_terms(rng, 4)
    pi_t = poly_terms(rng, 4)
    o = make(w, 0.005)
    o.set_padded(0, ev(ps_t, x, y, z), ev(pi_t, x, y, z))
    kps, kpi = o.eval_rhs(0, 0.0)
    sl = (slice(NG, -NG),) * 3
    X, Y, Z = x[sl], y[sl], z[sl]
    grad_ps = [ev(ps_t, X, Y, Z, d) for d in ((1, 0, 0), (0, 1, 0), (0, 0, 1))]
    grad_pi = [ev(pi_t, X, Y, Z, d) for d in ((1, 0, 0), (0, 1, 0), (0, 0, 1))]
    lap = sum(ev(ps_t, X, Y, Z, d) for d in ((2, 0, 0), (0, 2, 0), (0, 0, 2)))
    want_ps = ev(pi_t, X, Y, Z) + sum(w[a] * grad_ps[a] for a in range(3))
    want_pi = lap + sum(w[a] * grad_pi[a] for a in range(3))
    scale = max(1.0, np.abs(want_pi).max())
    assert np.abs(kps - want_ps).max() < 1e-9 * scale
    assert np.abs(kpi - want_pi).max() < 1e-9 * scale


def test_ko_and_d2_truncation_on_x6():
    """On psi = x^6: the 6th difference is 720 h^6, so KO adds +(eps/64) 720 h^5
    (dissipative sign, Sec. 2.3 with n = 5), and D2 x^6 = 30 x^4 - 8 h^4."""
    eps = 0.005
    h, x, y, z = grids()
    o = make((0.0, 0.0, 0.0), eps)
    pi = 0.25 * np.ones_like(x)
    o.set_padded(0, x ** 6, pi)
    kps, kpi = o.eval_rhs(0, 0.0)
    sl = (slice(NG, -NG),) * 3
    X = x[sl]
    np.testing.assert_allclose(kps, 0.25 + eps / 64.0 * 720.0 * h[0] ** 5, rtol=0, atol=1e-12)
    np.testing.assert_allclose(kpi, 30.0 * X ** 4 - 8.0 * h[0] ** 4, rtol=0, atol=1e-10)


def test_non_live_points_are_nan_and_ghosts_unused():
    """The RHS is defined on interior points only; NaN ghosts must not matter
    for an interior point farther than 3 cells from the boundary."""
    h, x, y, z = grids()
    psi = np.cos(x + 2 * y - z)
    pi = np.sin(x - y)
    o = make((0.0, 0.0, 0.0), 0.005)
    o.set_padded(0, psi, pi)
    k_full = o.eval_rhs(0, 0.0)
    psi2 = psi.copy()
    psi2[:NG] = np.nan
    psi2[-NG:] = np.nan
    o.set_padded(0, psi2, pi)
    k_nan = o.eval_rhs(0, 0.0)
    # points >= 3 cells from the z faces see no NaN
    np.testing.assert_array_equal(k_nan[0][3:-3], k_full[0][3:-3])
    assert np.isnan(k_nan[1][0]).all()
