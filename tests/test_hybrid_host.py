"""Host logic of hybrid stepping (no GPU): the weights that rebuild the global
patch's RK4 stage inputs from the quintic Hermite interpolant of a call.

Pin: for y' = lam y (one mode of the linear system) the interpolant of the
exact solution is within O((lam Delta)^6) of it, and the weights must then
reproduce the stage inputs that RK4 itself forms from the exact state at the
start of each step, u, u + dt/2 k1, u + dt/2 k2, u + dt k3 -- computed here by
running the stages, not from the weights' formula."""
import ctypes

import numpy as np
import pytest


def weights(mpw, m, l, delta):
    w = (ctypes.c_double * 6)()
    assert mpw.lib.mpw_sur_stage_weights(m, l, float(delta), w) == 0
    return np.array(list(w))


def rk4_stage_inputs(u, lam, dt):
    f = lambda y: lam * y
    k1 = f(u)
    y2 = u + dt / 2 * k1
    y3 = u + dt / 2 * f(y2)
    y4 = u + dt * f(y3)
    return [u, y2, y3, y4]


@pytest.mark.parametrize("lam", [1.0j * 3.0, -2.0, 1.0j * 1.5 - 0.3])
def test_stage_weights_reproduce_rk4_stage_inputs(mpw_lib, lam):
    delta = 0.05
    dt = delta / 4
    y = lambda t: np.exp(lam * t)
    ends = np.array([y(0), lam * y(0), lam ** 2 * y(0), y(delta), lam * y(delta), lam ** 2 * y(delta)])
    for m in range(4):
        want = rk4_stage_inputs(y(m * dt), lam, dt)
        for l in range(4):
            got = weights(mpw_lib, m, l, delta) @ ends
            # interpolation error of the quintic Hermite: O((|lam| delta)^6)
            assert abs(got - want[l]) <= 5e-9, (m, l, abs(got - want[l]))


def test_stage_weights_keep_constants_and_start_from_the_state(mpw_lib):
    """A constant state has every stage input equal to it: the value weights
    sum to one at every stage.  The first stage of the first step is y0."""
    np.testing.assert_array_equal(weights(mpw_lib, 0, 0, 0.1), [1, 0, 0, 0, 0, 0])
    for m in range(4):
        for l in range(4):
            w = weights(mpw_lib, m, l, 0.1)
            assert abs(w[0] + w[3] - 1.0) < 1e-14, (m, l)


def test_stage_weights_reject_bad_indices(mpw_lib):
    w = (ctypes.c_double * 6)()
    assert mpw_lib.lib.mpw_sur_stage_weights(4, 0, 0.1, w) == 1
    assert mpw_lib.lib.mpw_sur_stage_weights(0, -1, 0.1, w) == 1
