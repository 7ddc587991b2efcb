"""Pins of the surrogate layers' oracle (oracle/surrogate.py) against facts
that do not come from the oracle itself: brute-force loops on tiny volumes,
scipy's periodic correlation, the adjoint identity, finite differences,
Adam's closed form after one step, and torch's own bfloat16 rounding."""
import itertools

import numpy as np
import pytest

from oracle import surrogate as so
from paper_2002_00088_gb300 import workloads as wl


def rng(seed):
    return np.random.default_rng(seed)


def test_bf16_rounding_special_values():
    e = 2.0 ** -8
    cases = {
        1.0: 1.0,
        1.0 + e: 1.0,                       # halfway, ties to even (significand ...000)
        1.0 + 3 * e: 1.0 + 4 * e,           # halfway, ties to even (significand ...010)
        1.0 + e + 2.0 ** -20: 1.0 + 2 * e,  # above halfway rounds up
        -(1.0 + 3 * e): -(1.0 + 4 * e),
        (1.0 + 3 * e) * 2.0 ** 120: (1.0 + 4 * e) * 2.0 ** 120,  # the binary32 exponent range
        (1.0 + e) * 2.0 ** -120: 2.0 ** -120,
    }
    for x, want in cases.items():
        assert so.bf16(x) == pytest.approx(want, rel=1e-7), x


def test_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    x = rng(1).standard_normal(20000) * 10.0 ** rng(2).uniform(-20, 20, 20000)
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(so.bf16(x), want)
    np.testing.assert_array_equal(so.from_bf16_bits(so.bf16_bits(x)), want)


def brute_conv(x, W, b):
    B, n2, n1, n0, ci_n = x.shape
    co_n = W.shape[0]
    y = np.zeros((B, n2, n1, n0, co_n))
    for bb, z, yy, xx, co in itertools.product(range(B), range(n2), range(n1), range(n0), range(co_n)):
        s = b[co]
        for dz, dy, dx, ci in itertools.product(range(3), range(3), range(3), range(ci_n)):
            s += x[bb, (z + dz - 1) % n2, (yy + dy - 1) % n1, (xx + dx - 1) % n0, ci] * W[co, (dz * 3 + dy) * 3 + dx, ci]
        y[bb, z, yy, xx, co] = s
    return y


def test_conv3_matches_brute_force_loops():
    r = rng(3)
    x = r.standard_normal((2, 3, 4, 5, 2))
    W = r.standard_normal((3, 27, 2))
    b = r.standard_normal(3)
    np.testing.assert_allclose(so.conv3(x, W, b), brute_conv(x, W, b), rtol=0, atol=1e-12)
    np.testing.assert_allclose(so.conv3(x, W, b, relu=True), np.maximum(brute_conv(x, W, b), 0), atol=1e-12)


def test_conv3_matches_scipy_periodic_correlation():
    ndimage = pytest.importorskip("scipy.ndimage")
    r = rng(4)
    x = r.standard_normal((1, 6, 7, 8, 3))
    W = r.standard_normal((2, 27, 3))
    y = so.conv3(x, W)
    for co in range(2):
        want = sum(ndimage.correlate(x[0, ..., ci], W[co, :, ci].reshape(3, 3, 3), mode="wrap") for ci in range(3))
        np.testing.assert_allclose(y[0, ..., co], want, atol=1e-12)


def test_input_grad_is_the_adjoint():
    r = rng(5)
    x = r.standard_normal((2, 5, 4, 6, 3))
    W = r.standard_normal((4, 27, 3))
    gy = r.standard_normal((2, 5, 4, 6, 4))
    lhs = np.sum(so.conv3(x, W) * gy)
    rhs = np.sum(x * so.conv3_input_grad(gy, W))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)
    mask = r.standard_normal(x.shape)
    np.testing.assert_array_equal(so.conv3_input_grad(gy, W, mask)[mask <= 0], 0.0)


def test_weight_grad_matches_finite_differences():
    """L(W, b) = <conv3(x, W, b), gy> is linear in (W, b), so central differences
    are exact up to rounding."""
    r = rng(6)
    x = r.standard_normal((1, 4, 5, 3, 2))
    W = r.standard_normal((3, 27, 2))
    b = r.standard_normal(3)
    gy = r.standard_normal((1, 4, 5, 3, 3))
    gW, gb = so.conv3_weight_grad(x, gy)
    L = lambda W_, b_: np.sum(so.conv3(x, W_, b_) * gy)
    for idx in [(0, 0, 0), (2, 13, 1), (1, 26, 0), (0, 5, 1)]:
        d = np.zeros_like(W)
        d[idx] = 0.5
        assert (L(W + d, b) - L(W - d, b)) / 1.0 == pytest.approx(gW[idx], rel=1e-10, abs=1e-10)
    for co in range(3):
        d = np.zeros(3)
        d[co] = 0.5
        assert L(W, b + d) - L(W, b - d) == pytest.approx(gb[co], rel=1e-10, abs=1e-10)


def test_two_layer_chain_rule_matches_finite_differences():
    """The ReLU mask convention: gradient of sum(t * conv(relu(conv(x))))."""
    r = rng(7)
    x = r.standard_normal((1, 4, 4, 4, 2))
    W1 = r.standard_normal((3, 27, 2)) * 0.3
    b1 = r.standard_normal(3) * 0.1
    W2 = r.standard_normal((2, 27, 3)) * 0.3
    t = r.standard_normal((1, 4, 4, 4, 2))

    def loss(W1_):
        a = so.conv3(x, W1_, b1, relu=True)
        return np.sum(t * so.conv3(a, W2))

    a = so.conv3(x, W1, b1, relu=True)
    ga = so.conv3_input_grad(t, W2, mask=a)
    gW1, _ = so.conv3_weight_grad(x, ga)
    h = 1e-6
    for idx in [(0, 0, 0), (2, 13, 1), (1, 20, 0)]:
        d = np.zeros_like(W1)
        d[idx] = h
        fd = (loss(W1 + d) - loss(W1 - d)) / (2 * h)
        assert fd == pytest.approx(gW1[idx], rel=1e-6, abs=1e-8)


def test_adam_first_step_closed_form():
    """From m = v = 0 the bias-corrected moments are g and g^2, so the first
    update is lr * g / (|g| + eps)."""
    r = rng(8)
    w = r.standard_normal(100)
    g = r.standard_normal(100)
    lr, eps = 1e-3, 1e-8
    w1, m, v = so.adam(w, g, np.zeros(100), np.zeros(100), lr, 0.9, 0.999, eps, 1)
    np.testing.assert_allclose(w1, w - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m, 0.1 * g, atol=1e-16)
    # a constant gradient keeps the bias-corrected ratio at sign(g)
    w2, _, _ = so.adam(w1, g, m, v, lr, 0.9, 0.999, 0.0, 2)
    np.testing.assert_allclose(w2, w1 - lr * np.sign(g), atol=1e-15)


def test_mse_of_a_constant_offset():
    y = np.full((10, 2), 3.0)
    loss, g = so.mse(y + 0.5, y)
    assert loss == 0.25
    np.testing.assert_allclose(g, 2 * 0.5 / 20)


# ---------------------------------------------------------------- the surrogate's arithmetic

def mode(n, k, h):
    """A periodic Fourier mode on the grid x_i = (i + 1/2) h, shape (1, n2, n1, n0)."""
    ax = [(np.arange(m) + 0.5) * h for m in n]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return np.sin(k[0] * X + 0.3) * np.cos(k[1] * Y) * np.sin(k[2] * Z + 1.1)


def symbol(kh, h):
    """Eigenvalue of the 4th-order centred second difference on e^{i k x}."""
    return -(30.0 - 32.0 * np.cos(kh) + 2.0 * np.cos(2.0 * kh)) / (12.0 * h * h)


def test_lap4_of_a_fourier_mode_is_its_symbol():
    n = (16, 8, 12)
    h = 1.0 / 16
    k = [2 * np.pi * m / (n[a] * h) for a, m in enumerate((3, 2, 5))]
    u = mode(n, k, h)[None]
    lam = sum(symbol(k[a] * h, h) for a in range(3))
    np.testing.assert_allclose(so.lap4(u, h), lam * u, rtol=0, atol=1e-10 * abs(lam))


def test_taylor_step_with_zero_network_is_the_fourth_order_map():
    """With N = 0 one call maps a mode (psi, Pi) by the fourth-order Taylor
    polynomial of exp(D A), A = [[0, 1], [-l, 0]] (l = -symbol): since A^2 = -l I,
    T4 = (1 - D^2 l/2 + D^4 l^2/24) I + (D - D^3 l/6) A, i.e. one RK4 step."""
    n = (16, 8, 8)
    h, dt, sigma = 1.0 / 16, 0.01, 1e-3
    k = [2 * np.pi * m / (n[a] * h) for a, m in enumerate((1, 1, 2))]
    u = mode(n, k, h)[None]
    lam = -sum(symbol(k[a] * h, h) for a in range(3))
    D = 4 * dt
    c0 = 1 - D * D * lam / 2 + D ** 4 * lam * lam / 24
    c1 = D - D ** 3 * lam / 6
    psi0, pi0 = 0.7 * u, -1.3 * u
    y = np.zeros(u.shape + (2,))
    psi1, pi1 = so.apply(psi0, pi0, np.float32([2.0]), y, dt, h, sigma)
    np.testing.assert_allclose(psi1, c0 * psi0 + c1 * pi0, atol=1e-12)
    np.testing.assert_allclose(pi1, c0 * pi0 - lam * c1 * psi0, atol=1e-10)
    # one RK4 step of size D of the same linear system
    f = lambda p, q: (q, -lam * p)
    k1 = f(psi0, pi0)
    k2 = f(psi0 + D / 2 * k1[0], pi0 + D / 2 * k1[1])
    k3 = f(psi0 + D / 2 * k2[0], pi0 + D / 2 * k2[1])
    k4 = f(psi0 + D * k3[0], pi0 + D * k3[1])
    np.testing.assert_allclose(psi1, psi0 + D / 6 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0]), atol=1e-12)


def test_targets_recover_the_network_output():
    """targets(u0, apply(u0, N)) = N: the two definitions are inverse."""
    r = np.random.default_rng(9)
    h, dt, sigma = 1.0 / 32, 1.0 / 512, 1e-3
    psi0 = r.standard_normal((2, 8, 8, 16))
    pi0 = r.standard_normal((2, 8, 8, 16)) * 30
    _, s = so.features(psi0, pi0, dt, h)
    N = r.standard_normal((2, 8, 8, 16, 2))
    psi1, pi1 = so.apply(psi0, pi0, s, N, dt, h, sigma)
    np.testing.assert_allclose(so.targets(psi0, pi0, psi1, pi1, s, dt, h, sigma), N, rtol=1e-5, atol=1e-5)


def test_features_are_scale_invariant():
    r = np.random.default_rng(10)
    psi = r.standard_normal((1, 8, 8, 16))
    pi = r.standard_normal((1, 8, 8, 16))
    x1, s1 = so.features(psi, pi, 1e-3, 1.0 / 32)
    x2, s2 = so.features(psi * 2.0 ** 40, pi * 2.0 ** 40, 1e-3, 1.0 / 32)
    np.testing.assert_array_equal(x1, x2)
    assert s1[0] == s2[0] * 2.0 ** 40
    assert np.abs(x1[..., :2]).max() == 1.0 and x1.shape[-1] == 7


def test_network_gradient_matches_finite_differences():
    """Unrounded FP64 network: d loss / d params against central differences."""
    r = np.random.default_rng(11)
    x = r.standard_normal((1, 4, 4, 4, 7))
    t = r.standard_normal((1, 4, 4, 4, 2)) * 0.1
    p = wl.surrogate_init(12).astype(np.float64)
    loss, g = so.net_grads(x, p, t, rounded=False)
    layers = so.unpack_params(p)
    # probe one weight of each layer and one bias, in the flat padded layout
    offs, off = [], 0
    for (ci, co), (rc, ro, _) in zip(so.PADDED, so.LAYERS):
        offs.append(off + ((ro - 1) * 27 + 13) * ci + (rc - 1))
        offs.append(off + co * 27 * ci + 0)
        off += co * 27 * ci + co
    h = 1e-6
    for i in offs:
        d = np.zeros_like(p)
        d[i] = h
        fd = (so.net_grads(x, p + d, t, rounded=False)[0] - so.net_grads(x, p - d, t, rounded=False)[0]) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-9), i
    assert len(layers) == 4 and so.param_count() == p.size
    # padded entries carry no gradient
    W1 = np.zeros((32, 27, 8), bool)
    W1[:, :, 7:] = True
    assert (g[:W1.size][W1.ravel()] == 0).all()


def test_initial_parameters_follow_the_layout():
    p = wl.surrogate_init(3)
    assert p.size == so.param_count() and p.dtype == np.float32
    np.testing.assert_array_equal(so.pack_params(so.unpack_params(p)), p)


def test_quintic_hermite_reproduces_quintics():
    """The basis interpolates every polynomial of degree <= 5 exactly from its
    value and first two derivatives at both ends."""
    r = np.random.default_rng(13)
    c = r.standard_normal(6)
    p = np.polynomial.Polynomial(c)
    d1, d2 = p.deriv(1), p.deriv(2)
    for tau in np.linspace(0, 1, 11):
        w = so.hermite5(tau)
        val = w @ np.array([p(0), d1(0), d2(0), p(1), d1(1), d2(1)])
        assert val == pytest.approx(p(tau), abs=1e-13)


def test_residual_vanishes_on_a_discrete_standing_wave():
    """A standing mode of the semi-discrete system, psi = cos(w t) u(x),
    Pi = -w sin(w t) u(x) with w^2 = -symbol: the quadrature's error is O(D^5)."""
    n = (16, 16, 16)
    h = 1.0 / 16
    k = [2 * np.pi * 2 / (n[a] * h) for a in range(3)]
    u = mode(n, k, h)[None]
    w = np.sqrt(-sum(symbol(k[a] * h, h) for a in range(3)))
    for dt in (0.004, 0.002):
        D = 4 * dt
        r, m = so.residual(u, 0 * u, np.cos(w * D) * u, -w * np.sin(w * D) * u, dt, h)
        assert r[0] / m[0] <= (w * D) ** 5 / 100
