"""The learned surrogate (include/mpw_surrogate.h) against the numpy oracle.

Features, scales and training targets are defined to the bit (FP64
operations rounded once each, in a stated order) and must match exactly.
With all parameters zero the network output is zero and a surrogate call is
the Taylor step alone, so its result must match exactly too.  The network's
own output differs from the FP64 oracle by FP32 accumulation and the rare
bfloat16 rounding of a hidden activation that lands on the other side of a
tie; those comparisons use a tolerance.
"""
import numpy as np
import pytest

from oracle import surrogate as so
from paper_2002_00088_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

DT, H, SIGMA = 1.0 / 512, 2.0 / 128, 1e-4


@pytest.fixture(scope="module")
def sur_mod(mpw_lib):
    from paper_2002_00088_gb300 import surrogate
    return surrogate


def torch():
    import torch as t
    return t


def from_bf16(x):
    t = torch()
    return so.from_bf16_bits(x.view(t.int16).cpu().numpy().view(np.uint16))


def smooth_fields(seed, shape):
    """Random fields with a range of magnitudes (FP64)."""
    r = np.random.default_rng(seed)
    psi = r.standard_normal(shape) * 10.0 ** r.uniform(-2, 0, shape)
    pi = r.standard_normal(shape) * 30.0
    return psi, pi


SHAPES = [(2, 6, 8, 16), (1, 5, 16, 32)]


@pytest.mark.parametrize("shape", SHAPES)
def test_features_and_scales_are_exact(sur_mod, shape):
    t = torch()
    psi, pi = smooth_fields(1, shape)
    sur = sur_mod.Surrogate(DT, H, SIGMA)
    x, s = sur.features(t.tensor(psi).cuda(), t.tensor(pi).cuda())
    want_x, want_s = so.features(psi, pi, DT, H)
    np.testing.assert_array_equal(s.cpu().numpy(), want_s)
    got = from_bf16(x)
    np.testing.assert_array_equal(got[..., :7], want_x)
    assert (got[..., 7:] == 0).all()


@pytest.mark.parametrize("shape", SHAPES)
def test_targets_are_exact(sur_mod, shape):
    t = torch()
    psi0, pi0 = smooth_fields(2, shape)
    psi1, pi1 = smooth_fields(3, shape)
    sur = sur_mod.Surrogate(DT, H, SIGMA)
    d = [t.tensor(a).cuda() for a in (psi0, pi0, psi1, pi1)]
    _, s = sur.features(d[0], d[1])
    got = sur.targets(d[0], d[1], d[2], d[3], s).double().cpu().numpy()
    np.testing.assert_array_equal(got, so.targets(psi0, pi0, psi1, pi1, s.cpu().numpy(), DT, H, SIGMA))


def test_zero_network_call_is_the_taylor_step_exactly(sur_mod):
    t = torch()
    psi0, pi0 = smooth_fields(4, (2, 6, 8, 16))
    sur = sur_mod.Surrogate(DT, H, SIGMA, params=np.zeros(so.param_count(), np.float32))
    psi1, pi1 = sur.predict(t.tensor(psi0).cuda(), t.tensor(pi0).cuda())
    _, s = so.features(psi0, pi0, DT, H)
    want = so.apply(psi0, pi0, s, np.zeros(psi0.shape + (2,)), DT, H, SIGMA)
    np.testing.assert_array_equal(psi1.cpu().numpy(), want[0])
    np.testing.assert_array_equal(pi1.cpu().numpy(), want[1])


def test_forward_and_call_match_oracle(sur_mod):
    t = torch()
    psi0, pi0 = smooth_fields(5, (2, 6, 8, 16))
    params = wl.surrogate_init(21)
    sur = sur_mod.Surrogate(DT, H, SIGMA, params=params)
    d0, d1 = t.tensor(psi0).cuda(), t.tensor(pi0).cuda()
    x, s = sur.features(d0, d1)
    y = sur.forward(x).double().cpu().numpy()
    xo, so_ = so.features(psi0, pi0, DT, H)
    _, yo = so.net_forward(xo, params)
    scale = np.abs(yo).max()
    assert np.abs(y[..., :2] - yo).max() <= 1e-2 * scale
    assert np.median(np.abs(y[..., :2] - yo)) <= 1e-5 * scale
    assert (y[..., 2:] == 0).all()
    psi1, pi1 = sur.predict(d0, d1)
    want = so.apply(psi0, pi0, so_, yo, DT, H, SIGMA)
    for got, w, base in ((psi1, want[0], psi0), (pi1, want[1], pi0)):
        err = np.abs(got.cpu().numpy() - w).max()
        assert err <= 1e-6 * np.abs(base).max(), err


def test_train_step_gradients_and_update_match_oracle(sur_mod):
    t = torch()
    psi0, pi0 = smooth_fields(6, (1, 6, 8, 16))
    psi1, pi1 = smooth_fields(7, (1, 6, 8, 16))
    params = wl.surrogate_init(22)
    sur = sur_mod.Surrogate(DT, H, SIGMA, params=params)
    d = [t.tensor(a).cuda() for a in (psi0, pi0, psi1, pi1)]
    x, s = sur.features(d[0], d[1])
    tg = sur.targets(d[0], d[1], d[2], d[3], s)
    loss = sur.train_step(x, tg, lr=1e-3)
    g = sur.grads().astype(np.float64)
    want_loss, want_g = so.net_grads(from_bf16(x)[..., :7], params, tg.double().cpu().numpy())
    assert loss == pytest.approx(want_loss, rel=1e-4)
    off = 0
    for ci, co in so.PADDED:
        for size in (co * 27 * ci, co):
            a, b = g[off:off + size], want_g[off:off + size]
            assert np.linalg.norm(a - b) <= 1e-2 * np.linalg.norm(b) + 1e-30, (off, size)
            off += size
    # padded entries stay zero; the update is Adam's on the device's gradient
    upd, _, _ = so.adam(params.astype(np.float64), g, 0.0, 0.0, 1e-3, float(np.float32(0.9)),
                        float(np.float32(0.999)), float(np.float32(1e-8)), 1)
    after = sur.params().astype(np.float64)
    assert np.abs(after - upd).max() <= 1e-6
    assert (after[params == 0][np.asarray(want_g)[params == 0] == 0] == 0).all()
