"""Hybrid stepping (mpw_step_surrogate): the learned surrogate advances the
periodic global patch four steps per call while the local patches stay on the
method, fed from the quintic Hermite interpolant in time of the global state,
and refill the global's covered cells at the start of every call.

What is pinned exactly: a call whose residual is above the tolerance is the
method's own four steps (bit for bit), and with no local patch an accepted
call is the surrogate's state (bit for bit).  The residual and the Laplacians
of the check kernel match the oracle.  With local patches the result is an
approximation of the method whose error is bounded here against the plain
run, and matches the oracle's hybrid call (oracle/surrogate.py hybrid_call,
pinned piece by piece in tests/test_oracle_hybrid.py); a trained network must
beat the untrained Taylor step.
"""
import numpy as np
import pytest

from oracle import surrogate as so
from paper_2002_00088_gb300 import workloads as wl
from tests.helpers import gpu_from, oracle_from

pytestmark = pytest.mark.gpu
SIGMA = 1e-4


@pytest.fixture(scope="module")
def sur_mod(mpw_lib):
    from paper_2002_00088_gb300 import surrogate
    return surrogate


def torch():
    import torch as t
    return t


def started(mpw_lib, w, globals_only=False):
    g = gpu_from(mpw_lib, wl.Workload(w.name, w.patches[:1] if globals_only else w.patches, w.analytic_kind,
                                      w.analytic_params, w.analytic_count, w.interp_points, w.ko_eps, w.dt, w.steps))
    g.fill_analytic(0.0)
    return g


def surrogate(sur_mod, w, params):
    return sur_mod.Surrogate(w.dt, 2.0 / w.patches[0].n[0], SIGMA, params=params)


def domain_errors(a, b, npatch):
    out = []
    for f in range(2):
        want = [b.get_fields(q)[f] for q in range(npatch)]
        got = [a.get_fields(q)[f] for q in range(npatch)]
        scale = max(np.nanmax(np.abs(x)) for x in want)
        out.append(max(np.nanmax(np.abs(x - y)) for x, y in zip(got, want)) / scale)
    return out


def test_calls_above_the_tolerance_are_the_plain_method(mpw_lib, sur_mod):
    w = wl.surrogate_layout(scale=2)
    a, b = started(mpw_lib, w), started(mpw_lib, w)
    acc, r = sur_mod.step_hybrid(a, surrogate(sur_mod, w, wl.surrogate_init(31)), w.dt, 3, tol=-1.0)
    b.step(w.dt, 12)
    assert acc == 0 and r > 0 and a.time == b.time
    for q in range(3):
        for x, y in zip(a.get_fields(q), b.get_fields(q)):
            np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(a.get_flags(), b.get_flags())


def test_global_only_calls_are_the_surrogate_state(mpw_lib, sur_mod):
    t = torch()
    w = wl.surrogate_layout(scale=2)
    a = started(mpw_lib, w, globals_only=True)
    n = w.patches[0].n
    u = [t.empty((n[2], n[1], n[0]), dtype=t.float64, device="cuda") for _ in range(2)]
    a.get_fields(0, out=u)
    sur = surrogate(sur_mod, w, wl.surrogate_init(32))
    acc, _ = sur_mod.step_hybrid(a, sur, w.dt, 3, tol=np.inf)
    for _ in range(3):
        u = sur.predict(u[0], u[1])
    assert acc == 3 and a.time == pytest.approx(12 * w.dt, rel=1e-14)
    got = a.get_fields(0)
    np.testing.assert_array_equal(got[0], u[0].cpu().numpy())
    np.testing.assert_array_equal(got[1], u[1].cpu().numpy())


def test_check_kernel_matches_oracle(sur_mod):
    t = torch()
    r = np.random.default_rng(33)
    shape = (2, 6, 8, 16)
    f = [r.standard_normal(shape) * s for s in (1.0, 20.0, 1.0, 20.0)]
    dt, h = 1.0 / 512, 2.0 / 128
    sur = sur_mod.Surrogate(dt, h, SIGMA)
    out, lap = sur.check(*[t.tensor(a).cuda() for a in f], want_laplacians=True)
    res, mx = so.residual(f[0], f[1], f[2], f[3], dt, h)
    np.testing.assert_allclose(out[:, 0].double().cpu().numpy(), res, rtol=1e-6)
    np.testing.assert_allclose(out[:, 1].double().cpu().numpy(), mx, rtol=1e-7)
    for k in range(4):
        np.testing.assert_array_equal(lap[k].cpu().numpy(), so.lap4(f[k], h))


def test_taylor_calls_with_local_patches_stay_close_to_the_method(mpw_lib, sur_mod):
    """Zero network (the Taylor step alone), two calls: the local patches run on
    Hermite-interpolated global data; errors against the plain run stay at the
    Taylor step's own level and the cover flags are the method's."""
    w = wl.surrogate_layout(scale=2)
    a, b = started(mpw_lib, w), started(mpw_lib, w)
    acc, _ = sur_mod.step_hybrid(a, surrogate(sur_mod, w, np.zeros(so.param_count(), np.float32)), w.dt, 2,
                                 tol=np.inf)
    b.step(w.dt, 8)
    assert acc == 2
    errs = domain_errors(a, b, 3)
    assert np.isfinite(errs).all() and max(errs) < 3e-3, errs
    np.testing.assert_array_equal(a.get_flags(), b.get_flags())
    assert a.time == b.time


def heldout_loss(sur, src, first, count):
    """Mean squared error of the network on `count` held-out pairs (no update)."""
    t = torch()
    n = src.n
    total = 0.0
    for k in range(count):
        u0 = [t.empty((1, n, n, n), dtype=t.float64, device="cuda") for _ in range(2)]
        u1 = [t.empty((1, n, n, n), dtype=t.float64, device="cuda") for _ in range(2)]
        src.pair(first + k, (u0[0][0], u0[1][0]), (u1[0][0], u1[1][0]))
        x, s = sur.features(u0[0], u0[1])
        tg = sur.targets(u0[0], u0[1], u1[0], u1[1], s)
        y = sur.forward(x)[..., :2]
        total += float(((y - tg) ** 2).mean())
    return total / count


@pytest.fixture(scope="module")
def trained(mpw_lib, sur_mod):
    """A network trained on 512 trajectories of the method on the 64^3
    periodic global of the half-size surrogate workload."""
    w = wl.surrogate_layout(scale=2)
    n = w.patches[0].n[0]
    src = sur_mod.Trajectories(n, w.dt)
    sur = sur_mod.Surrogate(w.dt, 2.0 / n, SIGMA, params=wl.surrogate_init(34))
    before = heldout_loss(sur, src, 90000, 4)
    losses = sur_mod.train(sur, src, trajectories=512, batch=2, lr=2e-3, lr_end=1e-4)
    return w, src, sur, before, heldout_loss(sur, src, 90000, 4), losses


def test_training_on_the_methods_trajectories_lowers_the_loss(trained):
    _, _, _, before, after, losses = trained
    assert np.isfinite(losses).all()
    assert after < 0.5 * before, (before, after)


def test_trained_network_beats_the_taylor_step(sur_mod, trained):
    """What the learned part gains: on held-out trajectories, one call's error
    against the method's own four steps is at least 2x below that of the same
    call with the network off (the Taylor step alone)."""
    t = torch()
    w, src, sur, _, _, _ = trained
    n = src.n
    off = sur_mod.Surrogate(w.dt, 2.0 / n, SIGMA, params=np.zeros(so.param_count(), np.float32))
    errs = {"trained": 0.0, "off": 0.0}
    for k in range(4):
        u0 = [t.empty((n, n, n), dtype=t.float64, device="cuda") for _ in range(2)]
        u1 = [t.empty((n, n, n), dtype=t.float64, device="cuda") for _ in range(2)]
        src.pair(80000 + k, u0, u1)
        scale = max(float(u1[0].abs().max()), 4 * w.dt * float(u1[1].abs().max()))
        for name, s in (("trained", sur), ("off", off)):
            p1, q1 = s.predict(u0[0], u0[1])
            e = max(float((p1 - u1[0]).abs().max()), 4 * w.dt * float((q1 - u1[1]).abs().max())) / scale
            errs[name] = max(errs[name], e)
    assert errs["trained"] * 2 < errs["off"], errs


def test_hybrid_calls_with_local_patches_match_the_oracle(mpw_lib, sur_mod):
    """Two network-off calls (the fourth-order Taylor step) on the half-size
    surrogate layout, two orbiting local patches: the device's hybrid against
    the oracle's hybrid call (flags and revival at the call's start, the
    Local-to-Global refill and the dead-cell fill, the surrogate's state, the
    local patches' four RK4 steps on the Hermite stage states, the global at
    the surrogate's state).  Every patch within 1e-11 of the domain maximum of
    each field; cover flags equal."""
    w = wl.surrogate_layout(scale=2)
    h = 2.0 / w.patches[0].n[0]
    a = started(mpw_lib, w)
    sur = surrogate(sur_mod, w, np.zeros(so.param_count(), np.float32))
    o = oracle_from(w)
    o.fill_analytic(0.0)
    for _ in range(2):
        acc, _ = sur_mod.step_hybrid(a, sur, w.dt, 1, tol=np.inf)
        assert acc == 1
        so.hybrid_call(o, None, w.dt, h, SIGMA)
    npatch = len(w.patches)
    np.testing.assert_array_equal(a.get_flags(), o.get_flags())
    # the library reads the global's ghost and dead cells as NaN; compare the
    # live ones there
    fl = a.get_flags() & 3
    live = (fl == 0) | (fl == 3)
    for f in range(2):
        want = [o.get_fields(q)[f] for q in range(npatch)]
        scale = max(np.nanmax(np.abs(x)) for x in want)
        for q in range(npatch):
            got = a.get_fields(q)[f]
            ref = want[q]
            if q == 0:
                assert np.isnan(got[~live]).all()
                got, ref = got[live], ref[live]
            assert np.isfinite(got).all()
            err = np.abs(got - ref).max() / scale
            assert err < 1e-11, (f, q, err)
    assert a.time == o.time
