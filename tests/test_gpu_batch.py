"""Batched stepping (mpw_batch_*): several independent instances advanced with
one ghost-fill and one RHS launch per substage over all of them.  The batch
must reproduce, bit for bit, each instance stepped on its own, whether its
steps are launched directly or replayed from a captured CUDA graph; the
chunk-depth tuning that runs during the first steps must not change any
value."""
import numpy as np
import pytest

from paper_2002_00088_gb300 import workloads as wl
from tests.helpers import gpu_from

pytestmark = pytest.mark.gpu


def make_all(mpw, ws, precision):
    sims = []
    for w in ws:
        g = gpu_from(mpw, w, precision=precision)
        g.fill_analytic(0.0)
        sims.append(g)
    return sims


@pytest.mark.parametrize("precision", [64, 32])
def test_batch_matches_individual_steps(mpw_lib, precision):
    ws = wl.batch_instances(count=5, steps=12, seed_index=11, max_global=96)
    assert any(p.motion == wl.LINEAR and any(p.motion_params[3:6]) for w in ws for p in w.patches[1:])
    alone = make_all(mpw_lib, ws, precision)
    together = make_all(mpw_lib, ws, precision)
    steps = 10  # four tuning steps (chunk depths 8, 16, 32, 64), then the chosen depth
    for g, w in zip(alone, ws):
        g.step(w.dt, steps)
    b = mpw_lib.Batch(together)
    b.step([w.dt for w in ws], steps)
    zc, ms, launches, graph_steps = b.tuning()
    assert zc in (8, 16, 32, 64) and ms > 0.0
    # from the second step on (flags and exponent slots in place) the moving
    # instances' cover flags are batched too: a counter clear, the flags and
    # the revival, 3 launches per step
    assert launches == 8 * steps + 3 * (steps - 1)
    # after tuning, moving instances replay a captured graph too (grids padded
    # to a capacity; each step's arguments come from the page-locked buffers)
    assert graph_steps == steps - 4
    for g, h, w in zip(alone, together, ws):
        assert g.time == h.time
        np.testing.assert_array_equal(g.get_flags(), h.get_flags())
        for q in range(len(w.patches)):
            a, c = g.get_fields(q), h.get_fields(q)
            np.testing.assert_array_equal(a[0], c[0])
            np.testing.assert_array_equal(a[1], c[1])


def test_batch_rejects_mixed_precision(mpw_lib):
    ws = wl.batch_instances(count=2, steps=12, seed_index=12, max_global=64)
    a = gpu_from(mpw_lib, ws[0], precision=64)
    c = gpu_from(mpw_lib, ws[1], precision=32)
    with pytest.raises(mpw_lib.MpwError) as e:
        mpw_lib.Batch([a, c])
    assert e.value.status == 1


def test_static_batch_replays_a_captured_graph(mpw_lib):
    """Without moving patches the step is captured in a CUDA graph after the
    tuning steps; replaying it must give the same bits as stepping alone."""
    ws = [wl.static_gauss(interp_points=6), wl.plane_gauss(scale=8)]
    alone = make_all(mpw_lib, ws, 64)
    together = make_all(mpw_lib, ws, 64)
    steps = 9
    for g, w in zip(alone, ws):
        g.step(w.dt, steps)
    b = mpw_lib.Batch(together)
    b.step([w.dt for w in ws], 5)
    b.step([w.dt for w in ws], steps - 5)
    _, _, launches, graph_steps = b.tuning()
    assert launches == 8 * steps and graph_steps == steps - 4
    for g, h, w in zip(alone, together, ws):
        for q in range(len(w.patches)):
            a, c = g.get_fields(q), h.get_fields(q)
            np.testing.assert_array_equal(a[0], c[0])
            np.testing.assert_array_equal(a[1], c[1])


@pytest.mark.parametrize("precision", [64, 32])
def test_batch_with_rotating_instances_matches_individual_steps(mpw_lib, precision):
    """Rotating patches select the rotating-frame RHS kernels for the whole
    batch; the translating instances in it must still match their own steps
    bit for bit, and so must the rotating ones."""
    ws = wl.batch_instances(count=2, steps=12, seed_index=13, max_global=96)
    ws += [wl.rotating_plane(scale=2),
           wl.rotating_plane(scale=2, axis=(1.0, 2.0, 2.0), half_width=0.25, nl=16, omega=np.pi, phase=0.7,
                             velocity=(0.2, -0.1, 0.1))]
    alone = make_all(mpw_lib, ws, precision)
    together = make_all(mpw_lib, ws, precision)
    steps = 6
    for g, w in zip(alone, ws):
        g.step(w.dt, steps)
    b = mpw_lib.Batch(together)
    b.step([w.dt for w in ws], steps)
    for g, h, w in zip(alone, together, ws):
        assert g.time == h.time
        np.testing.assert_array_equal(g.get_flags(), h.get_flags())
        for q in range(len(w.patches)):
            a, c = g.get_fields(q), h.get_fields(q)
            np.testing.assert_array_equal(a[0], c[0])
            np.testing.assert_array_equal(a[1], c[1])


def test_failed_batch_step_leaves_instances_at_their_last_step(mpw_lib):
    """A batched step that one instance rejects (dt beyond its CFL bound) after
    the other instances' cover flags were prepared queues nothing, and leaves
    every instance as its last completed step left it: further batched steps
    give the same bits as a twin batch that never saw the failed calls."""
    # orbiting cubes cross about a third of a global cell per step, so the
    # covered boxes change between the steps around the failed calls
    ws = [wl.orbiting_gauss(scale=4, seed_index=k) for k in (1, 2, 3)]
    dts = [w.dt for w in ws]
    bad = dts[:-1] + [100.0]
    a = make_all(mpw_lib, ws, 64)
    twin = make_all(mpw_lib, ws, 64)
    ba, bt = mpw_lib.Batch(a), mpw_lib.Batch(twin)
    ba.step(dts, 2)  # cover flags and exponent slots in place: flags batched from here on
    bt.step(dts, 2)
    for _ in range(12):
        with pytest.raises(mpw_lib.MpwError) as e:
            ba.step(bad, 1)
        assert e.value.status in (mpw_lib.ERR_CFL, 4)  # CFL or traversal bound
        ba.step(dts, 1)
        bt.step(dts, 1)
    for g, h, w in zip(a, twin, ws):
        assert g.time == h.time
        np.testing.assert_array_equal(g.get_flags(), h.get_flags())
        for q in range(len(w.patches)):
            x, y = g.get_fields(q), h.get_fields(q)
            np.testing.assert_array_equal(x[0], y[0])
            np.testing.assert_array_equal(x[1], y[1])
