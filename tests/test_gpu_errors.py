"""Device-side error paths, driven without faulting, trapping or hanging the GPU.

- Bounded waits.  Every mbarrier wait of the RHS kernels' TMA pipeline is
  bounded; mpw_set_wait_limit(0) makes each one give up at its first try, so
  the kernels take their timeout path (set the error word, drain their own
  copies in flight with the full limit, return) and mpw_step reports
  MPW_ERR_TIMEOUT.  Afterwards the context must still work: restored from its
  checkpoint, it steps to the same result as the oracle.
- Skipped ghost points (Sec. 2.4.1: a point that cannot be interpolated keeps
  its lower-priority value and is counted).  Injected on the host through
  mpw_set_flags: a global cell far outside a rotated local cube, but inside
  that cube's bounding box, is marked as the cube's effective ghost.  The
  Local-to-Global pass of a rotated patch visits exactly such cells; the
  window of this one falls outside the local interior, which the fill checks
  before it reads any donor, so it is skipped and mpw_step reports
  MPW_ERR_GHOST_UNFILLED.
"""
import os

import numpy as np
import pytest

from paper_2002_00088_gb300 import workloads as wl
from tests.helpers import gpu_from, oracle_from

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1


def fields_from(o, npatch):
    o.fill_analytic(0.0)
    return [o.get_fields(q) for q in range(npatch)]


def max_rel(got, want):
    out = 0.0
    for f in range(2):
        scale = max(np.nanmax(np.abs(w[f])) for w in want)
        for a, b in zip(got, want):
            m = np.isfinite(b[f])
            assert np.array_equal(np.isfinite(a[f]), m)
            out = max(out, float(np.abs(a[f][m] - b[f][m]).max()) / scale)
    return out


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("make", [lambda: wl.orbiting_gauss(scale=4), lambda: wl.static_gauss()],
                         ids=["orbiting", "static"])
def test_expired_wait_reports_timeout_and_context_recovers(mpw_lib, make, precision):
    w = make()
    npatch = len(w.patches)
    o = oracle_from(w, THREADS)
    init = fields_from(o, npatch)
    g = gpu_from(mpw_lib, w, precision=precision)
    for q in range(npatch):
        g.set_fields(q, *init[q])
    g.time = 0.0
    g.set_wait_limit(0)
    with pytest.raises(mpw_lib.MpwError) as e:
        g.step(w.dt, 1)
    assert e.value.status == mpw_lib.ERR_TIMEOUT
    assert "wait ran out" in str(e.value)
    # back to the default limit and to the checkpoint (fields and time; the
    # flags of t = 0 are recomputed or still valid)
    g.set_wait_limit(1 << 20)
    for q in range(npatch):
        g.set_fields(q, *init[q])
    g.time = 0.0
    g.step(w.dt, 2)
    o.step(w.dt, 2)
    got = [g.get_fields(q) for q in range(npatch)]
    want = [o.get_fields(q) for q in range(npatch)]
    err = max_rel(got, want)
    # binary64: the parity bar; binary32: well inside its rounding bound
    # (tests/test_gpu_fp32.py) for two steps at h = 1/64
    assert err <= (1e-12 if precision == 64 else 2e-4), err
    np.testing.assert_array_equal(g.get_flags(), o.get_flags())


def test_injected_unfillable_ghost_is_reported(mpw_lib):
    # a local cube turned by pi/4 about z, not moving: its flags are computed
    # once and the flags set through the ABI stay in force for the step
    w = wl.rotating_plane(scale=1, omega=0.0, phase=np.pi / 4)
    g = gpu_from(mpw_lib, w)
    g.fill_analytic(0.0)
    g.compute_flags()
    flags = g.get_flags()
    # global cell (22, 22, 16): centre (0.406, 0.406, 0.031), inside the
    # bounding box |x|, |y| <= 0.3 sqrt(2) of the turned cube but 0.57 from its
    # axis along x', i.e. about 9 local cells outside the local interior
    k, j, i = 16, 22, 22
    h = 2.0 / 32
    x = -1.0 + (np.array([i, j, k]) + 0.5) * h
    xl = np.array([(x[0] + x[1]) / np.sqrt(2.0), (x[1] - x[0]) / np.sqrt(2.0), x[2]])
    assert np.abs(xl).max() > 0.3 + 3 * 0.03 and np.abs(x[:2]).max() < 0.3 * np.sqrt(2.0)
    assert flags[k, j, i] & 3 == mpw_lib.FLAG_LIVE
    bad = flags.copy()
    bad[k, j, i] = mpw_lib.FLAG_GHOST | (1 << 2)
    g.set_flags(bad)
    with pytest.raises(mpw_lib.MpwError) as e:
        g.step(w.dt, 1)
    assert e.value.status == mpw_lib.ERR_GHOST_UNFILLED
    # the error word was cleared when it was read: with the true flags back the
    # context steps without error
    g.fill_analytic(0.0)
    g.set_flags(flags)
    g.step(w.dt, 1)
