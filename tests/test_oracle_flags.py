"""Pins of the oracle's cover flags with buffer (Sec. 2.4.2).

Definition: a global cell is covered when its centre lies in a local live box
(closed); d = L-infinity index distance to the nearest uncovered cell; LIVE if
d <= NG+1 (the buffer), effective GHOST if NG+1 < d <= 2NG+1, DEAD beyond.
Checked against a brute-force distance computation and against the counts
that follow by hand for the aligned static layout.
"""
import numpy as np
import pytest

from oracle import pyoracle as po
from paper_2002_00088_gb300 import workloads as wl
from tests.golden_fixtures import key_values
from tests.helpers import oracle_from


def brute_force_states(covered, buffer=4, ng=3):
    n = covered.shape
    unc = np.argwhere(~covered)
    states = np.zeros(n, dtype=np.uint8)
    for idx in np.argwhere(covered):
        d = np.abs(unc - idx).max(1).min() if len(unc) else 10 ** 9
        # cells outside the grid count as uncovered
        d = min(d, *(idx + 1), *(np.array(n) - idx))
        states[tuple(idx)] = 0 if d <= buffer else (1 if d <= buffer + ng else 2)
    return states


def test_static_layout_counts():
    """Global 48^3 on [-1,1], local [-1/3,1/3]: global centres -1 + (i+1/2)/24 are
    covered for i = 16..31 (16 per axis); shrinking by the buffer (4) leaves 8^3,
    by buffer + NG leaves 2^3, so 504 effective ghost cells and 8 deactivated."""
    w = wl.static_gauss()
    o = oracle_from(w)
    o.compute_flags()
    f = o.get_flags()
    st = f & 3
    want = key_values("flags_static_layout.txt")
    assert (st == po.GHOST).sum() == want["ghost"]
    assert (st == po.DEAD).sum() == want["dead"]
    cov = (f >> 2) == 1
    assert cov.sum() == want["covered"]
    assert np.array_equal(np.argwhere(cov).min(0), [16, 16, 16])
    assert o.live_points() == 48 ** 3 - 512 + 32 ** 3


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_flags_match_brute_force(seed):
    rng = np.random.default_rng(seed)
    o = po.Oracle(interp_points=6)
    o.add_patch(po.GLOBAL, (20, 22, 24), (-1, -1.1, -1.2), (1, 1.1, 1.2), po.BC_ANALYTIC)
    boxes = []
    for q in range(2):
        half = rng.uniform(0.25, 0.45, 3)
        centre = np.array([-0.45 + 0.9 * q, 0.0, 0.0]) + rng.uniform(-0.05, 0.05, 3)
        o.add_patch(po.LOCAL, (10, 10, 10), -half, half, po.BC_INTERPATCH, po.STATIC, tuple(centre))
        boxes.append((centre - half, centre + half))
    o.compute_flags()
    f = o.get_flags()
    n = (20, 22, 24)
    lo = np.array([-1, -1.1, -1.2])
    h = (-2 * lo) / np.array(n)
    ax = [lo[a] + (np.arange(n[a]) + 0.5) * h[a] for a in range(3)]
    z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    covered = np.zeros((n[2], n[1], n[0]), bool)
    owner = np.zeros_like(covered, dtype=np.uint8)
    for q, (blo, bhi) in enumerate(boxes):
        inside = (x >= blo[0]) & (x <= bhi[0]) & (y >= blo[1]) & (y <= bhi[1]) & (z >= blo[2]) & (z <= bhi[2])
        covered |= inside
        owner[inside] = q + 1
    np.testing.assert_array_equal(f & 3, brute_force_states(covered))
    np.testing.assert_array_equal(f >> 2, owner)


def test_overlapping_patches_are_rejected():
    o = po.Oracle(interp_points=6)
    o.add_patch(po.GLOBAL, (16, 16, 16), (-1, -1, -1), (1, 1, 1), po.BC_ANALYTIC)
    o.add_patch(po.LOCAL, (8, 8, 8), (-0.3,) * 3, (0.3,) * 3, po.BC_INTERPATCH, po.STATIC, (0.1, 0, 0))
    o.add_patch(po.LOCAL, (8, 8, 8), (-0.3,) * 3, (0.3,) * 3, po.BC_INTERPATCH, po.STATIC, (-0.1, 0, 0))
    with pytest.raises(po.OracleError):
        o.compute_flags()


def test_revival_after_motion():
    """A patch moving by one global cell uncovers one layer: cells that were
    effective ghosts become live again (REVIVED) and take u_n from the local
    patch; deactivated cells are poisoned."""
    o = po.Oracle(interp_points=6)
    o.add_patch(po.GLOBAL, (32, 32, 32), (-1, -1, -1), (1, 1, 1), po.BC_ANALYTIC)
    o.add_patch(po.LOCAL, (32, 32, 32), (-0.5,) * 3, (0.5,) * 3, po.BC_INTERPATCH, po.LINEAR,
                (0.0, 0.0, 0.0, 1.0 / 16, 0.0, 0.0))
    o.set_analytic(po.PLANE_SUM, [3.0, 1.0, np.pi, 0.0, 0.0, 0.0], 1)
    o.fill_analytic(0.0)
    o.compute_flags()
    f0 = o.get_flags() & 3
    o.time = 1.0  # moved by one global cell (h = 1/16) along +x
    o.fill_analytic(1.0)
    o.time = 1.0
    o.compute_flags()
    f1 = o.get_flags() & 3
    revived = f1 == po.REVIVED
    assert revived.sum() > 0
    assert np.all((f0[revived] == po.GHOST) | (f0[revived] == po.DEAD))
    ps, _ = o.get_fields(0)
    assert np.isnan(ps[f1 == po.DEAD]).all()
    assert np.isfinite(ps[revived]).all()
    # revived values interpolate the local patch (plane wave, 6-point Lagrange)
    lo, h = -1.0, 2.0 / 32
    x = lo + (np.arange(32) + 0.5) * h
    want = np.broadcast_to(3.0 + np.sin(np.pi * (x - 1.0)), ps.shape)
    assert np.abs(ps[revived] - want[revived]).max() < 1e-5
