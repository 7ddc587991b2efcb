"""The oracle uses the constants the paper prints (tests/golden/)."""
import numpy as np

from oracle import pyoracle as po
from tests.golden_fixtures import key_values


def test_ko_strength_and_order_in_rhs():
    """Sec. 2.3: n = 5 (sixth difference), epsilon = 0.005.  A grid-scale
    checkerboard along x, u = (-1)^i, has sixth difference
    -1 - 6 - 15 - 20 - 15 - 6 - 1 = -64 times (-1)^i, so the KO term of the RHS
    is (eps/64)(-64)(-1)^i / h = -eps (-1)^i / h: it damps the grid mode."""
    g = key_values("ko_dissipation.txt")
    assert g["n"] == 5
    eps = g["epsilon"]
    n = (8, 6, 6)
    o = po.Oracle(interp_points=6, ko_eps=eps)
    o.add_patch(po.GLOBAL, n, (0, 0, 0), (1, 1, 1), po.BC_PERIODIC)
    i = np.arange(-3, n[0] + 3)
    cb = np.broadcast_to((-1.0) ** i, (n[2] + 6, n[1] + 6, n[0] + 6)).copy()
    o.set_padded(0, cb, np.zeros_like(cb))
    kps, _ = o.eval_rhs(0, 0.0)
    h = 1.0 / n[0]
    np.testing.assert_allclose(kps, -eps * cb[3:-3, 3:-3, 3:-3] / h, rtol=1e-13)
