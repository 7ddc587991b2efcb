"""Global 4th-order convergence of the oracle against a closed form (Sec. 3.2).

Reduced-size version of the paper's Test Two: global cube plus a 2:1 local
cube, fixed or translating, evolving the superposition of plane waves of Sec.
3.4.2 (scaled to the box) with analytic outer BCs.  The paper's error measure
(integral over live cells of both patches of |phi - phi_exact| / phi_exact)
must drop by ~16 when every spacing and dt halve; the paper reports slopes
-4.06 (fixed) and -4.03 (translating), tests/golden/convergence_slopes.txt.
"""
import numpy as np
import pytest

from oracle import pyoracle as po
from paper_2002_00088_gb300 import workloads as wl
from tests.golden_fixtures import key_values
from tests.helpers import oracle_from


def integrated_relative_error(w):
    o = oracle_from(w, threads=8)
    o.fill_analytic(0.0)
    o.step(w.dt, w.steps)
    total = 0.0
    for q, p in enumerate(w.patches):
        ps, _ = o.get_fields(q)
        h = [(p.hi[a] - p.lo[a]) / p.n[a] for a in range(3)]
        mp = list(p.motion_params) + [0.0] * (16 - len(p.motion_params))
        X0, _ = po.motion(p.motion, mp, o.time)
        ax = [p.lo[a] + (np.arange(p.n[a]) + 0.5) * h[a] + X0[a] for a in range(3)]
        z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        ex, _ = po.closed_form(w.analytic_kind, w.analytic_params, w.analytic_count, o.time, x, y, z)
        live = np.isfinite(ps)
        total += np.sum(np.abs(ps[live] - ex[live]) / np.abs(ex[live])) * h[0] * h[1] * h[2]
    return total


@pytest.mark.parametrize("label,velocity", [("fixed", (0.0, 0.0, 0.0)), ("translating", (0.4, 0.3, 0.0))])
def test_fourth_order_convergence(label, velocity):
    e1 = integrated_relative_error(wl.translating_plane(scale=1, velocity=velocity))
    e2 = integrated_relative_error(wl.translating_plane(scale=2, velocity=velocity))
    slope = -np.log2(e1 / e2)
    assert 11.0 < e1 / e2 < 22.0
    assert abs(slope - key_values("convergence_slopes.txt")[label]) < 0.3
