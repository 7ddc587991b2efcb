"""Shared test helpers: build an oracle or a GPU simulation from a workload."""
import os

import numpy as np

from oracle import pyoracle as po


def oracle_from(w, threads=None, buffer=4):
    o = po.Oracle(w.interp_points, w.ko_eps, buffer, threads or min(8, os.cpu_count() or 1))
    for p in w.patches:
        o.add_patch(p.kind, p.n, p.lo, p.hi, p.outer_bc, p.motion, p.motion_params, p.topology)
    o.set_analytic(w.analytic_kind, w.analytic_params, w.analytic_count)
    return o


def gpu_from(mpw, w, buffer=0, arith=0, precision=64):
    s = mpw.Multipatch(interp_points=w.interp_points, ko_eps=w.ko_eps, buffer=buffer, arith=arith,
                       precision=precision)
    for p in w.patches:
        s.create_patch(p.kind, p.n, p.lo, p.hi, p.outer_bc, p.motion, p.motion_params, p.topology)
    s.set_analytic(w.analytic_kind, w.analytic_params, w.analytic_count)
    return s


def initial_fields(o, npatch):
    """Closed-form initial data at t = 0, evaluated by the oracle."""
    o.fill_analytic(0.0)
    return [o.get_padded(q) for q in range(npatch)]


def interior(a):
    return a[3:-3, 3:-3, 3:-3]


def rel_err(a, b):
    """max |a - b| / max |b| over entries where b is finite."""
    m = np.isfinite(b)
    scale = np.max(np.abs(b[m]))
    return float(np.max(np.abs(a[m] - b[m])) / scale) if scale > 0 else float(np.max(np.abs(a[m] - b[m])))
