"""Pins of the oracle's 1-D Lagrange weights (Sec. 2.4, Eq. Pijk).

The window is fixed by the paper: i_c is the node closest to the point without
exceeding it, the window starts at i_c - 2 (P = 6: i_c-2..i_c+3).  Checked
against the defining properties (node values, partition of unity, exact
reproduction of every polynomial of degree <= P-1) and against numpy's
polynomial fit through the same nodes.
"""
import math

import numpy as np
import pytest

from oracle import pyoracle as po


@pytest.mark.parametrize("P", [5, 6])
@pytest.mark.parametrize("s", [3.0, 3.25, 3.999999, -1.5, 0.5, 17.75])
def test_window_start_and_partition_of_unity(P, s):
    start, w = po.lagrange(P, s)
    assert start == math.floor(s) - 2
    assert abs(w.sum() - 1.0) < 1e-14


@pytest.mark.parametrize("P", [5, 6])
def test_node_property(P):
    # at a node the weights are a unit vector on that node (it is i_c itself)
    start, w = po.lagrange(P, 7.0)
    assert start == 5
    expect = np.zeros(P)
    expect[2] = 1.0
    np.testing.assert_array_equal(w, expect)


@pytest.mark.parametrize("P", [5, 6])
def test_reproduces_polynomials_up_to_degree_P_minus_1(P):
    rng = np.random.default_rng(1)
    for trial in range(20):
        s = rng.uniform(-5, 5)
        coef = rng.normal(size=P)  # degree P-1
        start, w = po.lagrange(P, s)
        nodes = start + np.arange(P)
        got = np.dot(w, np.polyval(coef, nodes))
        want = np.polyval(coef, s)
        assert abs(got - want) <= 1e-13 * max(1.0, np.abs(np.polyval(np.abs(coef), abs(s) + P)))
    # one degree more is not reproduced: the window really holds P points
    s = 0.37
    coef = np.zeros(P + 1)
    coef[0] = 1.0
    start, w = po.lagrange(P, s)
    nodes = start + np.arange(P)
    assert abs(np.dot(w, np.polyval(coef, nodes)) - np.polyval(coef, s)) > 1e-3


@pytest.mark.parametrize("P", [5, 6])
def test_matches_numpy_polyfit(P):
    rng = np.random.default_rng(2)
    for trial in range(10):
        s = rng.uniform(-3, 3)
        start, w = po.lagrange(P, s)
        nodes = start + np.arange(P, dtype=float)
        vals = rng.normal(size=P)
        fit = np.polynomial.polynomial.Polynomial.fit(nodes, vals, P - 1)
        assert abs(np.dot(w, vals) - fit(s)) < 1e-11
