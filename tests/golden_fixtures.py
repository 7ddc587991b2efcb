"""Readers of the cited fixtures under tests/golden/."""
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def rk4_tableau():
    c, a, b = [], [], None
    for tok in _lines("rk4_tableau.txt"):
        if tok[0] == "c":
            c.append(float(Fraction(tok[1])))
            a.append([float(Fraction(v)) for v in tok[3:]])
        elif tok[0] == "b":
            b = [float(Fraction(v)) for v in tok[1:]]
    return np.array(c), np.array(a), np.array(b)


def key_values(name):
    return {tok[0]: float(tok[1]) for tok in _lines(name)}
