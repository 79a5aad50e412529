"""The oracle reproduces its committed golden output bit for bit (regression pin)."""
import os

import numpy as np

from tests.golden import make_golden as mg


def load():
    vals = {}
    with open(mg.OUT) as fh:
        for line in fh:
            if line.startswith("#"):
                continue
            name, *rest = line.split()
            vals[name] = np.array([float(v) for v in rest])
    return vals


def test_golden_regression(oracle_mod):
    g = load()
    f, ce, ch, dt = mg.inputs()
    oracle_mod.step(f, ce, ch, mg.STEPS)
    for name, a in zip(("Ex", "Ey", "Ez", "Hx", "Hy", "Hz"), f):
        assert np.array_equal(a.ravel(), g[name]), name
    assert oracle_mod.energy(f, ce, ch, dt) == g["energy"][0]
