"""How far one leapfrog step reaches, measured on the FP64 oracle, against the halo every fused kernel
loads.  The update is linear, so the difference between two runs whose inputs differ in one value at one
cell is that value's impulse response; its support after s steps is the set of outputs that can depend on
the cell.  A fused kernel that advances s steps per launch loads a box of (tile + 2 R) rows, R the reach
of s steps, so a stored value never needs an input outside its box:

  one-step kernel (Eq. 2)        s = 1, R = 1   box rows tile_y + 2
  two-step kernel (Eq. 2 twice)  s = 2, R = 2   box rows tile_y + 4
  fourth-order kernel            s = 1, R = 3   box rows tile_y + 6
  three-step kernel              s = 3, R = 3   box rows tile_y + 6 (the same branch as the fourth order)

The reach is also tight (some output does depend on a cell R away), so none of the boxes could be
smaller.  The box heights are read from the host code that encodes the tensor maps."""
import os
import re

import numpy as np
import pytest

import cavity_inputs as ci
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N = 20
C = (10, 10, 10)   # perturbed cell (k, j, i), far from the walls at these step counts


def reach(order, steps):
    """Largest |offset| per axis (z, y, x) of any output that one input cell influences after `steps`."""
    base = oracle.as_f64(ci.random_fields(3, N, N, N))
    oracle.pec_e(base)
    dt = ci.COURANT_HALF_DT
    run = (lambda f: oracle.step4(f, dt, dt, steps)) if order == 4 else (lambda f: oracle.step(f, dt, dt, steps))
    ref = [a.copy() for a in base]
    run(ref)
    out = np.zeros(3, int)
    for comp in range(6):
        f = [a.copy() for a in base]
        f[comp][C] += 1.0
        run(f)
        for a, b in zip(f, ref):
            idx = np.argwhere(a != b)
            if idx.size:
                out = np.maximum(out, np.abs(idx - np.array(C)).max(axis=0))
    return tuple(int(v) for v in out)


@pytest.mark.parametrize("order,steps,expected", [(2, 1, 1), (2, 2, 2), (2, 3, 3), (4, 1, 3), (4, 2, 6)])
def test_reach_of_the_schemes(order, steps, expected):
    assert reach(order, steps) == (expected,) * 3


def test_box_heights_cover_the_reach_exactly():
    src = open(os.path.join(ROOT, "paper_2504_09118_gb300", "csrc", "plan.cu")).read()
    m = re.search(r"encode_maps\(c, kind, s\.tile_y \+ \(kind == 0 \? (\d+) : kind == 1 \? (\d+) : (\d+)\)\)", src)
    assert m, "box-height expression not found in plan.cu"
    one_step, two_step, fourth = (int(g) for g in m.groups())
    assert one_step == 2 * reach(2, 1)[1]
    assert two_step == 2 * reach(2, 2)[1]
    assert fourth == 2 * reach(4, 1)[1]
    # kind 3 (three steps per launch) takes the last branch too
    assert fourth == 2 * reach(2, 3)[1]
