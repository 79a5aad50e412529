"""Write tests/golden/oracle_3x4x5_seed11_7steps.txt from the FP64 oracle only.

Inputs: 3x4x5 cells, random fields from cavity_inputs (seed 11), per-position
coefficients dt*U[0.5, 1) from numpy's default_rng(12) (ce for Ex, Ey, Ez then
ch for Hx, Hy, Hz), dt = 0.5/sqrt(3), dx = 1; 7 leapfrog steps.
Output: one line per quantity: name, then values (repr, canonical order).
Run:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import cavity_inputs as ci  # noqa: E402
import oracle  # noqa: E402

NX, NY, NZ, SEED, STEPS = 3, 4, 5, 11, 7
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_3x4x5_seed11_7steps.txt")


def inputs():
    dt = ci.COURANT_HALF_DT
    rng = np.random.default_rng(12)
    sh = (NZ + 1, NY + 1, NX + 1)
    ce = [dt * rng.uniform(0.5, 1.0, sh) for _ in range(3)]
    ch = [dt * rng.uniform(0.5, 1.0, sh) for _ in range(3)]
    f = oracle.as_f64(ci.random_fields(SEED, NX, NY, NZ))
    return f, ce, ch, dt


def main():
    f, ce, ch, dt = inputs()
    oracle.step(f, ce, ch, STEPS)
    w = oracle.energy(f, ce, ch, dt)
    de, dh = oracle.divergence(f, ce, ch)
    with open(OUT, "w") as fh:
        fh.write("# FP64 oracle, 3x4x5 cells, fields seed 11, coefficients default_rng(12), 7 steps\n")
        for name, a in zip(ci.COMPONENTS, f):
            fh.write(name + " " + " ".join(repr(float(v)) for v in a.ravel()) + "\n")
        fh.write("energy " + repr(w) + "\n")
        fh.write("divE_l2 " + repr(float(np.sqrt(np.sum(de * de)))) + "\n")
        fh.write("divH_l2 " + repr(float(np.sqrt(np.sum(dh * dh)))) + "\n")


if __name__ == "__main__":
    main()
