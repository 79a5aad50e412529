"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and compare with the oracle."""
from __future__ import annotations

import numpy as np

import cavity_inputs as ci

DT = ci.COURANT_HALF_DT
# Contract bounds: rel-L2 per field and relative energy drift for FP32 storage.
REL_L2_F32 = 1e-4
ENERGY_DRIFT_F32 = 1e-5


def rel_l2(got, ref, mask=None, state_norm=None):
    """Relative L2 error; when the reference is ~0 the error is taken relative to the whole state."""
    if mask is not None:
        got, ref = got[mask], ref[mask]
    d = float(np.linalg.norm(np.asarray(got, np.float64) - np.asarray(ref, np.float64)))
    r = float(np.linalg.norm(np.asarray(ref, np.float64)))
    if r <= 1e-30 * max(1, ref.size):
        return d / max(state_norm or 1.0, 1e-300)
    return d / r


def run_gpu(fields, dims, ce=None, ch=None, steps=1, storage=0, dt=DT, tuning=None, stream=None):
    """Create a cavity, load the fields, step, and return (fields, energy0, energy1, div0, div1)."""
    from paper_2504_09118_gb300 import Cavity
    nx, ny, nz = dims
    cav = Cavity(nx, ny, nz, dt, 1.0, ce, ch, storage, stream)
    try:
        if tuning:
            cav.tune(**tuning)
        cav.set_fields(fields)
        w0 = cav.energy()
        d0 = cav.divergence()
        cav.step(steps)
        w1 = cav.energy()
        d1 = cav.divergence()
        out = cav.get_fields()
    finally:
        cav.close()
    return out, w0, w1, d0, d1


def compare_fields(got, ref, dims, bound):
    nx, ny, nz = dims
    norm = float(np.sqrt(sum(np.sum(np.asarray(r, np.float64) ** 2) for r in ref)))
    errs = {}
    for c, name in enumerate(ci.COMPONENTS):
        m = ci.extent_mask(name, nx, ny, nz)
        errs[name] = rel_l2(got[c], ref[c], m, norm)
    worst = max(errs.values())
    assert worst <= bound, errs
    return errs
