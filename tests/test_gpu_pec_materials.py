"""PEC as materials in the two-step kernel.

A context whose coefficients compress to at most 31 material tuples also holds, for the two-step
kernels, a second id array: 1 + id + ntab x (one bit per low face the cell lies on: i = 0, j = 0,
k = 0), and 0 outside the cavity.  Its table zeroes the E coefficients of the components tangential to those
faces, since tangential E vanishes on the PEC walls (Sec. 2).  Entry 0 zeroes ce, so E stays at the 0
a box reads outside the cavity.  The kernel's steady planes then apply no per-cell masks.

Every value keeps the operation sequence of the one-step kernel: a masked coefficient was already a
zero multiplied into the same fused multiply-add.  FP32 results must therefore stay bit-identical to
the one-step kernel with the coded ids (31 materials) and without them (32 materials), with uniform
and per-material ch, and match the oracle.
"""
import numpy as np
import pytest

import cavity_inputs as ci
from tests.gpu_util import DT, ENERGY_DRIFT_F32, REL_L2_F32, compare_fields, run_gpu

pytestmark = pytest.mark.gpu

T2 = {"kernel": 3}
T1 = {"kernel": 2, "tile_y": 8}


def tuples(n, dims, seed, h_per_material):
    """n material tuples drawn per position: ce_m on all three components; ch uniform or ch_m."""
    rng = np.random.default_rng(seed)
    sh = (dims[2] + 1, dims[1] + 1, dims[0] + 1)
    m = rng.integers(0, n, sh)
    ce_lv = DT * (0.4 + 0.6 * np.arange(n) / n)
    ce = [ce_lv[m].astype(np.float32) for _ in range(3)]
    if not h_per_material:
        return ce, None
    ch_lv = DT * (0.5 + 0.5 * np.arange(n) / n)
    return ce, [ch_lv[m].astype(np.float32) for _ in range(3)]


def assert_bitwise(a, b):
    for n, (x, y) in enumerate(zip(a, b)):
        bad = np.argwhere(x != y)
        assert bad.size == 0, (ci.COMPONENTS[n], len(bad), bad[:6].tolist(), float(np.max(np.abs(x - y))))


@pytest.mark.parametrize("dims", [(130, 67, 45), (61, 13, 9), (7, 9, 11), (121, 40, 3)])
@pytest.mark.parametrize("n", [6, 31, 32])
@pytest.mark.parametrize("h_per_material", [False, True])
def test_coded_ids_bitwise_equal_one_step(dims, n, h_per_material):
    ce, ch = tuples(n, dims, 11 + n, h_per_material)
    f = ci.random_fields(23, *dims)
    for steps in (1, 2, 7):
        a, *_ = run_gpu(f, dims, ce=ce, ch=ch, steps=steps, tuning=T1)
        b, *_ = run_gpu(f, dims, ce=ce, ch=ch, steps=steps, tuning=T2)
        assert_bitwise(a, b)


@pytest.mark.parametrize("h_per_material", [False, True])
def test_coded_ids_vs_oracle(h_per_material):
    import oracle
    dims = (37, 21, 13)
    ce, ch = tuples(31, dims, 3, h_per_material)
    f = ci.random_fields(5, *dims)
    got, w0, w1, _, _ = run_gpu(f, dims, ce=ce, ch=ch, steps=24, tuning=T2)
    ref = oracle.as_f64(f)
    oracle.step(ref, [np.asarray(c, np.float64) for c in ce],
                DT if ch is None else [np.asarray(c, np.float64) for c in ch], 24, omp=True)
    compare_fields(got, ref, dims, REL_L2_F32)
    assert abs(w1 - w0) <= ENERGY_DRIFT_F32 * abs(w0)


def test_coded_ids_held_up_to_31_materials():
    """The coded ids cost one byte per cell and the 8 KiB table, and exist only up to 31 materials."""
    from paper_2504_09118_gb300 import Cavity
    nx, ny, nz = dims = (45, 30, 20)
    held = {}
    for n in (31, 32):
        ce, ch = tuples(n, dims, 2, False)
        cav = Cavity(nx, ny, nz, DT, 1.0, ce, ch, 0)
        try:
            held[n] = cav.device_bytes
        finally:
            cav.close()
    extra = held[31] - held[32]
    assert nx * ny * nz + 8192 <= extra <= (nx + 64) * ny * nz + 8192, held
