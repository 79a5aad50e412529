"""Temporal blocking: two leapfrog steps per launch (kernel TEMPORAL) against the oracle and the one-step kernel.

With FP32 storage the intermediate level (H^{n+1/2}, E^{n+1}) is FP32 in both
kernels and every value follows the same operation sequence (same fused
multiply-adds, same operand order), so two-step launches must reproduce the
one-step kernel bit for bit, whatever the tiling, the step count parity and the
graph chunking.  With 16-bit storage the two-step kernel skips one rounding per
pair of steps, so it is held to the oracle bound of the 16-bit tests instead,
and to bitwise independence of its own tiling.
"""
import math

import numpy as np
import pytest

import cavity_inputs as ci
from tests.gpu_util import DT, ENERGY_DRIFT_F32, REL_L2_F32, compare_fields, run_gpu

pytestmark = pytest.mark.gpu

T2 = {"kernel": 3}
T1 = {"kernel": 2, "tile_y": 8}


def oracle_run(fields, ce, ch, steps):
    import oracle
    f = oracle.as_f64(fields)
    ce64 = DT if ce is None else [np.asarray(c, np.float64) for c in ce]
    ch64 = DT if ch is None else (ch if np.isscalar(ch) else [np.asarray(c, np.float64) for c in ch])
    oracle.step(f, ce64, ch64, steps, omp=True)
    return f


def materials(kind, dims, seed):
    if kind == "vacuum":
        return None, None
    if kind == "spheres":
        sph = ci.sphere_list(seed, 4, dims, 2.0, max(2.5, min(dims) / 3))
        return ci.sphere_coefficients(sph, *dims, DT)
    # a few (ce, ch) tuples with per-position ch: material ids with a non-uniform H table
    rng = np.random.default_rng(seed)
    sh = (dims[2] + 1, dims[1] + 1, dims[0] + 1)
    lv = DT * np.array([0.5, 0.75, 1.0])
    ce = [lv[rng.integers(0, 3, sh)].astype(np.float32) for _ in range(3)]
    ch = [lv[rng.integers(0, 2, sh)].astype(np.float32) for _ in range(3)]
    return ce, ch


def assert_bitwise(a, b):
    for n, (x, y) in enumerate(zip(a, b)):
        bad = np.argwhere(x != y)
        assert bad.size == 0, (ci.COMPONENTS[n], len(bad), bad[:6].tolist(), float(np.max(np.abs(x - y))))


# x extents around the two-step kernel's tile edges (60 cells per tile)
@pytest.mark.parametrize("dims", [(4, 4, 4), (7, 9, 11), (130, 67, 45), (1, 3, 2), (64, 8, 3), (61, 13, 1),
                                  (121, 40, 33), (60, 12, 2), (120, 10, 6), (181, 17, 9), (2, 70, 5)])
@pytest.mark.parametrize("mat", ["vacuum", "spheres", "few"])
def test_two_step_equals_one_step_bitwise_f32(dims, mat):
    ce, ch = materials(mat, dims, 5)
    f = ci.random_fields(21, *dims)
    for steps in (1, 2, 7):
        a, *_ = run_gpu(f, dims, ce=ce, ch=ch, steps=steps, tuning=T1)
        b, *_ = run_gpu(f, dims, ce=ce, ch=ch, steps=steps, tuning=T2)
        assert_bitwise(a, b)


@pytest.mark.parametrize("tile_y", [8, 12, 16])
@pytest.mark.parametrize("stages", [3, 5, 8])
@pytest.mark.parametrize("zchunk", [0, 1, 2, 7])
def test_two_step_tuning_grid(tile_y, stages, zchunk):
    dims = (131, 37, 29)
    ce, ch = materials("spheres", dims, 7)
    f = ci.random_fields(8, *dims)
    a, *_ = run_gpu(f, dims, ce=ce, ch=ch, steps=10, tuning=T1)
    b, *_ = run_gpu(f, dims, ce=ce, ch=ch, steps=10,
                    tuning={"kernel": 3, "tile_y": tile_y, "stages": stages, "zchunk": zchunk})
    assert_bitwise(a, b)


@pytest.mark.parametrize("mat", ["spheres", "few"])
def test_two_step_vs_oracle(mat):
    dims = (70, 53, 41)
    ce, ch = materials(mat, dims, 1)
    f = ci.random_fields(2, *dims)
    ref = oracle_run(f, ce, ch, 61)
    got, w0, w1, _, _ = run_gpu(f, dims, ce=ce, ch=ch, steps=61, tuning=T2)
    compare_fields(got, ref, dims, REL_L2_F32)
    if mat == "spheres":
        assert abs(w1 - w0) / w0 <= ENERGY_DRIFT_F32


@pytest.mark.parametrize("steps", [16, 37, 48])
def test_two_step_graph_chunks_match_direct(steps):
    import torch
    dims = (96, 40, 33)
    f = ci.random_fields(9, *dims)
    s = torch.cuda.Stream()
    a, *_ = run_gpu(f, dims, steps=steps, tuning=T1, stream=s)
    b, *_ = run_gpu(f, dims, steps=steps, tuning={"kernel": 3, "use_graph": 1}, stream=s)
    assert_bitwise(a, b)


U = {1: 2.0 ** -11, 2: 2.0 ** -8}


def rel_err(got, ref, dims):
    nx, ny, nz = dims
    num = den = 0.0
    for c, name in enumerate(ci.COMPONENTS):
        m = ci.extent_mask(name, nx, ny, nz)
        num += float(np.sum((np.asarray(got[c], np.float64)[m] - np.asarray(ref[c], np.float64)[m]) ** 2))
        den += float(np.sum(np.asarray(ref[c], np.float64)[m] ** 2))
    return math.sqrt(num / den)


@pytest.mark.parametrize("storage", [1, 2])
def test_two_step_16bit_vs_oracle(storage):
    # one 16-bit rounding per stored value and launch: the random-walk bound of the one-step
    # kernel (3 u/sqrt(3) sqrt(N + 1)) covers it with room to spare
    dims = (70, 45, 37)
    steps = 100
    sph = ci.sphere_list(3, 5, dims, 4.0, 12.0)
    ce, ch = ci.sphere_coefficients(sph, *dims, DT)
    f = ci.random_fields(4, *dims)
    ref = oracle_run(f, ce, ch, steps)
    got, w0, w1, _, _ = run_gpu(f, dims, ce=ce, ch=ch, steps=steps, storage=storage, tuning=T2)
    bound = 3.0 * U[storage] / math.sqrt(3.0) * math.sqrt(steps + 1)
    err = rel_err(got, ref, dims)
    assert 0.05 * U[storage] <= err <= bound, (err, bound)
    assert abs(w1 - w0) / w0 <= bound


@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("dims", [(67, 29, 18), (113, 21, 9), (168, 11, 7)])   # around the 60-cell x tiles
def test_two_step_16bit_independent_of_tiling(storage, dims):
    f = ci.random_fields(6, *dims)
    a, *_ = run_gpu(f, dims, steps=12, storage=storage, tuning={"kernel": 3, "tile_y": 8})
    b, *_ = run_gpu(f, dims, steps=12, storage=storage, tuning={"kernel": 3, "tile_y": 12, "zchunk": 5, "stages": 3})
    assert_bitwise(a, b)


@pytest.mark.parametrize("storage", [0, 1])
def test_two_step_pec_and_far_faces(storage):
    from paper_2504_09118_gb300 import Cavity
    dims = (40, 33, 21)
    nx, ny, nz = dims
    f = ci.random_fields(5, *dims)
    with Cavity(nx, ny, nz, DT, 1.0, None, None, storage) as cav:
        cav.tune(**T2)
        cav.set_fields(f)
        g0 = cav.get_fields()
        cav.step(26)
        assert cav.steps_done == 26
        g = cav.get_fields()
    for c, name in enumerate(("Ex", "Ey", "Ez")):
        assert np.all(g[c][ci.tangential_e_mask(name, nx, ny, nz)] == 0.0)
    assert np.array_equal(g[3][:nz, :ny, [0, nx]], g0[3][:nz, :ny, [0, nx]])
    assert np.array_equal(g[4][:nz, [0, ny], :nx], g0[4][:nz, [0, ny], :nx])
    assert np.array_equal(g[5][[0, nz], :ny, :nx], g0[5][[0, nz], :ny, :nx])


def test_two_step_tuning_rejects_bad_tile():
    from paper_2504_09118_gb300 import Cavity, FdtdError
    with Cavity(8, 8, 8, DT, 1.0, None, None, 0) as cav:
        for bad in (4, 10, 20):
            with pytest.raises(FdtdError):
                cav.tune(kernel=3, tile_y=bad)
        cav.tune(kernel=3, tile_y=12)
