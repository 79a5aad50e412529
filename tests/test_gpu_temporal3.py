"""Temporal blocking with three leapfrog steps per launch (kernel TEMPORAL3) against the oracle and the
one-step kernel.

As in the two-step kernel, every intermediate level is FP32 and every value follows the same operation
sequence as in the one-step kernel, so with FP32 storage the three-step launches (and the one-step launches
that end a count not divisible by three) must reproduce the one-step kernel bit for bit, whatever the tiling,
ring depth, z-chunking and graph chunking.  With 16-bit storage the kernel rounds once per three steps: it is
held to the oracle's random-walk bound and to bitwise independence of its own tiling.
"""
import math

import numpy as np
import pytest

import cavity_inputs as ci
from tests.gpu_util import DT, ENERGY_DRIFT_F32, REL_L2_F32, compare_fields, run_gpu
from tests.test_gpu_temporal import U, assert_bitwise, materials, oracle_run, rel_err

pytestmark = pytest.mark.gpu

T3 = {"kernel": 5}
T1 = {"kernel": 2, "tile_y": 8}


# x extents around the three-step kernel's 58-cell tiles, y around its 8/10/12-row tiles, z down to one plane
@pytest.mark.parametrize("dims", [(4, 4, 4), (7, 9, 11), (130, 67, 45), (1, 3, 2), (58, 10, 3), (59, 13, 1),
                                  (117, 25, 8), (175, 21, 9)])
@pytest.mark.parametrize("mat", ["vacuum", "spheres", "few"])
def test_three_step_equals_one_step_bitwise(dims, mat):
    if mat != "vacuum" and min(dims) < 3:
        pytest.skip("materials need a few cells per axis")
    ce, ch = materials(mat, dims, 5)
    f = ci.random_fields(21, *dims)
    for steps in (1, 3, 7, 12):
        a, *_ = run_gpu(f, dims, ce=ce, ch=ch, steps=steps, tuning=T1)
        b, *_ = run_gpu(f, dims, ce=ce, ch=ch, steps=steps, tuning=T3)
        assert_bitwise(a, b)


@pytest.mark.parametrize("tile_y", [8, 10, 12])
@pytest.mark.parametrize("stages", [3, 5, 8])
@pytest.mark.parametrize("zchunk", [0, 1, 2, 7])
def test_three_step_tuning_grid(tile_y, stages, zchunk):
    dims = (131, 37, 29)
    ce, ch = materials("spheres", dims, 7)
    f = ci.random_fields(8, *dims)
    a, *_ = run_gpu(f, dims, ce=ce, ch=ch, steps=10, tuning=T1)
    b, *_ = run_gpu(f, dims, ce=ce, ch=ch, steps=10,
                    tuning={"kernel": 5, "tile_y": tile_y, "stages": stages, "zchunk": zchunk})
    assert_bitwise(a, b)


@pytest.mark.parametrize("mat", ["spheres", "few"])
def test_three_step_vs_oracle(mat):
    dims = (70, 53, 41)
    ce, ch = materials(mat, dims, 1)
    f = ci.random_fields(2, *dims)
    ref = oracle_run(f, ce, ch, 61)
    got, w0, w1, _, _ = run_gpu(f, dims, ce=ce, ch=ch, steps=61, tuning=T3)
    compare_fields(got, ref, dims, REL_L2_F32)
    if mat == "spheres":
        assert abs(w1 - w0) / w0 <= ENERGY_DRIFT_F32


@pytest.mark.parametrize("steps", [18, 37, 54])
def test_three_step_graph_chunks_match_direct(steps):
    import torch
    dims = (96, 40, 33)
    f = ci.random_fields(9, *dims)
    s = torch.cuda.Stream()
    a, *_ = run_gpu(f, dims, steps=steps, tuning=T1, stream=s)
    b, *_ = run_gpu(f, dims, steps=steps, tuning={"kernel": 5, "use_graph": 1}, stream=s)
    assert_bitwise(a, b)


@pytest.mark.parametrize("storage", [1, 2])
def test_three_step_16bit_vs_oracle(storage):
    # one 16-bit rounding per stored value and launch: within the one-step kernel's random-walk bound
    dims = (70, 45, 37)
    steps = 99
    sph = ci.sphere_list(3, 5, dims, 4.0, 12.0)
    ce, ch = ci.sphere_coefficients(sph, *dims, DT)
    f = ci.random_fields(4, *dims)
    ref = oracle_run(f, ce, ch, steps)
    got, w0, w1, _, _ = run_gpu(f, dims, ce=ce, ch=ch, steps=steps, storage=storage, tuning=T3)
    bound = 3.0 * U[storage] / math.sqrt(3.0) * math.sqrt(steps + 1)
    err = rel_err(got, ref, dims)
    assert 0.05 * U[storage] <= err <= bound, (err, bound)
    assert abs(w1 - w0) / w0 <= bound


@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("dims", [(67, 29, 18), (113, 21, 9), (175, 11, 7)])
def test_three_step_16bit_independent_of_tiling(storage, dims):
    f = ci.random_fields(6, *dims)
    a, *_ = run_gpu(f, dims, steps=12, storage=storage, tuning={"kernel": 5, "tile_y": 8})
    b, *_ = run_gpu(f, dims, steps=12, storage=storage, tuning={"kernel": 5, "tile_y": 12, "zchunk": 5, "stages": 3})
    assert_bitwise(a, b)


@pytest.mark.parametrize("storage", [0, 1])
def test_three_step_pec_and_far_faces(storage):
    from paper_2504_09118_gb300 import Cavity
    dims = (40, 33, 21)
    nx, ny, nz = dims
    f = ci.random_fields(5, *dims)
    with Cavity(nx, ny, nz, DT, 1.0, None, None, storage) as cav:
        cav.tune(**T3)
        cav.set_fields(f)
        g0 = cav.get_fields()
        cav.step(27)
        assert cav.steps_done == 27
        g = cav.get_fields()
    for c, name in enumerate(("Ex", "Ey", "Ez")):
        assert np.all(g[c][ci.tangential_e_mask(name, nx, ny, nz)] == 0.0)
    assert np.array_equal(g[3][:nz, :ny, [0, nx]], g0[3][:nz, :ny, [0, nx]])
    assert np.array_equal(g[4][:nz, [0, ny], :nx], g0[4][:nz, [0, ny], :nx])
    assert np.array_equal(g[5][[0, nz], :ny, :nx], g0[5][[0, nz], :ny, :nx])


def test_three_step_rules():
    import torch
    from paper_2504_09118_gb300 import Cavity, FdtdError, binding
    with Cavity(8, 8, 8, DT, 1.0, None, None, 0) as cav:
        for bad in (4, 16, 20):
            with pytest.raises(FdtdError):
                cav.tune(kernel=5, tile_y=bad)
        cav.tune(kernel=5, tile_y=10)
    with Cavity(16, 16, 16, DT, 1.0, None, None, 0, order=4) as cav:
        with pytest.raises(FdtdError):                 # the second-order scheme only
            cav.tune(kernel=5)
    b = binding.fdtd_batch_create(0, torch.cuda.Stream())
    try:
        with pytest.raises(FdtdError):                 # single cavities only
            binding.fdtd_batch_set_tuning(b, kernel=5)
    finally:
        binding.fdtd_batch_destroy(b)
