"""The two-step kernel with two rows per consumer warp (kernel TEMPORAL2).

It computes every value with the same operation sequence as the one-row two-step kernel (the level-2
E update reuses the masked coefficients of the level-1 update of the same cell instead of looking them
up again: the same numbers), so its results must equal that kernel bit for bit with every storage
precision, and with FP32 storage also the one-step kernel.  Sizes straddle the 60-cell x tiles (whose
TMA box origin shifts by 0-6 elements with 16-bit storage) and both tile heights; the idle upper row of the last warp, the rows shared
through registers and those exchanged between warps are all on the path of these cases.
"""
import numpy as np
import pytest

import cavity_inputs as ci
from tests.gpu_util import DT, ENERGY_DRIFT_F32, REL_L2_F32, compare_fields, run_gpu
from tests.test_gpu_temporal import assert_bitwise, materials, oracle_run

pytestmark = pytest.mark.gpu

T1 = {"kernel": 2, "tile_y": 8}


@pytest.mark.parametrize("dims", [(4, 4, 4), (7, 9, 11), (130, 67, 45), (1, 3, 2), (64, 8, 3), (61, 13, 1),
                                  (121, 40, 33), (60, 12, 2), (120, 10, 6), (2, 70, 5), (59, 19, 4)])
@pytest.mark.parametrize("mat", ["vacuum", "spheres", "few"])
@pytest.mark.parametrize("tile_y", [12, 16])
def test_rows2_equals_one_step_bitwise_f32(dims, mat, tile_y):
    ce, ch = materials(mat, dims, 5)
    f = ci.random_fields(21, *dims)
    for steps in (1, 2, 7):
        a, *_ = run_gpu(f, dims, ce=ce, ch=ch, steps=steps, tuning=T1)
        b, *_ = run_gpu(f, dims, ce=ce, ch=ch, steps=steps, tuning={"kernel": 4, "tile_y": tile_y})
        assert_bitwise(a, b)


@pytest.mark.parametrize("tile_y", [12, 16])
@pytest.mark.parametrize("stages", [3, 4, 5])
@pytest.mark.parametrize("zchunk", [0, 1, 2, 7])
def test_rows2_tuning_grid(tile_y, stages, zchunk):
    dims = (131, 37, 29)
    ce, ch = materials("spheres", dims, 7)
    f = ci.random_fields(8, *dims)
    a, *_ = run_gpu(f, dims, ce=ce, ch=ch, steps=10, tuning=T1)
    b, *_ = run_gpu(f, dims, ce=ce, ch=ch, steps=10,
                    tuning={"kernel": 4, "tile_y": tile_y, "stages": stages, "zchunk": zchunk})
    assert_bitwise(a, b)


@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("dims", [(67, 29, 18), (113, 21, 9), (168, 11, 7), (56, 17, 5)])
@pytest.mark.parametrize("mat", ["vacuum", "few"])
def test_rows2_equals_one_row_two_step_16bit(storage, dims, mat):
    ce, ch = materials(mat, dims, 3)
    f = ci.random_fields(6, *dims)
    for steps in (2, 13):
        a, *_ = run_gpu(f, dims, ce=ce, ch=ch, steps=steps, storage=storage, tuning={"kernel": 3, "tile_y": 16})
        b, *_ = run_gpu(f, dims, ce=ce, ch=ch, steps=steps, storage=storage,
                        tuning={"kernel": 4, "tile_y": 12, "zchunk": 5, "stages": 3})
        assert_bitwise(a, b)


@pytest.mark.parametrize("mat", ["spheres", "few"])
def test_rows2_vs_oracle(mat):
    dims = (70, 53, 41)
    ce, ch = materials(mat, dims, 1)
    f = ci.random_fields(2, *dims)
    ref = oracle_run(f, ce, ch, 61)
    got, w0, w1, _, _ = run_gpu(f, dims, ce=ce, ch=ch, steps=61, tuning={"kernel": 4})
    compare_fields(got, ref, dims, REL_L2_F32)
    if mat == "spheres":
        assert abs(w1 - w0) / w0 <= ENERGY_DRIFT_F32


def test_rows2_pec_and_far_faces():
    from paper_2504_09118_gb300 import Cavity
    dims = (40, 33, 21)
    nx, ny, nz = dims
    f = ci.random_fields(5, *dims)
    with Cavity(nx, ny, nz, DT, 1.0, None, None, 0) as cav:
        cav.tune(kernel=4)
        cav.set_fields(f)
        g0 = cav.get_fields()
        cav.step(26)
        g = cav.get_fields()
    for c, name in enumerate(("Ex", "Ey", "Ez")):
        assert np.all(g[c][ci.tangential_e_mask(name, nx, ny, nz)] == 0.0)
    assert np.array_equal(g[3][:nz, :ny, [0, nx]], g0[3][:nz, :ny, [0, nx]])
    assert np.array_equal(g[4][:nz, [0, ny], :nx], g0[4][:nz, [0, ny], :nx])
    assert np.array_equal(g[5][[0, nz], :ny, :nx], g0[5][[0, nz], :ny, :nx])


@pytest.mark.parametrize("storage", [0, 2])
def test_rows2_batch_members_equal_solo(storage):
    """Batched launches of the two-row kernel with per-member step counts (odd ones end on a level-1
    store inside a two-step launch) equal each member stepped alone by the one-row two-step kernel."""
    import torch
    from paper_2504_09118_gb300 import Cavity, binding
    rng = np.random.default_rng(11)
    stream = torch.cuda.Stream()
    members, steps = [], []
    for q in range(7):
        dims = tuple(int(v) for v in rng.integers(5, 70, 3))
        f = ci.random_fields(100 + q, *dims)
        cav = Cavity(*dims, DT, 1.0, None, None, storage, stream)
        cav.set_fields(f)
        members.append((cav, dims, f))
        steps.append(int(rng.integers(3, 40)))
    b = binding.fdtd_batch_create(storage, stream)
    try:
        binding.fdtd_batch_set_tuning(b, kernel=4, tile_y=16, use_graph=1)
        for (cav, _, _), n in zip(members, steps):
            binding.fdtd_batch_add(b, cav.handle)
            binding.fdtd_batch_set_steps(b, cav.handle, n)
        binding.fdtd_batch_step(b, max(steps) + 5)
        binding.fdtd_batch_sync(b)
        got = []
        for cav, _, _ in members:
            binding.fdtd_batch_remove(b, cav.handle)
            got.append(cav.get_fields())
    finally:
        binding.fdtd_batch_destroy(b)
        for cav, _, _ in members:
            cav.close()
    for (cav, dims, f), n, g in zip(members, steps, got):
        ref, *_ = run_gpu(f, dims, steps=n, storage=storage, tuning={"kernel": 3, "tile_y": 16})
        assert_bitwise(g, ref)


def test_rows2_tuning_rejects_bad_tile():
    from paper_2504_09118_gb300 import Cavity, FdtdError
    with Cavity(8, 8, 8, DT, 1.0, None, None, 0) as cav:
        for bad in (4, 8, 10, 20):
            with pytest.raises(FdtdError):
                cav.tune(kernel=4, tile_y=bad)
        cav.tune(kernel=4, tile_y=12)
    with Cavity(8, 8, 8, DT, 1.0, None, None, 0, order=4) as cav:
        with pytest.raises(FdtdError):
            cav.tune(kernel=4)
