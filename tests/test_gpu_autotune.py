"""Autotuning (fdtd_autotune, fdtd_batch_autotune): the state is untouched and the pick is a valid shape.

With FP32 storage every candidate produces bit-identical fields (same operation sequence per value),
so a tuned run must equal an untuned run bit for bit.
"""
import numpy as np
import pytest

import cavity_inputs as ci
from tests.gpu_util import DT
from tests.test_gpu_batch import make_members

pytestmark = pytest.mark.gpu


def test_autotune_keeps_state_and_result():
    from paper_2504_09118_gb300 import Cavity
    dims = (130, 67, 45)
    sph = ci.sphere_list(4, 5, dims, 3.0, 12.0)
    ce, ch = ci.sphere_coefficients(sph, *dims, DT)
    f = ci.random_fields(12, *dims)
    with Cavity(*dims, DT, 1.0, ce, ch) as cav:
        cav.set_fields(f)
        cav.step(3)
        before = cav.get_fields()
        tuning, ms = cav.autotune(16)
        assert tuning["kernel"] in (2, 3, 4, 5) and ms > 0
        assert tuning["tile_y"] in {2: (4, 8, 16), 3: (8, 12, 16), 4: (12, 16), 5: (8, 10, 12)}[tuning["kernel"]]
        assert cav.steps_done == 3
        for x, y in zip(cav.get_fields(), before):
            assert np.array_equal(x, y)
        cav.step(17)
        tuned = cav.get_fields()
        t2, ms2 = cav.autotune(16)        # same shape: the cached choice, no trials
        assert t2 == tuning and ms2 == ms
    with Cavity(*dims, DT, 1.0, ce, ch) as ref:
        ref.tune(kernel=2, tile_y=8)
        ref.set_fields(f)
        ref.step(20)
        for x, y in zip(tuned, ref.get_fields()):
            assert np.array_equal(x, y)


def test_autotune_full_coefficients_keeps_unfused_kernel():
    from paper_2504_09118_gb300 import Cavity
    dims = (12, 10, 9)
    rng = np.random.default_rng(2)
    sh = (dims[2] + 1, dims[1] + 1, dims[0] + 1)
    ce = [(DT * rng.uniform(0.5, 1.0, sh)).astype(np.float32) for _ in range(3)]
    with Cavity(*dims, DT, 1.0, ce, None) as cav:
        cav.set_fields(ci.random_fields(1, *dims))
        tuning, _ = cav.autotune()
        assert tuning["kernel"] == 1


def test_batch_autotune_keeps_members():
    import torch
    from paper_2504_09118_gb300 import binding
    s = torch.cuda.Stream()
    solo = make_members(0, s, seed=21)
    for c, *_ in solo:
        c.tune(kernel=2, tile_y=8)
        c.step(5 + 19)
    ref = [c.get_fields() for c, *_ in solo]
    mem = make_members(0, s, seed=21)
    b = binding.fdtd_batch_create(0, s)
    for c, *_ in mem:
        binding.fdtd_batch_add(b, c.handle)
    binding.fdtd_batch_set_steps(b, mem[0][0].handle, 7)   # one member stops during the trials
    binding.fdtd_batch_step(b, 5)
    tuning, ms = binding.fdtd_batch_autotune(b, 16)
    assert tuning["kernel"] in (2, 3, 4) and ms > 0      # batches: no three-step kernel
    assert binding.fdtd_batch_steps_done(b) == 5
    binding.fdtd_batch_step(b, 19)
    binding.fdtd_batch_destroy(b)
    solo7 = make_members(0, s, seed=21)[0][0]
    solo7.tune(kernel=2)
    solo7.step(7)
    r7 = solo7.get_fields()
    for n, ((c, *_), r) in enumerate(zip(mem, ref)):
        want = r7 if n == 0 else r
        assert c.steps_done == (7 if n == 0 else 24)
        for x, y in zip(c.get_fields(), want):
            assert np.array_equal(x, y)
    for c, *_ in solo + mem:
        c.close()
    solo7.close()


def test_batch_retune_uses_the_size_bucket_model():
    """The first retune of a size bucket times the candidates on the live members (state restored); the
    next call in the same bucket applies the model's choice without trials; results stay bit-exact."""
    import torch
    from paper_2504_09118_gb300 import binding
    s = torch.cuda.Stream()
    solo = make_members(0, s, seed=31)
    for c, *_ in solo:
        c.tune(kernel=2, tile_y=8)
        c.step(3 + 29)
    ref = [c.get_fields() for c, *_ in solo]
    mem = make_members(0, s, seed=31)
    b = binding.fdtd_batch_create(0, s)
    try:
        for c, *_ in mem:
            binding.fdtd_batch_add(b, c.handle)
        binding.fdtd_batch_step(b, 3)
        t1, ms1, _ = binding.fdtd_batch_retune(b, 16)
        assert t1["kernel"] in (2, 3, 4) and ms1 > 0
        t2, ms2, timed2 = binding.fdtd_batch_retune(b, 16)
        assert not timed2 and t2 == t1 and ms2 == ms1
        assert binding.fdtd_batch_steps_done(b) == 3
        binding.fdtd_batch_step(b, 29)
        for (c, *_), r in zip(mem, ref):
            binding.fdtd_batch_remove(b, c.handle)
            for x, y in zip(c.get_fields(), r):
                assert np.array_equal(x, y)
    finally:
        binding.fdtd_batch_destroy(b)
