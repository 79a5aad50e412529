"""Batches of fourth-order contexts: one persistent launch of the fused fourth-order kernel per step over
the packed tiles of every member.

The kernel computes every value with one operation sequence whatever the tiling, so a member stepped in a
batch equals the same cavity stepped alone by that kernel bit for bit (FP32 and BF16), also when members
stop at their own step counts; the kernel alone is pinned to the fourth-order oracle elsewhere, and a
batch member is compared with it here too.
"""
import numpy as np
import pytest

import cavity_inputs as ci
from tests.gpu_util import DT, REL_L2_F32, compare_fields
from tests.test_gpu_batch import DIMS

pytestmark = pytest.mark.gpu


def members(storage, stream, seed):
    from paper_2504_09118_gb300 import Cavity
    out = []
    for n, d in enumerate(DIMS):
        ce = ch = None
        if n % 2 == 0 and min(d) >= 8:
            sph = ci.sphere_list(seed + n, 3, d, 2.0, max(2.5, min(d) / 4))
            ce, ch = ci.sphere_coefficients(sph, *d, DT)
        f = ci.random_fields(seed + 100 + n, *d)
        c = Cavity(*d, DT, 1.0, ce, ch, storage, stream, order=4)
        c.set_fields(f)
        out.append((c, f, ce, ch))
    return out


@pytest.mark.parametrize("storage", [0, 2])
@pytest.mark.parametrize("use_graph", [0, 1])
def test_order4_batch_equals_alone_bitwise(storage, use_graph):
    import torch
    from paper_2504_09118_gb300 import binding
    s = torch.cuda.Stream()
    steps = [3 + 5 * n for n in range(len(DIMS))]   # every member stops at its own count
    alone = members(storage, s, 3)
    for (c, *_), n in zip(alone, steps):
        c.tune(kernel=2, tile_y=12)
        c.step(n)
    ref = [c.get_fields() for c, *_ in alone]
    mixed = members(storage, s, 3)
    b = binding.fdtd_batch_create(storage, s)
    try:
        binding.fdtd_batch_set_tuning(b, kernel=2, tile_y=12, use_graph=use_graph)
        for (c, *_), n in zip(mixed, steps):
            binding.fdtd_batch_add(b, c.handle)
            binding.fdtd_batch_set_steps(b, c.handle, n)
        binding.fdtd_batch_step(b, max(steps) + 3)
        binding.fdtd_batch_sync(b)
        for c, *_ in mixed:
            binding.fdtd_batch_remove(b, c.handle)
    finally:
        binding.fdtd_batch_destroy(b)
    for (c, *_), r, n in zip(mixed, ref, steps):
        assert c.steps_done == n
        for x, y in zip(c.get_fields(), r):
            assert np.array_equal(x, y)
    for c, *_ in alone + mixed:
        c.close()


def test_order4_batch_member_matches_oracle():
    import oracle
    import torch
    from paper_2504_09118_gb300 import binding
    s = torch.cuda.Stream()
    mem = members(0, s, 11)
    b = binding.fdtd_batch_create(0, s)
    binding.fdtd_batch_set_tuning(b, kernel=2, use_graph=1)
    for c, *_ in mem:
        binding.fdtd_batch_add(b, c.handle)
    binding.fdtd_batch_step(b, 33)
    binding.fdtd_batch_sync(b)
    for c, *_ in mem:
        binding.fdtd_batch_remove(b, c.handle)
    binding.fdtd_batch_destroy(b)
    for c, f, ce, ch in mem[:6]:
        ref = oracle.as_f64(f)
        ce64 = DT if ce is None else [x.astype(np.float64) for x in ce]
        oracle.step4(ref, ce64, DT if ch is None else ch, 33, omp=True)
        compare_fields(c.get_fields(), ref, c.dims, REL_L2_F32)
        c.close()
    for c, *_ in mem[6:]:
        c.close()


def test_batch_keeps_one_order_and_tunes_order4():
    import torch
    from paper_2504_09118_gb300 import Cavity, FdtdError, binding
    s = torch.cuda.Stream()
    mem = members(0, s, 21)[:4]
    c2 = Cavity(20, 20, 20, DT, 1.0, None, None, 0, s)
    c2.set_fields(ci.random_fields(5, 20, 20, 20))
    b = binding.fdtd_batch_create(0, s)
    try:
        for c, *_ in mem:
            binding.fdtd_batch_add(b, c.handle)
        with pytest.raises(FdtdError):   # a second-order context does not join a fourth-order batch
            binding.fdtd_batch_add(b, c2.handle)
        tuning, ms = binding.fdtd_batch_autotune(b, 16)
        assert tuning["kernel"] == 2 and tuning["tile_y"] in (4, 8, 12, 16) and ms > 0
        assert binding.fdtd_batch_steps_done(b) == 0
        binding.fdtd_batch_step(b, 5)
        binding.fdtd_batch_sync(b)
        for c, *_ in mem:
            binding.fdtd_batch_remove(b, c.handle)
            assert c.steps_done == 5
    finally:
        binding.fdtd_batch_destroy(b)
        for c, *_ in mem:
            c.close()
        c2.close()
