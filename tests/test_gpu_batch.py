"""Batches: many cavities advanced by one persistent launch per step over a packed tile list.

Every output value is produced by the same FP32 operation sequence whatever the
tiling, so a cavity stepped inside a batch must equal, bit for bit, the same
cavity stepped alone with the same kernel template (same storage and tile height).
"""
import numpy as np
import pytest

import cavity_inputs as ci
from tests.gpu_util import DT, REL_L2_F32, compare_fields

pytestmark = pytest.mark.gpu

DIMS = [(16, 17, 19), (90, 40, 33), (33, 96, 20), (64, 64, 64), (21, 16, 75), (1, 5, 7), (70, 19, 16),
        (48, 31, 50), (17, 80, 23), (96, 96, 16), (25, 25, 25), (40, 66, 40)]


def make_members(storage=0, stream=None, seed=0):
    from paper_2504_09118_gb300 import Cavity
    out = []
    for n, d in enumerate(DIMS):
        ce = ch = None
        if n % 2 == 0 and min(d) >= 8:
            sph = ci.sphere_list(seed + n, 3, d, 2.0, max(2.5, min(d) / 4))
            ce, ch = ci.sphere_coefficients(sph, *d, DT)
        f = ci.random_fields(seed + 100 + n, *d)
        c = Cavity(*d, DT, 1.0, ce, ch, storage, stream)
        c.set_fields(f)
        out.append((c, f, ce, ch))
    return out


@pytest.mark.parametrize("storage", [0, 2])
@pytest.mark.parametrize("use_graph", [0, 1])
@pytest.mark.parametrize("kernel", [2, 3])
def test_batch_equals_alone_bitwise(storage, use_graph, kernel):
    # the same kernel alone and in the batch; 37 steps: two-step launches end with a one-step launch
    import torch
    from paper_2504_09118_gb300 import binding
    s = torch.cuda.Stream()
    alone = make_members(storage, s)
    for c, *_ in alone:
        c.tune(kernel=kernel, tile_y=8)
        c.step(37)
    ref = [c.get_fields() for c, *_ in alone]
    mixed = make_members(storage, s)
    b = binding.fdtd_batch_create(storage, s)
    try:
        binding.fdtd_batch_set_tuning(b, kernel=kernel, tile_y=8, use_graph=use_graph)
        for c, *_ in mixed:
            binding.fdtd_batch_add(b, c.handle)
        assert binding.fdtd_batch_size(b) == len(DIMS)
        binding.fdtd_batch_step(b, 37)
        binding.fdtd_batch_sync(b)
        for c, *_ in mixed:
            binding.fdtd_batch_remove(b, c.handle)
    finally:
        binding.fdtd_batch_destroy(b)
    for (c, *_), r in zip(mixed, ref):
        assert c.steps_done == 37
        g = c.get_fields()
        for x, y in zip(g, r):
            assert np.array_equal(x, y)
    for c, *_ in alone + mixed:
        c.close()


@pytest.mark.parametrize("kernel", [2, 3])
def test_batch_member_matches_oracle(kernel):
    import oracle
    import torch
    from paper_2504_09118_gb300 import binding
    s = torch.cuda.Stream()
    mem = make_members(0, s, seed=7)
    b = binding.fdtd_batch_create(0, s)
    binding.fdtd_batch_set_tuning(b, kernel=kernel, use_graph=1)
    for c, *_ in mem:
        binding.fdtd_batch_add(b, c.handle)
    binding.fdtd_batch_step(b, 40)
    binding.fdtd_batch_destroy(b)   # removes the members
    for (c, f, ce, ch), d in zip(mem, DIMS):
        ref = oracle.as_f64(f)
        oracle.step(ref, ci.COURANT_HALF_DT if ce is None else [x.astype(np.float64) for x in ce],
                    ci.COURANT_HALF_DT if ch is None else ch, 40)
        compare_fields(c.get_fields(), ref, d, REL_L2_F32)
        c.close()


@pytest.mark.parametrize("kernel", [2, 3])
def test_continuous_batching_join_and_leave(kernel):
    """Members join and leave between steps (odd clocks included); each result equals its solo run."""
    import torch
    from paper_2504_09118_gb300 import binding
    s = torch.cuda.Stream()
    solo = make_members(0, s, seed=3)
    plan = [(0, 30), (5, 20), (9, 41), (12, 16)]   # (join after global step, steps to run) per member 0..3
    for (c, *_), (_, n) in zip(solo, plan):
        c.tune(kernel=2, tile_y=8)
        c.step(n)
    ref = [c.get_fields() for c, *_ in solo[:4]]
    mem = make_members(0, s, seed=3)[:4]
    b = binding.fdtd_batch_create(0, s)
    binding.fdtd_batch_set_tuning(b, kernel=kernel, tile_y=8, use_graph=1)
    remaining = {}
    t = 0
    while True:
        for n, (join, steps) in enumerate(plan):
            if join == t:
                binding.fdtd_batch_add(b, mem[n][0].handle)
                remaining[n] = steps
        if not remaining and t > max(j for j, _ in plan):
            break
        if remaining:
            k = min(remaining.values())
            nxt = [j for j, _ in plan if j > t]
            if nxt:
                k = min(k, min(nxt) - t)
            binding.fdtd_batch_step(b, k)
            t += k
            for n in list(remaining):
                remaining[n] -= k
                if remaining[n] == 0:
                    binding.fdtd_batch_remove(b, mem[n][0].handle)
                    del remaining[n]
        else:
            t = min(j for j, _ in plan if j > t)
    binding.fdtd_batch_sync(b)
    binding.fdtd_batch_destroy(b)
    for n in range(4):
        assert mem[n][0].steps_done == plan[n][1]
        for x, y in zip(mem[n][0].get_fields(), ref[n]):
            assert np.array_equal(x, y)
    for c, *_ in solo + mem:
        c.close()


def test_batch_rejects_mismatches():
    import torch
    from paper_2504_09118_gb300 import Cavity, FdtdError, binding
    s = torch.cuda.Stream()
    b = binding.fdtd_batch_create(0, s)
    try:
        c16 = Cavity(8, 8, 8, DT, 1.0, None, None, 1, s)
        c16.set_fields(ci.random_fields(1, 8, 8, 8))
        with pytest.raises(FdtdError):
            binding.fdtd_batch_add(b, c16.handle)          # storage mismatch
        c = Cavity(8, 8, 8, DT, 1.0, None, None, 0, s)
        with pytest.raises(FdtdError):
            binding.fdtd_batch_add(b, c.handle)            # no fields yet
        c.set_fields(ci.random_fields(1, 8, 8, 8))
        binding.fdtd_batch_add(b, c.handle)
        with pytest.raises(FdtdError):
            c.step(1)                                        # members are stepped through the batch
        with pytest.raises(FdtdError):
            binding.fdtd_batch_add(b, c.handle)            # already a member
        binding.fdtd_batch_remove(b, c.handle)
        c.step(1)
        c16.close()
        c.close()
    finally:
        binding.fdtd_batch_destroy(b)


@pytest.mark.parametrize("kernel", [2, 3])
def test_members_stop_at_their_own_step_counts(kernel):
    """fdtd_batch_set_steps freezes each member after its own count, inside graph-replayed chunks
    (with two-step launches, a member with an odd count takes its last step as a one-step store)."""
    import torch
    from paper_2504_09118_gb300 import binding
    s = torch.cuda.Stream()
    counts = [7, 16, 23, 40, 41, 0]
    solo = make_members(0, s, seed=11)[:len(counts)]
    for (c, *_), n in zip(solo, counts):
        c.tune(kernel=2, tile_y=8)
        c.step(n)
    ref = [c.get_fields() for c, *_ in solo]
    load = torch.cuda.Stream()   # members on their own stream: removal orders it after the batch
    mem = make_members(0, load, seed=11)[:len(counts)]
    b = binding.fdtd_batch_create(0, s)
    binding.fdtd_batch_set_tuning(b, kernel=kernel, tile_y=8, use_graph=1)
    for (c, *_), n in zip(mem, counts):
        binding.fdtd_batch_add(b, c.handle)
        binding.fdtd_batch_set_steps(b, c.handle, n)
    binding.fdtd_batch_step(b, 48)          # three 16-step graph chunks: everyone is done by then
    assert binding.fdtd_batch_steps_done(b) == 48
    for c, *_ in mem:
        binding.fdtd_batch_remove(b, c.handle)
    binding.fdtd_batch_destroy(b)
    for (c, *_), n, r in zip(mem, counts, ref):
        assert c.steps_done == n
        for x, y in zip(c.get_fields(), r):
            assert np.array_equal(x, y)
    for c, *_ in solo + mem:
        c.close()


def test_batch_switches_kernels_between_steps():
    """One-step and two-step launches interleaved in one batch: every member stays bit-identical."""
    import torch
    from paper_2504_09118_gb300 import binding
    s = torch.cuda.Stream()
    solo = make_members(0, s, seed=13)[:6]
    for c, *_ in solo:
        c.tune(kernel=2, tile_y=8)
        c.step(3 + 16 + 5 + 2)
    ref = [c.get_fields() for c, *_ in solo]
    mem = make_members(0, s, seed=13)[:6]
    b = binding.fdtd_batch_create(0, s)
    for c, *_ in mem:
        binding.fdtd_batch_add(b, c.handle)
    for kernel, n in ((3, 3), (2, 16), (3, 5), (2, 2)):
        binding.fdtd_batch_set_tuning(b, kernel=kernel, use_graph=1)
        binding.fdtd_batch_step(b, n)
    assert binding.fdtd_batch_steps_done(b) == 26
    binding.fdtd_batch_destroy(b)
    for (c, *_), r in zip(mem, ref):
        assert c.steps_done == 26
        for x, y in zip(c.get_fields(), r):
            assert np.array_equal(x, y)
    for c, *_ in solo + mem:
        c.close()
