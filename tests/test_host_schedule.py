"""Host logic of the fused kernels' work split (one persistent CTA per SM), through the host-only
diagnostic fdtd_debug_tile_plan: no GPU is needed.

A tile is one x-y column over a z-chunk and costs (chunk + prologue) plane-times.  The library picks the
chunk plan with the shortest makespan of greedy list scheduling (tiles listed chunk-major, each to the CTA
that frees first, lowest index on ties) among n equal chunks (n = 1..64) and n chunks of one length plus
the rest in 1-4 pieces.  The checks: the plan tiles [0, nz); the makespan respects the two lower bounds of
any schedule and equals a heap-based list scheduler written here; it is the minimum over the candidate
family; every tile is assigned once, to the CTA that heap scheduler picks; the per-CTA loads peak at the
makespan."""
import heapq
import math

import numpy as np
import pytest

CASES = [  # (cols, nz, ctas, prologue)
    (1, 1, 152, 1), (1, 7, 1, 3), (5, 3, 152, 3), (12, 40, 8, 3), (37, 29, 16, 1), (288, 512, 152, 3),
    (387, 512, 152, 3), (576, 384, 152, 1), (100, 97, 152, 4), (9, 300, 152, 3), (153, 2, 152, 3),
]


def greedy(plan, cols, G, prologue):
    """Greedy list scheduling of the chunk-major listing: (makespan, CTA of each tile)."""
    heap = [(0, b) for b in range(G)]
    cta = []
    for length in plan:
        for _ in range(cols):
            t, b = heapq.heappop(heap)
            cta.append(b)
            heapq.heappush(heap, (t + length + prologue, b))
    return max(t for t, _ in heap), np.array(cta)


def candidates(nz):
    for n in range(1, min(nz, 64) + 1):
        yield [nz // n + (1 if q < nz % n else 0) for q in range(n)]
    for n in range(1, min(nz, 64) + 1):
        for L in range(max(1, nz // (n + 1)), nz // n + 1):
            rest = nz - n * L
            if rest <= 0:
                continue
            for pieces in range(1, min(4, rest) + 1):
                yield [L] * n + [rest // pieces + (1 if q < rest % pieces else 0) for q in range(pieces)]


@pytest.mark.parametrize("cols,nz,ctas,prologue", CASES)
def test_plan_is_valid_and_optimal_over_its_candidates(cols, nz, ctas, prologue):
    from paper_2504_09118_gb300 import binding as B
    plan, makespan, cta = B.fdtd_debug_tile_plan(cols, nz, ctas, prologue)
    G = min(ctas, cols * nz)
    assert sum(plan) == nz and min(plan) >= 1
    work = sum((length + prologue) * cols for length in plan)
    assert makespan >= math.ceil(work / G) and makespan >= max(plan) + prologue
    ref, ref_cta = greedy(plan, cols, G, prologue)
    assert makespan == ref
    best = min(greedy(p, cols, G, prologue)[0] for p in candidates(nz))
    assert makespan == best
    # every tile assigned once, to the CTA the heap scheduler picks; loads peak at the makespan
    assert cta.shape == (len(plan) * cols,) and cta.min() >= 0 and cta.max() < G
    ntiles = len(plan) * cols
    grid = min(ntiles, G)
    exp_ms, exp_cta = greedy(plan, cols, grid, prologue)
    assert np.array_equal(cta, exp_cta)
    cost = np.repeat([length + prologue for length in plan], cols)
    loads = np.bincount(cta, weights=cost, minlength=grid)
    assert loads.max() == makespan == exp_ms


def test_fixed_chunk_length():
    from paper_2504_09118_gb300 import binding as B
    plan, makespan, cta = B.fdtd_debug_tile_plan(20, 50, 16, 3, zchunk=8)
    assert plan == [8] * 6 + [2]
    assert makespan == greedy(plan, 20, 16, 3)[0]
    plan, _, _ = B.fdtd_debug_tile_plan(4, 5, 8, 1, zchunk=9, assignment=False)
    assert plan == [5]
    plan, _, _ = B.fdtd_debug_tile_plan(2, 300, 8, 1, zchunk=1, assignment=False)   # more chunks than the search tries
    assert plan == [1] * 300


def test_512_cube_schedule_efficiency():
    # 512^3, two-step kernel (60-column tiles, prologue 3) on 152 CTAs: 16-row tiles give 9 x 32 columns,
    # 12-row tiles 9 x 43; efficiency = useful plane-times / (CTAs x makespan)
    from paper_2504_09118_gb300 import binding as B
    for cols, plan_expected, eff_expected in ((288, [488, 24], 0.988), (387, [402, 55, 55], 0.979)):
        plan, makespan, _ = B.fdtd_debug_tile_plan(cols, 512, 152, 3, assignment=False)
        assert plan == plan_expected
        assert round(cols * 512 / (152 * makespan), 3) == eff_expected
        # equal chunks dealt round-robin (every CTA takes every 152nd tile): the alternative it replaced
        rr = min(math.ceil(cols * n / 152) * (math.ceil(512 / n) + 3) for n in range(1, 65))
        assert makespan < rr


@pytest.mark.parametrize("args", [(0, 8, 4, 3, 0), (4, 0, 4, 3, 0), (4, 8, 0, 3, 0), (4, 8, 4, -1, 0),
                                  (4, 8, 4, 3, -2)])
def test_bad_arguments_are_rejected(args):
    import ctypes
    from paper_2504_09118_gb300 import binding as B
    chunks = np.zeros(128, np.int32)
    n, ms = ctypes.c_int(0), ctypes.c_longlong(0)
    rc = B.lib().fdtd_debug_tile_plan(*args, chunks.ctypes.data, 128, ctypes.byref(n), ctypes.byref(ms), None)
    assert rc == B.FDTD_ERR_ARG
    # too small a capacity for the plan
    rc = B.lib().fdtd_debug_tile_plan(4, 100, 4, 3, 1, chunks.ctypes.data, 99, ctypes.byref(n), ctypes.byref(ms), None)
    assert rc == B.FDTD_ERR_ARG
