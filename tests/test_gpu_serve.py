"""Continuous batching: requests join while others run, and each result equals the same solve run alone."""
import numpy as np
import pytest

import cavity_inputs as ci
from tests.gpu_util import DT

pytestmark = pytest.mark.gpu


def stream_requests(n, seed, max_side=48, max_steps=300, gap_s=0.0005):
    from paper_2504_09118_gb300.serve import Request
    rng = np.random.default_rng(seed)
    reqs, t = [], 0.0
    for i in range(n):
        t += float(rng.exponential(gap_s))
        nx, ny, nz = (int(v) for v in rng.integers(12, max_side + 1, 3))
        f = ci.random_fields(1000 + i, nx, ny, nz)
        reqs.append(Request(i, t, nx, ny, nz, int(rng.integers(5, max_steps + 1)), bool(rng.random() < 0.5), f))
    return reqs


def solo(r, kernel=2):
    from paper_2504_09118_gb300 import Cavity
    with Cavity(r.nx, r.ny, r.nz, DT, 1.0, None, None, r.storage) as c:
        c.tune(kernel=kernel, tile_y=8)
        c.set_fields(r.fields)
        c.step(r.steps)
        return c.get_fields()


@pytest.mark.parametrize("kernel", [2, 3])
def test_served_results_equal_solo_runs(kernel):
    # every member joins at a 16-step chunk boundary, so with two-step launches its steps pair up as
    # in a solo two-step run (FP32 results of both kernels agree bit for bit; BF16 follows the kernel)
    from paper_2504_09118_gb300.serve import Server
    reqs = stream_requests(24, 1)
    srv = Server(DT, result="fields", K=16, tuning={"kernel": kernel, "tile_y": 8})
    try:
        st = srv.run(reqs)
    finally:
        srv.close()
    assert st.n == 24 and st.max_active >= 2          # requests overlapped on the GPU
    assert all(r.t_done >= r.t_admit >= r.arrival_s for r in reqs)
    for r in reqs:
        ref = solo(r, kernel)
        for a, b in zip(r.result, ref):
            assert np.array_equal(a, b), r.id


def test_budget_limits_concurrency():
    from paper_2504_09118_gb300.serve import Server, device_bytes_estimate
    reqs = stream_requests(10, 2, max_side=24, max_steps=20)
    cap = 2 * max(device_bytes_estimate(r.nx, r.ny, r.nz, r.storage) for r in reqs)
    srv = Server(DT, hbm_budget_bytes=cap, result="energy")
    try:
        st = srv.run(reqs)
    finally:
        srv.close()
    assert st.n == 10 and 1 <= st.max_active <= 2
    assert all(np.isfinite(r.result) for r in reqs)


def test_sequential_baseline_same_results():
    from paper_2504_09118_gb300.serve import serve_sequential
    reqs = stream_requests(6, 3, max_side=30, max_steps=25)
    st = serve_sequential(reqs, DT, result="fields")
    assert st.n == 6
    for r in reqs:
        ref = solo(r)
        for a, b in zip(r.result, ref):
            assert np.array_equal(a, b)


def test_online_retune_keeps_results():
    """With online re-tuning the batch's kernel may change between chunks; FP32 results of both fused
    kernels agree bit for bit, so every result still equals its solo run."""
    from paper_2504_09118_gb300.serve import Server
    reqs = [r for r in stream_requests(30, 3) if r.storage == 0]
    srv = Server(DT, result="fields", K=16, tuning={"kernel": 3, "tile_y": 12}, retune=True)
    try:
        st = srv.run(reqs)
    finally:
        srv.close()
    assert st.n == len(reqs)
    assert srv.retunes["timed"] + srv.retunes["model"] >= 1
    for r in reqs:
        ref = solo(r, 2)
        for a, b in zip(r.result, ref):
            assert np.array_equal(a, b), r.id


def test_failed_request_is_retired_and_the_stream_goes_on():
    """Host-side fault injection: one request's context allocation fails (as out of memory); the server
    retires it with the error and every other request still equals its solo run."""
    from paper_2504_09118_gb300 import binding
    from paper_2504_09118_gb300.serve import Server
    reqs = [r for r in stream_requests(12, 4) if r.storage == 0]
    srv = Server(DT, result="fields", K=16, tuning={"kernel": 3, "tile_y": 16})
    try:
        binding.fdtd_debug_fail_alloc(6)       # a few allocations in: inside one request's context
        st = srv.run(reqs)
    finally:
        binding.fdtd_debug_fail_alloc(-1)
        srv.close()
    failed = [r for r in reqs if r.error is not None]
    assert st.failed == len(failed) == 1 and "OOM" in failed[0].error
    assert st.n == len(reqs) - 1
    for r in reqs:
        if r.error is None:
            for a, b in zip(r.result, solo(r, 2)):
                assert np.array_equal(a, b), r.id
