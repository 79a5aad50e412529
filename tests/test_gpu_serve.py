"""Continuous batching: requests join while others run, and each result equals the same solve run alone."""
import math

import numpy as np
import pytest

import cavity_inputs as ci
from tests.gpu_util import DT, ENERGY_DRIFT_F32, REL_L2_F32, compare_fields

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


def _oracle_run(r):
    import oracle
    ref = oracle.as_f64(r.fields)
    oracle.step(ref, DT, DT, r.steps, omp=True)
    return ref


def _random_walk_bound(steps):
    # 16-bit storage (BF16, unit roundoff 2^-8): rounding errors of a norm-preserving map add as a random
    # walk, rel-L2 about (u / sqrt(3)) sqrt(N + 1); 3x that estimate, as for the single-cavity tests
    return 3.0 * 2.0 ** -8 / math.sqrt(3.0) * math.sqrt(steps + 1)


@pytest.mark.parametrize("kernel,K", [(2, 16), (3, 16), (3, 5)])
def test_served_results_match_oracle(kernel, K):
    """Every served result against the FP64 oracle run on its own FP32 input (Eq. 2 in the order of
    Listing 1): FP32 requests per field within rel-L2 1e-4 and energy drift 1e-5, BF16 requests within
    the 16-bit random-walk bound.  The budget admits about three of the largest requests at a time, so later ones wait
    for a retirement to free memory and then join a batch whose other members are running; with K = 5
    and the two-step kernel members also join at odd batch clocks, inside a two-step pair."""
    import oracle
    from paper_2504_09118_gb300.serve import Server, device_bytes_estimate
    reqs = stream_requests(16, 7, max_side=36, max_steps=160, gap_s=0.0002)
    cap = 3 * max(device_bytes_estimate(r.nx, r.ny, r.nz, r.storage) for r in reqs)
    srv = Server(DT, hbm_budget_bytes=cap, result="fields", K=K, tuning={"kernel": kernel, "tile_y": 8})
    try:
        st = srv.run(reqs)
    finally:
        srv.close()
    assert st.n == len(reqs) and st.failed == 0 and st.max_active >= 2
    assert any(r.join_active > 0 for r in reqs)      # joined while other members of its batch ran
    done = sorted(r.t_done for r in reqs)
    waited = [r for r in reqs if r.t_admit > r.arrival_s + 1e-4 and done[0] <= r.t_admit]
    assert waited                                    # admitted only after an earlier request retired
    if K % 2:
        assert any(r.join_clock % 2 == 1 and r.join_active > 0 for r in reqs)
    for r in reqs:
        ref = _oracle_run(r)
        w0 = oracle.energy(oracle.as_f64(r.fields), DT, DT, DT)
        w1 = oracle.energy(oracle.as_f64(r.result), DT, DT, DT)
        dims = (r.nx, r.ny, r.nz)
        if r.storage == 0:
            compare_fields(r.result, ref, dims, REL_L2_F32)
            assert abs(w1 - w0) / w0 <= ENERGY_DRIFT_F32, (r.id, w0, w1)
            assert all(np.array_equal(a, b) for a, b in zip(r.result, solo(r, kernel))), r.id
        else:
            bnd = _random_walk_bound(r.steps)
            compare_fields(r.result, ref, dims, bnd)
            assert abs(w1 - w0) / w0 <= bnd, (r.id, w0, w1)
            if K % 2 == 0:   # chunk boundaries keep the two-step pairs of a solo run: same roundings
                assert all(np.array_equal(a, b) for a, b in zip(r.result, solo(r, kernel))), r.id


def test_mixed_order_stream_matches_oracle():
    """Second and fourth-order requests in one stream: each order runs in batches of its own (FP32 and
    BF16), and every result matches the FP64 oracle of its own scheme."""
    import oracle
    from paper_2504_09118_gb300 import Cavity
    from paper_2504_09118_gb300.serve import Server
    reqs = stream_requests(15, 9, max_side=32, max_steps=90)
    for r in reqs[::3]:
        r.order = 4
    srv = Server(DT, result="fields", K=16, tuning={"kernel": 3, "tile_y": 16})
    try:
        st = srv.run(reqs)
        keys = set(srv.batches)
    finally:
        srv.close()
    assert st.n == len(reqs) and st.failed == 0
    assert {(0, 4), (2, 4)} & keys and (0, 2) in keys
    for r in reqs:
        ref = oracle.as_f64(r.fields)
        (oracle.step4 if r.order == 4 else oracle.step)(ref, DT, DT, r.steps, omp=True)
        dims = (r.nx, r.ny, r.nz)
        if r.storage == 0:
            compare_fields(r.result, ref, dims, REL_L2_F32)
            if r.order == 4:   # equal to the fourth-order kernel stepping the request alone
                with Cavity(*dims, DT, 1.0, None, None, 0, order=4) as c:
                    c.set_fields(r.fields)
                    c.step(r.steps)
                    assert all(np.array_equal(a, b) for a, b in zip(r.result, c.get_fields())), r.id
        else:
            compare_fields(r.result, ref, dims, _random_walk_bound(r.steps))


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
