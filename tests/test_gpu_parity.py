"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same seeded inputs."""
import numpy as np
import pytest

import cavity_inputs as ci
from tests import yee_closed_forms as cf
from tests.gpu_util import DT, ENERGY_DRIFT_F32, REL_L2_F32, compare_fields, rel_l2, run_gpu

pytestmark = pytest.mark.gpu


def oracle_run(fields, ce, ch, steps, omp=True):
    import oracle
    f = oracle.as_f64(fields)
    ce64 = DT if ce is None else [np.asarray(c, np.float64) for c in ce]
    ch64 = DT if ch is None else (ch if np.isscalar(ch) else [np.asarray(c, np.float64) for c in ch])
    oracle.step(f, ce64, ch64, steps, omp=omp)
    return f, ce64, ch64


KERNELS = {"fused": {"kernel": 2}, "simple": {"kernel": 1}}


@pytest.mark.parametrize("kernel", sorted(KERNELS))
@pytest.mark.parametrize("dims,steps", [((4, 4, 4), 10), ((7, 9, 11), 25), ((32, 32, 32), 100),
                                        ((130, 67, 45), 20), ((1, 3, 2), 5), ((64, 8, 3), 7)])
def test_random_vacuum_parity(dims, steps, kernel):
    f = ci.random_fields(0, *dims)
    ref, _, _ = oracle_run(f, None, None, steps)
    got, w0, w1, d0, d1 = run_gpu(f, dims, steps=steps, tuning=KERNELS[kernel])
    compare_fields(got, ref, dims, REL_L2_F32)
    if w0 > 0:
        assert abs(w1 - w0) / w0 <= ENERGY_DRIFT_F32


@pytest.mark.parametrize("kernel", sorted(KERNELS))
def test_sphere_dielectric_parity(kernel):
    dims = (70, 53, 41)
    sph = ci.sphere_list(1, 6, dims, 4.0, 15.0)
    ce, ch = ci.sphere_coefficients(sph, *dims, DT)
    f = ci.random_fields(2, *dims)
    ref, _, _ = oracle_run(f, ce, ch, 60)
    got, w0, w1, _, _ = run_gpu(f, dims, ce=ce, ch=ch, steps=60, tuning=KERNELS[kernel])
    compare_fields(got, ref, dims, REL_L2_F32)
    assert abs(w1 - w0) / w0 <= ENERGY_DRIFT_F32


def test_per_position_h_coefficients_and_full_mode():
    # random per-position ce and ch: > 256 distinct tuples -> per-position arrays (unfused path)
    dims = (19, 14, 11)
    rng = np.random.default_rng(3)
    sh = (dims[2] + 1, dims[1] + 1, dims[0] + 1)
    ce = [(DT * rng.uniform(0.5, 1.0, sh)).astype(np.float32) for _ in range(3)]
    ch = [(DT * rng.uniform(0.5, 1.0, sh)).astype(np.float32) for _ in range(3)]
    f = ci.random_fields(4, *dims)
    ref, _, _ = oracle_run(f, ce, ch, 30)
    got, w0, w1, _, _ = run_gpu(f, dims, ce=ce, ch=ch, steps=30)
    compare_fields(got, ref, dims, REL_L2_F32)
    assert abs(w1 - w0) / w0 <= ENERGY_DRIFT_F32


def test_few_materials_with_h_coefficients_fused():
    # <= 256 distinct (ce, ch) tuples incl. per-position ch -> material-id path of the fused kernel
    dims = (66, 20, 13)
    rng = np.random.default_rng(5)
    sh = (dims[2] + 1, dims[1] + 1, dims[0] + 1)
    lv = DT * np.array([0.5, 0.75, 1.0])
    ce = [lv[rng.integers(0, 3, sh)].astype(np.float32) for _ in range(3)]
    ch = [lv[rng.integers(0, 2, sh)].astype(np.float32) for _ in range(3)]
    f = ci.random_fields(6, *dims)
    ref, _, _ = oracle_run(f, ce, ch, 40)
    got, w0, w1, _, _ = run_gpu(f, dims, ce=ce, ch=ch, steps=40, tuning={"kernel": 2})
    compare_fields(got, ref, dims, REL_L2_F32)


@pytest.mark.parametrize("tile_y", [4, 8, 16])
@pytest.mark.parametrize("stages", [3, 4, 6])
@pytest.mark.parametrize("zchunk", [0, 5])
def test_tuning_grid_parity(tile_y, stages, zchunk):
    dims = (131, 37, 29)
    sph = ci.sphere_list(7, 4, dims, 3.0, 10.0)
    ce, ch = ci.sphere_coefficients(sph, *dims, DT)
    f = ci.random_fields(8, *dims)
    ref, _, _ = oracle_run(f, ce, ch, 9)
    got, *_ = run_gpu(f, dims, ce=ce, ch=ch, steps=9,
                      tuning={"kernel": 2, "tile_y": tile_y, "stages": stages, "zchunk": zchunk})
    compare_fields(got, ref, dims, REL_L2_F32)


def test_graph_replay_matches_direct():
    import torch
    dims = (96, 40, 33)
    f = ci.random_fields(9, *dims)
    s = torch.cuda.Stream()
    a, *_ = run_gpu(f, dims, steps=37, tuning={"kernel": 2}, stream=s)
    b, *_ = run_gpu(f, dims, steps=37, tuning={"kernel": 2, "use_graph": 1}, stream=s)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_pec_bit_invariants_gpu():
    dims = (45, 38, 27)
    f = ci.random_fields(10, *dims)
    from paper_2504_09118_gb300 import Cavity
    nx, ny, nz = dims
    with Cavity(nx, ny, nz, DT) as cav:
        cav.set_fields(f)
        g0 = cav.get_fields()
        for _ in range(3):
            cav.step(7)
            g = cav.get_fields()
            for c, name in enumerate(("Ex", "Ey", "Ez")):
                assert np.all(g[c][ci.tangential_e_mask(name, nx, ny, nz)] == 0.0)
            assert np.array_equal(g[3][:nz, :ny, [0, nx]], g0[3][:nz, :ny, [0, nx]])
            assert np.array_equal(g[4][:nz, [0, ny], :nx], g0[4][:nz, [0, ny], :nx])
            assert np.array_equal(g[5][[0, nz], :ny, :nx], g0[5][[0, nz], :ny, :nx])
        assert cav.steps_done == 21


def test_tm110_closed_form_gpu():
    dims = (32, 32, 32)
    f, _ = cf.tm110(*dims, DT, 0)
    got, w0, w1, _, _ = run_gpu([a.astype(np.float32) for a in f], dims, steps=100)
    ref, _ = cf.tm110(*dims, DT, 100)
    norm = float(np.sqrt(sum(np.sum(r * r) for r in ref)))
    for c in range(6):
        assert np.linalg.norm(got[c] - ref[c]) <= 1e-5 * norm


def test_energy_and_divergence_match_oracle():
    import oracle
    dims = (23, 17, 31)
    sph = ci.sphere_list(11, 3, dims, 3.0, 8.0)
    ce, ch = ci.sphere_coefficients(sph, *dims, DT)
    f = ci.random_fields(12, *dims)
    f64 = oracle.as_f64(f)
    ce64 = [c.astype(np.float64) for c in ce]
    w_ref = oracle.energy(f64, ce64, ch, DT)
    de, dh = oracle.divergence(f64, ce64, ch)
    _, w0, w1, d0, d1 = run_gpu(f, dims, ce=ce, ch=ch, steps=50)
    # both sides form every term in FP64 from the same FP32 values: only the summation order differs
    assert abs(w0 - w_ref) / w_ref <= 1e-12
    assert abs(d0[0] - np.sqrt(np.sum(de * de))) / d0[0] <= 1e-12
    assert abs(d0[1] - np.sqrt(np.sum(dh * dh))) / d0[1] <= 1e-12
    assert abs(w1 - w0) / w0 <= ENERGY_DRIFT_F32
    assert abs(d1[0] - d0[0]) / d0[0] <= 1e-5 and abs(d1[1] - d0[1]) / d0[1] <= 1e-5


def test_device_pointer_roundtrip():
    import torch
    dims = (33, 12, 9)
    f = ci.random_fields(13, *dims)
    from paper_2504_09118_gb300 import Cavity
    dev = [torch.from_numpy(a).cuda().contiguous() for a in f]
    with Cavity(*dims, DT) as cav:
        cav.set_fields(dev, on_device=True)
        cav.step(5)
        out = [torch.empty_like(t) for t in dev]
        cav.get_fields(out, on_device=True)
        host = cav.get_fields()
    for a, b in zip(out, host):
        assert np.array_equal(a.cpu().numpy(), b)


@pytest.mark.parametrize("order", [2, 4])
def test_injected_timeout_is_reported_and_context_recovers(order):
    from paper_2504_09118_gb300 import Cavity, FdtdError, binding
    dims = (64, 32, 40)
    f = ci.random_fields(14, *dims)
    with Cavity(*dims, DT, order=order) as cav:
        cav.set_fields(f)
        binding.fdtd_debug_inject_timeout(cav.handle, 20000)   # 20 ms
        cav.step(1)
        with pytest.raises(FdtdError) as ei:
            cav.sync()
        assert ei.value.code == binding.FDTD_ERR_TIMEOUT
        # the context stays usable: reload and step normally
        cav.set_fields(f)
        cav.step(3)
        cav.sync()
        w = cav.energy()
        assert np.isfinite(w) and w > 0


def test_error_paths_gpu():
    from paper_2504_09118_gb300 import Cavity, FdtdError, binding
    with Cavity(8, 8, 8, DT) as cav:
        with pytest.raises(FdtdError) as ei:
            cav.step(1)                      # no fields yet
        assert ei.value.code == binding.FDTD_ERR_STATE
        with pytest.raises(FdtdError):
            cav.tune(tile_y=5)
    with pytest.raises(FdtdError) as ei:
        Cavity(8, 8, 8, 0.7)                   # violates Courant
    assert ei.value.code == binding.FDTD_ERR_UNSTABLE


@pytest.mark.parametrize("storage", [0, 2])
def test_prefetched_fields_load_like_set_fields(storage):
    """fdtd_prefetch_fields + fdtd_set_fields_prefetched give the same state as fdtd_set_fields, also
    when the copy runs while the context steps; misuse is reported."""
    import torch
    from paper_2504_09118_gb300 import Cavity, FdtdError
    dims = (70, 41, 33)
    f0 = ci.random_fields(15, *dims)
    f1 = ci.random_fields(16, *dims)
    pinned = [torch.from_numpy(a).pin_memory().numpy() for a in f1]
    with Cavity(*dims, DT, 1.0, None, None, storage) as ref:
        ref.set_fields(f1)
        ref.step(9)
        want = ref.get_fields()
    with Cavity(*dims, DT, 1.0, None, None, storage) as cav:
        with pytest.raises(FdtdError):
            cav.set_fields_prefetched()              # nothing prefetched
        cav.set_fields(f0)
        cav.prefetch_fields(pinned)                  # copied while the current state steps
        cav.step(40)
        with pytest.raises(FdtdError):
            cav.prefetch_fields(pinned)              # the first one is not loaded yet
        cav.set_fields_prefetched()
        assert cav.steps_done == 0
        cav.step(9)
        got = cav.get_fields()
        for a, b in zip(got, want):
            assert np.array_equal(a, b)
        cav.prefetch_fields(f1)                      # pageable arrays work too; destroy with one pending
