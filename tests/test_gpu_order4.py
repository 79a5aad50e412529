"""GPU parity of the fourth-order (2,4) scheme (fdtd_set_order(ctx, 4)) with the FP64 oracle's step4,
through the C ABI: unfused and fused kernels, every coefficient mode, ragged and degenerate sizes,
16-bit storage, currents and probes, the scheme's energy and divergences, and its API rules."""
import math

import numpy as np
import pytest

import cavity_inputs as ci
from tests import yee_closed_forms as cf
from tests.gpu_util import DT, ENERGY_DRIFT_F32, REL_L2_F32, compare_fields

pytestmark = pytest.mark.gpu

TUNINGS = {
    "simple": dict(kernel=1),
    "fused8": dict(kernel=2, tile_y=8, stages=5),
    "fused4": dict(kernel=2, tile_y=4, stages=4),
    "fused16": dict(kernel=2, tile_y=16, stages=4),
    "fused12": dict(kernel=2, tile_y=12, stages=5),
    "fused8_s8_graph": dict(kernel=2, tile_y=8, stages=8, use_graph=1),
    "auto": dict(kernel=0),
}


def oracle4(fields, ce, ch, steps, **kw):
    import oracle
    f = oracle.as_f64(fields)
    ce64 = DT if ce is None else (ce if np.isscalar(ce) else [np.asarray(c, np.float64) for c in ce])
    ch64 = DT if ch is None else (ch if np.isscalar(ch) else [np.asarray(c, np.float64) for c in ch])
    oracle.step4(f, ce64, ch64, steps, omp=True, **kw)
    return f, ce64, ch64


def run4(fields, dims, ce=None, ch=None, steps=1, storage=0, tuning=None):
    from paper_2504_09118_gb300 import Cavity
    with Cavity(*dims, DT, 1.0, ce, ch, storage, order=4) as cav:
        if tuning:
            cav.tune(**tuning)
        cav.set_fields(fields)
        w0 = cav.energy()
        d0 = cav.divergence()
        cav.step(steps)
        w1 = cav.energy()
        d1 = cav.divergence()
        out = cav.get_fields()
    return out, w0, w1, d0, d1


def table_coefficients(seed, dims, ntuples=5):
    """Per-cell coefficient tuples drawn from a small set: material-id mode with non-uniform ch."""
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    tup = DT * rng.uniform(0.5, 1.0, (ntuples, 6))
    idx = rng.integers(0, ntuples, (nz + 1, ny + 1, nx + 1))
    ce = [tup[idx, c].astype(np.float32) for c in range(3)]
    ch = [tup[idx, 3 + c].astype(np.float32) for c in range(3)]
    return ce, ch


@pytest.mark.parametrize("tuning", sorted(TUNINGS))
@pytest.mark.parametrize("dims,steps", [((130, 37, 29), 20), ((64, 16, 12), 9), ((7, 9, 11), 25),
                                        ((1, 3, 2), 5), ((3, 2, 2), 6), ((65, 5, 70), 17)])
def test_random_vacuum_parity(dims, steps, tuning):
    f = ci.random_fields(40, *dims)
    ref, _, _ = oracle4(f, None, None, steps)
    got, w0, w1, _, _ = run4(f, dims, steps=steps, tuning=TUNINGS[tuning])
    compare_fields(got, ref, dims, REL_L2_F32)
    if w0 > 0:
        assert abs(w1 - w0) / w0 <= ENERGY_DRIFT_F32


@pytest.mark.parametrize("tuning", ["simple", "fused8", "fused12", "fused16", "auto"])
def test_sphere_dielectric_parity(tuning):
    dims = (70, 53, 41)
    sph = ci.sphere_list(41, 6, dims, 4.0, 15.0)
    ce, ch = ci.sphere_coefficients(sph, *dims, DT)
    f = ci.random_fields(42, *dims)
    ref, _, _ = oracle4(f, ce, ch, 40)
    got, w0, w1, _, _ = run4(f, dims, ce=ce, ch=ch, steps=40, tuning=TUNINGS[tuning])
    compare_fields(got, ref, dims, REL_L2_F32)
    assert abs(w1 - w0) / w0 <= ENERGY_DRIFT_F32


@pytest.mark.parametrize("tuning", ["simple", "fused8", "fused4", "fused12", "fused16"])
def test_nonuniform_ch_table_parity(tuning):
    dims = (67, 21, 13)
    ce, ch = table_coefficients(43, dims)
    f = ci.random_fields(44, *dims)
    ref, _, _ = oracle4(f, ce, ch, 15)
    got, w0, w1, _, _ = run4(f, dims, ce=ce, ch=ch, steps=15, tuning=TUNINGS[tuning])
    compare_fields(got, ref, dims, REL_L2_F32)
    assert abs(w1 - w0) / w0 <= ENERGY_DRIFT_F32


def test_per_position_arrays_parity():
    dims = (19, 14, 11)
    rng = np.random.default_rng(45)
    sh = (dims[2] + 1, dims[1] + 1, dims[0] + 1)
    ce = [(DT * rng.uniform(0.5, 1.0, sh)).astype(np.float32) for _ in range(3)]
    ch = [(DT * rng.uniform(0.5, 1.0, sh)).astype(np.float32) for _ in range(3)]
    f = ci.random_fields(46, *dims)
    ref, _, _ = oracle4(f, ce, ch, 20)
    got, w0, w1, _, _ = run4(f, dims, ce=ce, ch=ch, steps=20, tuning=dict(kernel=0))
    compare_fields(got, ref, dims, REL_L2_F32)
    assert abs(w1 - w0) / w0 <= ENERGY_DRIFT_F32


@pytest.mark.parametrize("coef", ["vacuum", "spheres", "table"])
@pytest.mark.parametrize("dims", [(130, 37, 29), (65, 5, 70), (2, 3, 4)])
def test_fused_bitwise_equals_unfused(coef, dims):
    """Both kernels evaluate the same expression in the same order: FP32 results are identical."""
    ce = ch = None
    if coef == "spheres":
        ce, ch = ci.sphere_coefficients(ci.sphere_list(47, 4, dims, 2.0, 9.0), *dims, DT)
    elif coef == "table":
        ce, ch = table_coefficients(48, dims)
    f = ci.random_fields(49, *dims)
    a = run4(f, dims, ce, ch, steps=11, tuning=TUNINGS["simple"])[0]
    for name in ("fused8", "fused4", "fused12", "fused16"):
        b = run4(f, dims, ce, ch, steps=11, tuning=TUNINGS[name])[0]
        for c in range(6):
            assert np.array_equal(a[c], b[c]), (name, ci.COMPONENTS[c])


@pytest.mark.parametrize("tuning", ["simple", "fused8"])
def test_tm110_closed_form(tuning):
    dims, steps = (32, 32, 32), 100
    f, _ = cf.tm110(*dims, DT, 0, order=4)
    g, _ = cf.tm110(*dims, DT, steps, order=4)
    got = run4([a.astype(np.float32) for a in f], dims, steps=steps, tuning=TUNINGS[tuning])[0]
    compare_fields(got, g, dims, 1e-4)


def test_energy_and_divergence_match_oracle():
    import oracle
    dims = (37, 29, 23)
    ce, ch = table_coefficients(50, dims)
    f = ci.random_fields(51, *dims)
    f64 = oracle.as_f64(f)
    ce64 = [c.astype(np.float64) for c in ce]
    ch64 = [c.astype(np.float64) for c in ch]
    _, w0, _, d0, _ = run4(f, dims, ce, ch, steps=0, tuning=TUNINGS["fused8"])
    assert abs(w0 - oracle.energy4(f64, ce64, ch64, DT)) <= 1e-6 * abs(w0)
    de, dh = oracle.divergence4(f64, ce64, ch64)
    assert abs(d0[0] - math.sqrt(float(np.sum(de * de)))) <= 1e-5 * d0[0]
    assert abs(d0[1] - math.sqrt(float(np.sum(dh * dh)))) <= 1e-5 * d0[1]
    # and both stay put over a run (invariants of the scheme)
    _, w0, w1, d0, d1 = run4(f, dims, ce, ch, steps=64, tuning=TUNINGS["fused8_s8_graph"])
    assert abs(w1 - w0) / w0 <= ENERGY_DRIFT_F32
    assert abs(d1[0] - d0[0]) <= 1e-5 * d0[0] and abs(d1[1] - d0[1]) <= 1e-5 * d0[1]


@pytest.mark.parametrize("storage", [1, 2])
def test_16bit_storage_within_bound(storage):
    dims, steps = (66, 40, 30), 30
    sph = ci.sphere_list(52, 5, dims, 3.0, 12.0)
    ce, ch = ci.sphere_coefficients(sph, *dims, DT)
    f = ci.random_fields(53, *dims)
    ref, _, _ = oracle4(f, ce, ch, steps)
    u = 2.0 ** -11 if storage == 1 else 2.0 ** -8      # unit roundoff of the storage format
    bound = 3 * u / math.sqrt(3) * math.sqrt(steps + 1)
    for name in ("simple", "fused8"):
        got = run4(f, dims, ce, ch, steps=steps, storage=storage, tuning=TUNINGS[name])[0]
        compare_fields(got, ref, dims, bound)


@pytest.mark.parametrize("tuning", ["simple", "fused8"])
def test_currents_and_probes(tuning):
    from paper_2504_09118_gb300 import Cavity
    dims = (40, 33, 21)
    sources = [(2, 11, 7, 5), (0, 20, 16, 10), (1, 30, 4, 15)]
    probes = [(2, 11, 7, 5), (3, 20, 16, 10), (5, 39, 32, 20)]
    f = ci.random_fields(54, *dims)
    waves = np.random.default_rng(55).uniform(-3.0, 3.0, (len(sources), 30))
    import oracle
    ref = oracle.as_f64(f)
    steps = 37
    trace = np.zeros((len(probes), steps))
    for n in range(steps):
        oracle.step4(ref, DT, DT, 1, sources=sources, wave=waves, n0=n)
        for p, (c, i, j, k) in enumerate(probes):
            trace[p, n] = ref[c][k, j, i]
    with Cavity(*dims, DT, 1.0, order=4) as cav:
        cav.tune(**TUNINGS[tuning], use_graph=1)
        cav.set_fields(f)
        cav.set_sources(sources, waves)
        cav.set_probes(probes, 64)
        cav.step(steps)
        got = cav.get_fields()
        tr = cav.get_probes()
    compare_fields(got, ref, dims, REL_L2_F32)
    for p in range(len(probes)):
        assert float(np.linalg.norm(tr[p] - trace[p])) <= REL_L2_F32 * float(np.linalg.norm(trace[p]))


def test_api_rules():
    from paper_2504_09118_gb300 import Cavity, FdtdError, binding
    dims = (16, 12, 10)
    f = ci.random_fields(56, *dims)
    with Cavity(*dims, DT, 1.0) as cav:
        assert cav.order == 2
        with pytest.raises(FdtdError):
            binding.fdtd_set_order(cav.handle, 3)
        cav.tune(kernel=3)
        with pytest.raises(FdtdError):          # the two-step kernel is second-order only
            binding.fdtd_set_order(cav.handle, 4)
        cav.tune(kernel=2)
        binding.fdtd_set_order(cav.handle, 4)
        with pytest.raises(FdtdError):
            cav.tune(kernel=3)
        with pytest.raises(FdtdError):
            cav.tune(kernel=2, stages=3)
        cav.set_fields(f)
        other = Cavity(*dims, DT, 1.0)
        other.set_fields(f)
        b = binding.fdtd_batch_create(0)
        try:
            binding.fdtd_batch_add(b, other.handle)     # a second-order batch
            with pytest.raises(FdtdError):               # takes no fourth-order member
                binding.fdtd_batch_add(b, cav.handle)
            with pytest.raises(FdtdError):               # and its members keep their order
                binding.fdtd_set_order(other.handle, 4)
            binding.fdtd_batch_remove(b, other.handle)
        finally:
            binding.fdtd_batch_destroy(b)
            other.close()
        # back to Eq. 2: the step is the second-order oracle's again
        binding.fdtd_set_order(cav.handle, 2)
        cav.step(5)
        got = cav.get_fields()
    import oracle
    ref = oracle.step(oracle.as_f64(f), DT, DT, 5)
    compare_fields(got, ref, dims, REL_L2_F32)
    # a time step stable for Eq. 2 but not for the (2,4) scheme: sqrt(3) dt / dx = 0.9, times 7/6 > 1
    with Cavity(*dims, 0.9 / math.sqrt(3), 1.0) as cav:
        with pytest.raises(FdtdError) as e:
            binding.fdtd_set_order(cav.handle, 4)
        assert e.value.code == binding.FDTD_ERR_UNSTABLE
        assert cav.order == 2


def test_autotune_restores_state():
    from paper_2504_09118_gb300 import Cavity
    dims = (96, 40, 33)
    f = ci.random_fields(57, *dims)
    with Cavity(*dims, DT, 1.0, order=4) as cav:
        cav.set_fields(f)
        tuning, ms = cav.autotune(16)
        assert tuning["kernel"] == 2 and tuning["tile_y"] in (4, 8, 12, 16) and ms > 0
        assert cav.steps_done == 0
        assert all(np.array_equal(a, b) for a, b in zip(cav.get_fields(), f))
        cav.step(12)
        got = cav.get_fields()
    ref, _, _ = oracle4(f, None, None, 12)
    compare_fields(got, ref, dims, REL_L2_F32)
