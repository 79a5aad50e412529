"""Point currents (Eq. 1's J) and probes on the GPU against the FP64 oracle's step with currents."""
import math

import numpy as np
import pytest

import cavity_inputs as ci
from tests.gpu_util import DT, REL_L2_F32, compare_fields
from tests.test_oracle_sources import pulse, spectrum_peaks
from tests.yee_matrix import mode_frequencies

pytestmark = pytest.mark.gpu

DIMS = (40, 33, 21)
SOURCES = [(2, 11, 7, 5), (0, 20, 16, 10), (1, 30, 4, 15), (2, 11, 7, 5)]   # the last adds to the first
PROBES = [(2, 11, 7, 5), (0, 3, 3, 3), (3, 20, 16, 10), (5, 39, 32, 20), (4, 7, 9, 11)]


def oracle_run(f, ce, ch, steps, waves, dx=1.0):
    import oracle
    ref = oracle.as_f64(f)
    ce64 = DT if ce is None else [c.astype(np.float64) for c in ce]
    ch64 = DT if ch is None else ch
    trace = np.zeros((len(PROBES), steps))
    for n in range(steps):
        oracle.step_sources(ref, ce64, ch64, 1, SOURCES, waves, n0=n, dx=dx)
        for p, (c, i, j, k) in enumerate(PROBES):
            trace[p, n] = ref[c][k, j, i]
    return ref, trace


def setup():
    sph = ci.sphere_list(8, 4, DIMS, 3.0, 9.0)
    ce, ch = ci.sphere_coefficients(sph, *DIMS, DT)
    f = ci.random_fields(9, *DIMS)
    rng = np.random.default_rng(10)
    waves = rng.uniform(-3.0, 3.0, (len(SOURCES), 30))
    return ce, ch, f, waves


@pytest.mark.parametrize("tuning", [dict(kernel=1), dict(kernel=2, use_graph=0), dict(kernel=2, use_graph=1),
                                    dict(kernel=3, use_graph=1), dict(kernel=4, use_graph=1),
                                    dict(kernel=5, use_graph=1)])
def test_currents_and_probes_match_oracle(tuning):
    from paper_2504_09118_gb300 import Cavity
    ce, ch, f, waves = setup()
    steps = 37                      # two 16-step graphs and 5 single steps; the currents stop at 30
    ref, trace = oracle_run(f, ce, ch, steps, waves)
    with Cavity(*DIMS, DT, 1.0, ce, ch) as cav:
        cav.tune(**tuning)
        cav.set_fields(f)
        cav.set_sources(SOURCES, waves)
        cav.set_probes(PROBES, 64)
        cav.step(steps)
        got = cav.get_fields()
        tr = cav.get_probes()
    compare_fields(got, ref, DIMS, REL_L2_F32)
    assert tr.shape == (len(PROBES), steps)
    for p in range(len(PROBES)):
        scale = max(float(np.linalg.norm(trace[p])), 1e-30)
        assert float(np.linalg.norm(tr[p] - trace[p])) / scale <= REL_L2_F32, p


def test_currents_bf16_within_storage_bound():
    from paper_2504_09118_gb300 import Cavity
    ce, ch, f, waves = setup()
    steps = 40
    ref, trace = oracle_run(f, ce, ch, steps, waves)
    with Cavity(*DIMS, DT, 1.0, ce, ch, 2) as cav:
        cav.set_fields(f)
        cav.set_sources(SOURCES, waves)
        cav.set_probes(PROBES, steps)
        cav.step(steps)
        got = cav.get_fields()
    bound = 3 * 2.0 ** -8 / math.sqrt(3) * math.sqrt(steps + 1)
    compare_fields(got, ref, DIMS, bound)


def test_gpu_driven_cavity_resonances():
    """The resonance pin of the oracle, through the GPU path: currents, steps and probes on the device."""
    from paper_2504_09118_gb300 import Cavity
    nx, ny, nz = 12, 10, 8
    zero = [np.zeros((nz + 1, ny + 1, nx + 1), np.float32) for _ in range(6)]
    N = 4096
    with Cavity(nx, ny, nz, DT, 1.0) as cav:
        cav.tune(kernel=2, use_graph=1)
        cav.set_fields(zero)
        cav.set_sources([(2, 3, 4, 2)], pulse(200, 12.0, 50.0)[None, :])
        cav.set_probes([(2, 8, 6, 5)], N)
        cav.step(N)
        tr = cav.get_probes()[0]
        w_end = cav.energy()
    modes = mode_frequencies(nx, ny, nz, DT, DT, DT)
    peaks, bin_w = spectrum_peaks(tr.astype(np.float64), 3, 0.21)
    assert len(peaks) == 3
    for w in peaks:
        assert np.min(np.abs(modes - w)) <= bin_w, w
    assert w_end > 0


def test_recording_restarts_and_bad_arguments():
    from paper_2504_09118_gb300 import Cavity, FdtdError, binding
    nx, ny, nz = 16, 12, 10
    f = ci.random_fields(3, nx, ny, nz)
    with Cavity(nx, ny, nz, DT, 1.0) as cav:
        cav.set_fields(f)
        cav.step(5)
        cav.set_probes([(0, 4, 4, 4)], 10)   # records from the next step on
        cav.step(3)
        assert cav.get_probes().shape == (1, 3)
        cav.set_fields(f)                    # restarts the recording
        assert cav.get_probes().shape == (1, 0)
        cav.step(12)
        assert cav.get_probes().shape == (1, 10)   # capacity reached
        for bad in ([(0, 4, 0, 4)], [(1, 0, 4, 4)], [(2, 4, 4, 10)], [(3, 4, 4, 4)], [(2, 4, 12, 4)]):
            with pytest.raises(FdtdError):   # tangential, outside, or not an E component
                cav.set_sources(bad, [[1.0]])
        with pytest.raises(FdtdError):
            cav.set_probes([(6, 1, 1, 1)], 4)
        with pytest.raises(FdtdError):
            cav.autotune()                   # tune before currents or probes
        b = binding.fdtd_batch_create(0)
        try:
            with pytest.raises(FdtdError):
                binding.fdtd_batch_add(b, cav.handle)
        finally:
            binding.fdtd_batch_destroy(b)
        cav.set_probes([], 1)
        cav.set_sources([], [])
        cav.autotune()                       # allowed again


@pytest.mark.parametrize("kernel", [3, 5])
def test_multi_step_kernels_resume_after_currents(kernel):
    """While currents are set a multi-step tuning steps one step per launch; removing them resumes the two-
    or three-step launches.  With FP32 storage both give the one-step kernel's values bit for bit."""
    from paper_2504_09118_gb300 import Cavity
    ce, ch, f, waves = setup()
    runs = []
    for k in (2, kernel):
        with Cavity(*DIMS, DT, 1.0, ce, ch) as cav:
            cav.tune(kernel=k, use_graph=1)
            cav.set_fields(f)
            cav.set_sources(SOURCES, waves)
            cav.step(31)
            cav.set_sources([], [])
            cav.step(38)
            assert cav.steps_done == 69
            runs.append(cav.get_fields())
    for name, a, b in zip(ci.COMPONENTS, *runs):
        assert np.array_equal(a, b), name
