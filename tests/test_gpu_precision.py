"""FP16 / BF16 storage (FP32 arithmetic): error against the FP64 oracle and the FP32 GPU run.

Tolerance derivation: a 16-bit store rounds to nearest with unit roundoff u
(FP16: 2^-11, BF16: 2^-8), a relative error of RMS about u/sqrt(3) per value.
Each leapfrog step stores every field once and the Yee map preserves the
discrete energy norm, so rounding errors add as a random walk: after N steps
(plus the quantisation of the initial state) the relative L2 error is about
(u/sqrt(3)) * sqrt(N + 1).  The tests allow 3x that estimate.
"""
import math

import numpy as np
import pytest

import cavity_inputs as ci
from tests.gpu_util import DT, rel_l2, run_gpu

pytestmark = pytest.mark.gpu

U = {1: 2.0 ** -11, 2: 2.0 ** -8}


def bound(storage, steps):
    return 3.0 * U[storage] / math.sqrt(3.0) * math.sqrt(steps + 1)


def field_errors(got, ref, dims):
    nx, ny, nz = dims
    num = den = 0.0
    for c, name in enumerate(ci.COMPONENTS):
        m = ci.extent_mask(name, nx, ny, nz)
        num += float(np.sum((np.asarray(got[c], np.float64)[m] - np.asarray(ref[c], np.float64)[m]) ** 2))
        den += float(np.sum(np.asarray(ref[c], np.float64)[m] ** 2))
    return math.sqrt(num / den)


@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("kernel", [1, 2])
def test_16bit_storage_vs_oracle(storage, kernel):
    import oracle
    dims = (70, 45, 37)
    steps = 100
    sph = ci.sphere_list(3, 5, dims, 4.0, 12.0)
    ce, ch = ci.sphere_coefficients(sph, *dims, DT)
    f = ci.random_fields(4, *dims)
    ref = oracle.as_f64(f)
    oracle.step(ref, [c.astype(np.float64) for c in ce], ch, steps, omp=True)
    got, w0, w1, d0, d1 = run_gpu(f, dims, ce=ce, ch=ch, steps=steps, storage=storage, tuning={"kernel": kernel})
    err = field_errors(got, ref, dims)
    assert err <= bound(storage, steps), (err, bound(storage, steps))
    assert err >= 0.05 * U[storage]          # the run really stored 16-bit values
    # energy: rounding is unbiased, the drift stays far below the field error
    assert abs(w1 - w0) / w0 <= bound(storage, steps)


@pytest.mark.parametrize("storage", [1, 2])
def test_16bit_pec_and_far_faces_exact(storage):
    dims = (40, 33, 21)
    f = ci.random_fields(5, *dims)
    from paper_2504_09118_gb300 import Cavity
    nx, ny, nz = dims
    with Cavity(nx, ny, nz, DT, 1.0, None, None, storage) as cav:
        cav.set_fields(f)
        g0 = cav.get_fields()
        cav.step(25)
        g = cav.get_fields()
    for c, name in enumerate(("Ex", "Ey", "Ez")):
        assert np.all(g[c][ci.tangential_e_mask(name, nx, ny, nz)] == 0.0)
    assert np.array_equal(g[3][:nz, :ny, [0, nx]], g0[3][:nz, :ny, [0, nx]])
    assert np.array_equal(g[5][[0, nz], :ny, :nx], g0[5][[0, nz], :ny, :nx])


@pytest.mark.parametrize("storage", [1, 2])
def test_16bit_fused_independent_of_tiling(storage):
    # (the unfused pair re-reads the rounded H it just stored while the fused kernel feeds the
    # FP32 H^{n+1/2} straight into the E update, so the two round differently; each is held to the
    # oracle bound above.  Within the fused kernel every value follows one operation sequence.)
    dims = (67, 29, 18)
    f = ci.random_fields(6, *dims)
    a, *_ = run_gpu(f, dims, steps=12, storage=storage, tuning={"kernel": 2, "tile_y": 8})
    b, *_ = run_gpu(f, dims, steps=12, storage=storage, tuning={"kernel": 2, "tile_y": 8, "zchunk": 5, "stages": 3})
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def _per_field(got, ref, dims):
    nx, ny, nz = dims
    norm = math.sqrt(sum(float(np.sum(np.asarray(r, np.float64) ** 2)) for r in ref))
    own, state = {}, {}
    for c, name in enumerate(ci.COMPONENTS):
        m = ci.extent_mask(name, nx, ny, nz)
        d = float(np.linalg.norm(np.asarray(got[c], np.float64)[m] - np.asarray(ref[c], np.float64)[m]))
        own[name] = d / float(np.linalg.norm(np.asarray(ref[c], np.float64)[m]))
        state[name] = d / norm
    return own, state


@pytest.mark.parametrize("storage", [1, 2])
def test_16bit_per_field_errors_with_components_far_apart(storage):
    """One storage scale per field (E, H), components 2^12 apart in magnitude, per-field errors against
    the FP64 oracle.  (a) Random state with Ex and Hz scaled by 2^-12: the curl mixes the components
    within a step, and every component, the small two included, stays within the random-walk bound of
    its own norm.  (b) A z-invariant (Ez, Hx, Hy) field plus a 2^-12 perturbation, which keeps
    (Ex, Ey, Hz) about 2^12 below the others for the whole run: relative to the state every component
    is within the bound, the large ones also relative to their own norms.  The small ones carry
    errors set by the rounding of the large ones they couple to, which a scale of their own would not
    change (tests/test_storage_scale.py shows the same errors with per-component scales)."""
    import oracle
    from tests.test_storage_scale import tm_plus_small_state
    dims = (40, 33, 21)
    steps = 60
    b = bound(storage, steps)
    f = ci.random_fields(8, *dims)
    for c in (0, 5):
        f[c] = (f[c] * np.float32(2.0 ** -12)).astype(np.float32)
    for case, fields in (("scaled", f), ("tm_plus_small", tm_plus_small_state(*dims, 9))):
        ref = oracle.as_f64(fields)
        oracle.step(ref, DT, DT, steps, omp=True)
        got, w0, w1, *_ = run_gpu(fields, dims, steps=steps, storage=storage)
        own, state = _per_field(got, ref, dims)
        print(f"storage {storage} {case}: own-norm " + " ".join(f"{k} {v:.2e}" for k, v in own.items()) +
              " | state-norm " + " ".join(f"{k} {v:.2e}" for k, v in state.items()))
        assert max(state.values()) <= b, (case, state)
        large = ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz") if case == "scaled" else ("Ez", "Hx", "Hy")
        for name in large:
            assert own[name] <= b, (case, name, own[name])
        assert abs(w1 - w0) / w0 <= b
