"""16-bit storage scales: one power-of-two scale per field (E, H) against one per component.

The library stores E as round16(s_E E) and H as round16(s_H H), one scale for the three
components of a field, s = 2^(8 - ceil(log2 max|F|)) fixed at load.  A power-of-two factor
commutes with round-to-nearest as long as the scaled value stays in the format's normal range
(FP16: [2^-14, 65504]; BF16: FP32's range), so for a component whose values lie within 2^22 of
the field's maximum (FP16) a scale of its own would store exactly the same values.  These CPU
tests check that fact, and that a 16-bit run whose components differ by 2^12 in magnitude has the
same per-component errors with either choice of scale (an emulation: FP32 stepping of Eq. 2 with
every stored value rounded to 16 bits, restated here with array slices).
"""
import math

import numpy as np

import cavity_inputs as ci
from tests.test_oracle_pins import numpy_step

DT = ci.COURANT_HALF_DT


def round_bf16(x: np.ndarray) -> np.ndarray:
    """FP32 -> BF16 (round to nearest, ties to even) -> FP32, by integer arithmetic on the bits."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16 << 16
    return b.astype(np.uint32).view(np.float32)


def round16(x: np.ndarray, storage: int) -> np.ndarray:
    x = np.asarray(x, np.float32)
    return x.astype(np.float16).astype(np.float32) if storage == 1 else round_bf16(x)


def scale_of(m: float) -> np.float32:
    return np.float32(2.0 ** (8 - math.ceil(math.log2(m)))) if m > 0 else np.float32(1.0)


def quantise(f, storage, shared: bool):
    """Stored values (in physical units) of the six components under shared or per-component scales."""
    mx = [float(np.max(np.abs(a))) for a in f]
    if shared:
        s = [scale_of(max(mx[:3]))] * 3 + [scale_of(max(mx[3:]))] * 3
    else:
        s = [scale_of(m) for m in mx]
    return s, [round16(a * sc, storage) / sc for a, sc in zip(f, s)]


def test_power_of_two_scale_commutes_with_rounding():
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(200000) * np.exp2(rng.integers(-30, 30, 200000))).astype(np.float32)
    for storage, lo, hi in ((1, 2.0 ** -14, 65504.0), (2, 2.0 ** -126, 3.0e38)):
        for k in (-20, -12, -5, 3, 12):
            s1, s2 = np.float32(2.0 ** 8), np.float32(2.0 ** (8 + k))
            ok = (np.abs(x * s1) >= lo) & (np.abs(x * s1) <= hi) & (np.abs(x * s2) >= lo) & (np.abs(x * s2) <= hi)
            a = round16(x[ok] * s1, storage) / s1
            b = round16(x[ok] * s2, storage) / s2
            assert np.array_equal(a, b), (storage, k)
    # outside FP16's normal range the scale does matter (subnormals keep fewer bits): the limit of
    # sharing a scale is a component more than 2^22 below the largest of its field
    tiny = np.float32(2.0 ** -25) * (1 + np.arange(1, 100, dtype=np.float32) / np.float32(1000))
    a = round16(tiny * np.float32(256), 1) / np.float32(256)
    b = round16(tiny * np.float32(2.0 ** 30), 1) / np.float32(2.0 ** 30)
    assert not np.array_equal(a, b)


def tm_plus_small_state(nx, ny, nz, seed, eps=2.0 ** -12):
    """z-invariant random (Ez, Hx, Hy), which the curl keeps decoupled from (Ex, Ey, Hz), plus a small
    random perturbation of all six components: Ex, Ey, Hz stay about eps times the others."""
    rng = np.random.default_rng(seed)
    shp = (nz + 1, ny + 1, nx + 1)
    f = [np.zeros(shp, np.float32) for _ in range(6)]
    for c in (2, 3, 4):
        plane = rng.uniform(-1, 1, (ny + 1, nx + 1)).astype(np.float32)
        f[c][:] = plane[None, :, :]
    small = ci.random_fields(seed, nx, ny, nz)
    for c in range(6):
        f[c] = (f[c] + np.float32(eps) * small[c]).astype(np.float32)
        f[c][~ci.extent_mask(ci.COMPONENTS[c], nx, ny, nz)] = 0
    for c, name in enumerate(("Ex", "Ey", "Ez")):
        f[c][ci.tangential_e_mask(name, nx, ny, nz)] = 0
    return f


def run16(f0, steps, storage, shared):
    """Emulated 16-bit run: the scales are fixed at load (as the library does), every step computes in
    FP32 from the stored values and stores again."""
    nx, ny, nz = f0[0].shape[2] - 1, f0[0].shape[1] - 1, f0[0].shape[0] - 1
    s, f = quantise(f0, storage, shared)
    c = [np.full(f0[0].shape, DT, np.float32)] * 3
    for _ in range(steps):
        numpy_step(f, c, c)
        f = [round16(a * sc, storage) / sc for a, sc in zip(f, s)]
    return f


def errors(got, ref, nx, ny, nz):
    norm = math.sqrt(sum(float(np.sum(r ** 2)) for r in ref))
    own, state = {}, {}
    for c, name in enumerate(ci.COMPONENTS):
        m = ci.extent_mask(name, nx, ny, nz)
        d = float(np.linalg.norm(got[c][m].astype(np.float64) - ref[c][m]))
        own[name] = d / float(np.linalg.norm(ref[c][m]))
        state[name] = d / norm
    return own, state


def test_shared_and_per_component_scales_give_the_same_errors():
    nx, ny, nz = 20, 18, 14
    steps = 60
    f0 = tm_plus_small_state(nx, ny, nz, 3)
    mags = [float(np.sqrt(np.mean(a.astype(np.float64) ** 2))) for a in f0]
    assert min(mags[2], mags[3], mags[4]) > 1000 * max(mags[0], mags[1], mags[5])   # 2^10 apart and more
    ref = [a.astype(np.float64) for a in f0]
    c64 = [np.full(f0[0].shape, DT)] * 3
    for _ in range(steps):
        numpy_step(ref, c64, c64)
    for storage in (1, 2):
        sh = errors(run16(f0, steps, storage, True), ref, nx, ny, nz)
        pc = errors(run16(f0, steps, storage, False), ref, nx, ny, nz)
        for name in ci.COMPONENTS:
            # the same stored values up to the rare subnormal: the same errors
            assert abs(sh[0][name] - pc[0][name]) <= 0.01 * pc[0][name], (storage, name, sh[0][name], pc[0][name])
        # relative to the state, every component stays within the random-walk bound of 16-bit storage
        u = 2.0 ** -11 if storage == 1 else 2.0 ** -8
        bound = 3 * u / math.sqrt(3) * math.sqrt(steps + 1)
        assert max(sh[1].values()) <= bound
