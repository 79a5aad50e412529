"""Seeded fuzzing of the fused kernels' tiling: random sizes (down to one cell per axis), tile heights, ring
depths, z-chunks, graph use, step counts and coefficient modes.  With FP32 storage every fused kernel
computes the same operations per value as the unfused kernel of its order, so each run must equal the
unfused run bit for bit; the unfused kernels are pinned to the oracle by the parity tests."""
import numpy as np
import pytest

import cavity_inputs as ci
from tests.gpu_util import DT

pytestmark = pytest.mark.gpu

N_CASES = 40


def _case(seed):
    rng = np.random.default_rng(seed)
    order = int(rng.choice([2, 4]))
    dims = (int(rng.integers(1, 141)), int(rng.integers(1, 71)), int(rng.integers(1, 41)))
    steps = int(rng.integers(1, 14))
    coef = str(rng.choice(["vacuum", "spheres", "table"]))
    if order == 2:
        kernel = int(rng.choice([2, 3, 4, 5]))
        tile_y = int(rng.choice({2: [4, 8, 16], 3: [8, 12, 16], 4: [12, 16], 5: [8, 10, 12]}[kernel]))
        stages = int(rng.integers(3, 9))
    else:
        kernel = 2
        tile_y = int(rng.choice([4, 8, 12, 16]))
        stages = int(rng.integers(4, 9))
    zchunk = int(rng.choice([0, 0, int(rng.integers(1, 9))]))
    use_graph = int(rng.integers(0, 2))
    return order, dims, steps, coef, dict(kernel=kernel, tile_y=tile_y, stages=stages, zchunk=zchunk,
                                          use_graph=use_graph)


def _coefs(coef, dims, seed):
    if coef == "spheres" and min(dims) >= 4:
        sph = ci.sphere_list(seed, 3, dims, 1.0, max(1.5, min(dims) / 3))
        return ci.sphere_coefficients(sph, *dims, DT)
    if coef == "table":
        nx, ny, nz = dims
        rng = np.random.default_rng(seed)
        tup = DT * rng.uniform(0.5, 1.0, (4, 6))
        idx = rng.integers(0, 4, (nz + 1, ny + 1, nx + 1))
        return [tup[idx, c].astype(np.float32) for c in range(3)], [tup[idx, 3 + c].astype(np.float32) for c in range(3)]
    return None, None


@pytest.mark.parametrize("seed", range(N_CASES))
def test_fused_tilings_equal_unfused(seed):
    from paper_2504_09118_gb300 import Cavity
    order, dims, steps, coef, tuning = _case(1000 + seed)
    ce, ch = _coefs(coef, dims, 2000 + seed)
    f = ci.random_fields(3000 + seed, *dims)
    out = []
    for t in (dict(kernel=1), tuning):
        with Cavity(*dims, DT, 1.0, ce, ch, order=order) as cav:
            cav.tune(**t)
            cav.set_fields(f)
            cav.step(steps)
            out.append(cav.get_fields())
    for a, b, name in zip(out[0], out[1], ci.COMPONENTS):
        assert np.array_equal(a, b), (order, dims, steps, coef, tuning, name)


N_CASES_16 = 24


@pytest.mark.parametrize("seed", range(N_CASES_16))
def test_16bit_fused_tilings_agree(seed):
    # With 16-bit storage the kernels round at different points (the fused ones keep the intermediate H in
    # FP32, the two-step kernel skips one rounding per pair), so each random tile shape is compared with a
    # fixed shape of the same kernel, storage and launch sequence (step count and graph use).
    from paper_2504_09118_gb300 import Cavity
    order, dims, steps, coef, tuning = _case(4000 + seed)
    storage = 1 + seed % 2
    ce, ch = _coefs(coef, dims, 5000 + seed)
    f = ci.random_fields(6000 + seed, *dims)
    base = dict(kernel=tuning["kernel"], tile_y=12 if tuning["kernel"] == 4 else 8, use_graph=tuning["use_graph"])
    out = []
    for t in (base, tuning):
        with Cavity(*dims, DT, 1.0, ce, ch, storage, order=order) as cav:
            cav.tune(**t)
            cav.set_fields(f)
            cav.step(steps)
            out.append(cav.get_fields())
    for a, b, name in zip(out[0], out[1], ci.COMPONENTS):
        assert np.array_equal(a, b), (order, storage, dims, steps, coef, tuning, name)
