"""The synthetic workloads match their stated recipes (seeded; no dataset is involved):

* serving stream: Poisson arrivals at 200/s (mean gap 5 ms), sides log-uniform in [16, 256] per axis
  (E[side] = 240 / ln 16 = 86.6, E[cells] = E[side]^3 = 6.5e5), steps uniform in {100..2000} (mean 1050),
  BF16 flag Bernoulli(1/2): offered load rate x E[cells] x E[steps] = 136 Gcell-updates/s;
* batch: 256 cavities with sides uniform in {16..96} per axis, vacuum or spheres with probability 1/2;
* sphere cavities: centres in the box, radii in [8, 40], eps_r in {2.25, 4.0}, Courant number 0.5.
Tolerances are several standard errors of the sample means."""
import math

import numpy as np

import cavity_inputs as ci


def test_serving_stream_recipe():
    reqs = ci.serve_stream(6, 10000)
    t = np.array([r["arrival_s"] for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0) and abs(gaps.mean() - 0.005) < 0.005 * 0.04
    sides = np.array([[r["nx"], r["ny"], r["nz"]] for r in reqs])
    assert sides.min() >= 16 and sides.max() <= 256
    e_side = 240 / math.log(16)
    assert abs(sides.mean() - e_side) < 0.02 * e_side
    assert abs(np.log(sides).mean() - math.log(64)) < 0.02          # log-uniform: mean of log = log 64
    cells = sides.prod(axis=1).astype(float)
    assert abs(cells.mean() - e_side ** 3) < 0.05 * e_side ** 3
    steps = np.array([r["steps"] for r in reqs])
    assert steps.min() >= 100 and steps.max() <= 2000 and abs(steps.mean() - 1050) < 15
    assert abs(np.mean([r["bf16"] for r in reqs]) - 0.5) < 0.02
    offered = 200.0 * e_side ** 3 * 1050 / 1e9
    assert abs(offered - 136.3) < 0.5
    assert ci.serve_stream(6, 50) == reqs[:50]          # seeded: a prefix of the same stream


def test_batch_recipe():
    cav = ci.batch_cavities(5)
    assert len(cav) == 256
    sides = np.array([[c["nx"], c["ny"], c["nz"]] for c in cav])
    assert sides.min() >= 16 and sides.max() <= 96 and abs(sides.mean() - 56) < 3
    frac = np.mean([c["spheres"] is not None for c in cav])
    assert abs(frac - 0.5) < 0.1
    total = sides.prod(axis=1).sum()
    assert 3.5e7 < total < 5.5e7                         # about 256 x 56^3 = 4.5e7 cells
    for c in cav:
        for (cx, cy, cz, r, e) in c["spheres"] or []:
            assert 0 <= cx <= c["nx"] and 0 <= cy <= c["ny"] and 0 <= cz <= c["nz"]
            assert r >= 2.0 and e in (2.25, 4.0)


def test_sphere_cavity_recipe_and_courant():
    n = (512, 512, 512)
    sph = ci.sphere_list(1, 32, n, 8.0, 40.0)
    assert len(sph) == 32
    for (cx, cy, cz, r, e) in sph:
        assert all(0 <= c <= b for c, b in zip((cx, cy, cz), n)) and 8.0 <= r <= 40.0 and e in (2.25, 4.0)
    assert {e for *_, e in sph} == {2.25, 4.0}
    dt = ci.COURANT_HALF_DT
    assert abs(math.sqrt(3) * dt - 0.5) < 1e-15           # Courant number 0.5 at dx = 1
    ce, ch = ci.sphere_coefficients(sph[:4], 40, 40, 40, dt)
    assert max(float(c.max()) for c in ce) * ch * 3 <= 0.25 + 1e-7   # local Courant bound 3 ce ch <= 1 with margin
