"""Seeded synthetic inputs for the PEC box-cavity workloads.

This module is the only code shared by the CUDA path's tests/bench and the
FP64 oracle.  It draws random numbers and lays them out; it contains none of
the Yee update arithmetic.

Workload recipe (the paper benchmarks "a simple 3D cavity with PEC boundary
conditions" started from "a random initial state", Sec. 4 and Fig. 1b):

* fields: six components, i.i.d. uniform[-1, 1) from a counter-based
  SplitMix64 stream keyed on (seed, component, canonical index), rounded to
  float32; tangential E on the six faces and entries outside a component's
  Yee extent are zero;
* dielectric: background eps_r = 1 plus seeded random spheres (centre uniform
  in the box, radius uniform in [rmin, rmax], eps_r drawn from a small set),
  sampled at each E component's own Yee position, later spheres overriding
  earlier ones; mu_r = 1;
* coefficients handed to the solver: ce = dt / (eps_r * dx) at the Ex, Ey, Ez
  positions and ch = dt / (mu_r * dx) (a scalar when mu_r = 1).

Canonical layout (every component): a C-contiguous float array of shape
(nz+1, ny+1, nx+1), x fastest.  Component c at canonical index (i, j, k) sits at
its Yee position:

    Ex (i+1/2, j, k)      i < nx, j <= ny, k <= nz
    Ey (i, j+1/2, k)      i <= nx, j < ny, k <= nz
    Ez (i, j, k+1/2)      i <= nx, j <= ny, k < nz
    Hx (i, j+1/2, k+1/2)  i <= nx, j < ny, k < nz
    Hy (i+1/2, j, k+1/2)  i < nx, j <= ny, k < nz
    Hz (i+1/2, j+1/2, k)  i < nx, j < ny, k <= nz
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

COMPONENTS = ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz")

# Offsets (in cells) of each component's Yee position from its canonical index.
YEE_OFFSET = {
    "Ex": (0.5, 0.0, 0.0), "Ey": (0.0, 0.5, 0.0), "Ez": (0.0, 0.0, 0.5),
    "Hx": (0.0, 0.5, 0.5), "Hy": (0.5, 0.0, 0.5), "Hz": (0.5, 0.5, 0.0),
}

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser (Steele, Lea and Flood, OOPSLA 2014), in place."""
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _stream_key(seed: int, comp: int) -> np.uint64:
    k = np.array([((int(seed) & 0xFFFFFFFFFFFF) << 8) ^ (int(comp) & 0xFF)], dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(k * _GAMMA)[0]


def uniform_pm1(seed: int, comp: int, count: int, start: int = 0) -> np.ndarray:
    """Counter-based uniform[-1, 1) draws, as float32.

    Draw n of stream (seed, comp) is SplitMix64's n-th output from initial
    state key(seed, comp): mix64(key + (n + 1) * gamma).  The top 53 bits give
    u in [0, 1); the value is 2u - 1 in float64, then rounded to float32.
    Draw n only depends on (seed, comp, n), so any slice can be generated alone.
    """
    out = np.empty(count, dtype=np.float32)
    key = _stream_key(seed, comp)
    chunk = 1 << 22
    starts = list(range(0, count, chunk))

    def work(s: int) -> None:
        e = min(count, s + chunk)
        with np.errstate(over="ignore"):
            z = np.arange(start + s + 1, start + e + 1, dtype=np.uint64)
            z *= _GAMMA
            z += key
            _mix64(z)
        z >>= np.uint64(11)
        u = z.astype(np.float64)
        u *= 2.0 ** -52          # (z >> 11) * 2^-53 * 2
        u -= 1.0
        out[s:e] = u.astype(np.float32)

    if len(starts) <= 1:
        for s in starts:
            work(s)
    else:
        nthreads = min(len(starts), max(1, (os.cpu_count() or 1)))
        with ThreadPoolExecutor(nthreads) as ex:
            list(ex.map(work, starts))
    return out


def extent_mask(comp: str, nx: int, ny: int, nz: int) -> np.ndarray:
    """Boolean (nz+1, ny+1, nx+1) mask of the component's Yee extent."""
    m = np.zeros((nz + 1, ny + 1, nx + 1), dtype=bool)
    ox, oy, oz = YEE_OFFSET[comp]
    m[: nz + (0 if oz else 1), : ny + (0 if oy else 1), : nx + (0 if ox else 1)] = True
    return m


def tangential_e_mask(comp: str, nx: int, ny: int, nz: int) -> np.ndarray:
    """Boolean mask of E entries tangential to a PEC face (held at zero)."""
    m = np.zeros((nz + 1, ny + 1, nx + 1), dtype=bool)
    if comp == "Ex":
        m[:, [0, ny], :] = True
        m[[0, nz], :, :] = True
    elif comp == "Ey":
        m[:, :, [0, nx]] = True
        m[[0, nz], :, :] = True
    elif comp == "Ez":
        m[:, :, [0, nx]] = True
        m[:, [0, ny], :] = True
    else:
        raise ValueError(comp)
    return m


def random_fields(seed: int, nx: int, ny: int, nz: int) -> list[np.ndarray]:
    """Six canonical float32 arrays, uniform[-1,1), tangential E and out-of-extent zeroed."""
    n = (nx + 1) * (ny + 1) * (nz + 1)
    out = []
    for c, name in enumerate(COMPONENTS):
        f = uniform_pm1(seed, c, n).reshape(nz + 1, ny + 1, nx + 1)
        f[~extent_mask(name, nx, ny, nz)] = 0.0
        if name[0] == "E":
            f[tangential_e_mask(name, nx, ny, nz)] = 0.0
        out.append(f)
    return out


def sphere_list(seed: int, count: int, box: tuple[int, int, int], rmin: float, rmax: float,
                eps_choices=(2.25, 4.0)) -> list[tuple[float, float, float, float, float]]:
    """Seeded spheres (cx, cy, cz, r, eps_r); centres uniform in the box (cell units)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        cx, cy, cz = (float(rng.uniform(0.0, b)) for b in box)
        r = float(rng.uniform(rmin, rmax))
        eps = float(eps_choices[int(rng.integers(0, len(eps_choices)))])
        out.append((cx, cy, cz, r, eps))
    return out


def eps_r_at(comp: str, spheres, nx: int, ny: int, nz: int) -> np.ndarray:
    """eps_r sampled at the component's Yee positions (canonical layout, float64).

    A point p is inside a sphere when |p - c|^2 <= r^2; overlaps go to the later sphere.
    """
    eps = np.ones((nz + 1, ny + 1, nx + 1), dtype=np.float64)
    ox, oy, oz = YEE_OFFSET[comp]
    for (cx, cy, cz, r, e) in spheres:
        lo = [max(0, int(math.floor(c - o - r))) for c, o in ((cx, ox), (cy, oy), (cz, oz))]
        hi = [min(n, int(math.ceil(c - o + r))) for c, o, n in ((cx, ox, nx), (cy, oy, ny), (cz, oz, nz))]
        if any(h < l for l, h in zip(lo, hi)):
            continue
        xs = np.arange(lo[0], hi[0] + 1) + ox - cx
        ys = np.arange(lo[1], hi[1] + 1) + oy - cy
        zs = np.arange(lo[2], hi[2] + 1) + oz - cz
        d2 = zs[:, None, None] ** 2 + ys[None, :, None] ** 2 + xs[None, None, :] ** 2
        sub = eps[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1]
        sub[d2 <= r * r] = e
    return eps


def sphere_coefficients(spheres, nx: int, ny: int, nz: int, dt: float, dx: float = 1.0):
    """(ce[3], ch) for a dielectric-sphere cavity: ce float32 canonical arrays, ch scalar."""
    ce = [(dt / (eps_r_at(c, spheres, nx, ny, nz) * dx)).astype(np.float32) for c in ("Ex", "Ey", "Ez")]
    return ce, float(np.float32(dt / dx))


COURANT_HALF_DT = 0.5 / math.sqrt(3.0)


def batch_cavities(seed: int, count: int = 256, lo: int = 16, hi: int = 96, p_spheres: float = 0.5):
    """Independent cavities: sides iid uniform-int in [lo, hi]; vacuum or spheres scaled to the size."""
    rng = np.random.default_rng(seed)
    out = []
    for n in range(count):
        nx, ny, nz = (int(v) for v in rng.integers(lo, hi + 1, size=3))
        spheres = None
        if rng.random() < p_spheres:
            m = min(nx, ny, nz)
            ns = int(rng.integers(1, 9))
            spheres = sphere_list(int(rng.integers(0, 2**31)), ns, (nx, ny, nz),
                                  max(2.0, m / 64 * 8), max(2.0, m / 64 * 40) if m >= 8 else 2.0)
        out.append({"nx": nx, "ny": ny, "nz": nz, "spheres": spheres,
                    "field_seed": int(rng.integers(0, 2**31))})
    return out


def serve_stream(seed: int, count: int = 10000, rate_hz: float = 200.0, side_lo: int = 16,
                 side_hi: int = 256, steps_lo: int = 100, steps_hi: int = 2000, p_bf16: float = 0.5):
    """Poisson request stream: exponential inter-arrivals, log-uniform sides, uniform step counts."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for n in range(count):
        t += float(rng.exponential(1.0 / rate_hz))
        sides = np.rint(np.exp(rng.uniform(math.log(side_lo), math.log(side_hi), size=3))).astype(int)
        out.append({"id": n, "arrival_s": t, "nx": int(sides[0]), "ny": int(sides[1]), "nz": int(sides[2]),
                    "steps": int(rng.integers(steps_lo, steps_hi + 1)), "bf16": bool(rng.random() < p_bf16),
                    "field_seed": int(rng.integers(0, 2**31))})
    return out
