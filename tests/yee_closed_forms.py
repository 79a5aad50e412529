"""Closed-form discrete cavity eigenmodes of the Yee scheme (used to pin the oracle and the GPU path).

Derived by substituting separable standing waves into the update equations of
Eq. 2 (vacuum, scalar ce = ch = dt/dx, PEC walls):

TM110 (Ez, Hx, Hy):  with s_x = sin(pi/(2 nx)), s_y = sin(pi/(2 ny)) and
    sin^2(w dt / 2) = ce ch (s_x^2 + s_y^2)
  Ez^n      = cos(w n dt) sin(pi i/nx) sin(pi j/ny)
  Hx^{n+1/2} = a_x sin(w (n+1/2) dt) sin(pi i/nx) cos(pi (j+1/2)/ny),  a_x = -ch s_y / sin(w dt/2)
  Hy^{n+1/2} = a_y sin(w (n+1/2) dt) cos(pi (i+1/2)/nx) sin(pi j/ny),  a_y = +ch s_x / sin(w dt/2)

TE101 (Ey, Hx, Hz):  sin^2(w dt/2) = ce ch (s_x^2 + s_z^2)
  Ey^n       = cos(w n dt) sin(pi i/nx) sin(pi k/nz)
  Hx^{n+1/2} = b_x sin(w (n+1/2) dt) sin(pi i/nx) cos(pi (k+1/2)/nz),  b_x = +ch s_z / sin(w dt/2)
  Hz^{n+1/2} = b_z sin(w (n+1/2) dt) cos(pi (i+1/2)/nx) sin(pi k/nz),  b_z = -ch s_x / sin(w dt/2)

The general dispersion relation for mode (m, n, p) is
  sin^2(w dt/2) = ce ch (sin^2(pi m/(2nx)) + sin^2(pi n/(2ny)) + sin^2(pi p/(2nz))).

With the fourth-order differences (order=4) the same standing waves are exact
eigenmodes (the image-closed walls keep sine and cosine profiles intact); every
sin(pi m/(2n)) above becomes c1 sin(pi m/(2n)) + c2 sin(3 pi m/(2n)).
"""
from __future__ import annotations

import math

import numpy as np

import cavity_inputs as ci
from tests.yee_matrix import sigma


def omega(ce: float, ch: float, dt: float, sx2: float, sy2: float, sz2: float = 0.0) -> float:
    s = math.sqrt(ce * ch * (sx2 + sy2 + sz2))
    return 2.0 * math.asin(s) / dt


def _grids(nx, ny, nz):
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    return i.astype(np.float64), j.astype(np.float64), k.astype(np.float64)


def _clean(fields, nx, ny, nz):
    for c, name in enumerate(ci.COMPONENTS):
        fields[c][~ci.extent_mask(name, nx, ny, nz)] = 0.0
        if name[0] == "E":
            fields[c][ci.tangential_e_mask(name, nx, ny, nz)] = 0.0
    return fields


def tm110(nx, ny, nz, dt, n, ce=None, ch=None, order=2):
    """State (H^{n-1/2}, E^n) of the TM110 mode, float64 canonical arrays."""
    ce = dt if ce is None else ce
    ch = dt if ch is None else ch
    sx, sy = float(sigma(1, nx, order)), float(sigma(1, ny, order))
    w = omega(ce, ch, dt, sx * sx, sy * sy)
    sig = math.sin(w * dt / 2)
    ax, ay = -ch * sy / sig, ch * sx / sig
    i, j, k = _grids(nx, ny, nz)
    f = [np.zeros_like(i) for _ in range(6)]
    f[2] = math.cos(w * n * dt) * np.sin(math.pi * i / nx) * np.sin(math.pi * j / ny)
    th = math.sin(w * (n - 0.5) * dt)
    f[3] = ax * th * np.sin(math.pi * i / nx) * np.cos(math.pi * (j + 0.5) / ny)
    f[4] = ay * th * np.cos(math.pi * (i + 0.5) / nx) * np.sin(math.pi * j / ny)
    return _clean(f, nx, ny, nz), w


def te101(nx, ny, nz, dt, n, ce=None, ch=None, order=2):
    """State (H^{n-1/2}, E^n) of the TE101 mode, float64 canonical arrays."""
    ce = dt if ce is None else ce
    ch = dt if ch is None else ch
    sx, sz = float(sigma(1, nx, order)), float(sigma(1, nz, order))
    w = omega(ce, ch, dt, sx * sx, 0.0, sz * sz)
    sig = math.sin(w * dt / 2)
    bx, bz = ch * sz / sig, -ch * sx / sig
    i, j, k = _grids(nx, ny, nz)
    f = [np.zeros_like(i) for _ in range(6)]
    f[1] = math.cos(w * n * dt) * np.sin(math.pi * i / nx) * np.sin(math.pi * k / nz)
    th = math.sin(w * (n - 0.5) * dt)
    f[3] = bx * th * np.sin(math.pi * i / nx) * np.cos(math.pi * (k + 0.5) / nz)
    f[5] = bz * th * np.cos(math.pi * (i + 0.5) / nx) * np.sin(math.pi * k / nz)
    return _clean(f, nx, ny, nz), w
