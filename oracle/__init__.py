"""FP64 CPU oracle for the Yee FDTD step (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline legs may import
this package.  The CUDA library never links or calls it.

The C source (yee_oracle.c) is compiled twice with gcc: a serial build and an
OpenMP build whose only difference is the "omp parallel for" on outer loops of
the field updates (bit-identical results).  Both use -ffp-contract=off so no
fused multiply-add changes rounding between x86 and Arm hosts.

Python API (arrays are canonical (nz+1, ny+1, nx+1) float64, x fastest):
    step(fields, ce, ch, nsteps, omp=False)       in place, Listing 1 order
    update_h(fields, ch) / update_e(fields, ce) / pec_e(fields)
    energy(fields, ce, ch, dt_over_dx) -> float
    divergence(fields, ce, ch) -> (divE nodes, divH cells)
    step4 / update_h4 / update_e4 / energy4 / divergence4: the same with the fourth-order
        differences c1 [f(p+1/2) - f(p-1/2)] + c2 [f(p+3/2) - f(p-3/2)] (default c1 = 9/8,
        c2 = -1/24) and image-closed PEC walls
ce / ch may be a scalar or a list of three scalars/arrays; they are broadcast
to full canonical arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "yee_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIBS: dict[bool, ctypes.CDLL] = {}
_LOCK = threading.Lock()


def _lib_path(omp: bool) -> str:
    return os.path.join(_BUILD, "liboracle_omp.so" if omp else "liboracle.so")


def build(force: bool = False) -> None:
    """Compile the serial and OpenMP oracle libraries with gcc (skipped when up to date)."""
    os.makedirs(_BUILD, exist_ok=True)
    for omp in (False, True):
        out = _lib_path(omp)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-ffp-contract=off", "-fno-fast-math"]
        if omp:
            cmd.append("-fopenmp")
        tmp = out + f".tmp{os.getpid()}"
        subprocess.run(cmd + ["-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, out)


def _lib(omp: bool = False) -> ctypes.CDLL:
    with _LOCK:
        if omp not in _LIBS:
            build()
            lib = ctypes.CDLL(_lib_path(omp))
            P = ctypes.POINTER(ctypes.c_double)
            PP = ctypes.POINTER(P)
            i = ctypes.c_int
            lib.oracle_update_h.argtypes = [i, i, i] + [P] * 9
            lib.oracle_update_e.argtypes = [i, i, i] + [P] * 9
            lib.oracle_pec_e.argtypes = [i, i, i, P, P, P]
            lib.oracle_step.argtypes = [i, i, i, PP, PP, PP, i]
            PI = ctypes.POINTER(ctypes.c_int)
            lib.oracle_step_sources.argtypes = [i, i, i, PP, PP, PP, i, i, i, PI, PI, PI, PI, P, i,
                                                ctypes.c_double]
            lib.oracle_energy.argtypes = [i, i, i, PP, PP, PP, ctypes.c_double]
            lib.oracle_energy.restype = ctypes.c_double
            lib.oracle_divergence.argtypes = [i, i, i, PP, PP, PP, P, P]
            lib.oracle_threads.restype = ctypes.c_int
            d = ctypes.c_double
            lib.oracle_update_h4.argtypes = [i, i, i] + [P] * 9 + [d, d]
            lib.oracle_update_e4.argtypes = [i, i, i] + [P] * 9 + [d, d]
            lib.oracle_step4.argtypes = [i, i, i, PP, PP, PP, i, d, d, i, i, PI, PI, PI, PI, P, i, d]
            lib.oracle_energy4.argtypes = [i, i, i, PP, PP, PP, d, d, d]
            lib.oracle_energy4.restype = ctypes.c_double
            lib.oracle_divergence4.argtypes = [i, i, i, PP, PP, PP, P, P, d, d]
            _LIBS[omp] = lib
        return _LIBS[omp]


def _dims(fields):
    nz1, ny1, nx1 = fields[0].shape
    return nx1 - 1, ny1 - 1, nz1 - 1


def _ptr(a: np.ndarray):
    if a.dtype != np.float64 or not a.flags.c_contiguous:
        raise TypeError("oracle arrays must be C-contiguous float64")
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _pp(arrs):
    P = ctypes.POINTER(ctypes.c_double)
    return (P * len(arrs))(*[_ptr(a) for a in arrs])


def full_coef(c, shape) -> list[np.ndarray]:
    """Broadcast a scalar, or three scalars/arrays, to three canonical float64 arrays."""
    if np.isscalar(c):
        c = [c, c, c]
    return [np.ascontiguousarray(np.broadcast_to(np.asarray(v, dtype=np.float64), shape)) for v in c]


def threads(omp: bool = True) -> int:
    return int(_lib(omp).oracle_threads())


def update_h(f, ch):
    nx, ny, nz = _dims(f)
    ch = full_coef(ch, f[0].shape)
    _lib().oracle_update_h(nx, ny, nz, *[_ptr(a) for a in (f[3], f[4], f[5], f[0], f[1], f[2])], *[_ptr(a) for a in ch])


def update_e(f, ce):
    nx, ny, nz = _dims(f)
    ce = full_coef(ce, f[0].shape)
    _lib().oracle_update_e(nx, ny, nz, *[_ptr(a) for a in (f[0], f[1], f[2], f[3], f[4], f[5])], *[_ptr(a) for a in ce])


def pec_e(f):
    nx, ny, nz = _dims(f)
    _lib().oracle_pec_e(nx, ny, nz, _ptr(f[0]), _ptr(f[1]), _ptr(f[2]))


def step(f, ce, ch, nsteps: int, omp: bool = False):
    """Advance the six float64 canonical arrays in place by nsteps leapfrog steps."""
    nx, ny, nz = _dims(f)
    ce = full_coef(ce, f[0].shape)
    ch = full_coef(ch, f[0].shape)
    _lib(omp).oracle_step(nx, ny, nz, _pp(f), _pp(ce), _pp(ch), int(nsteps))
    return f


def step_sources(f, ce, ch, nsteps: int, sources, wave, n0: int = 0, dx: float = 1.0, omp: bool = False):
    """oracle.step with point currents: sources = [(comp, i, j, k), ...] (comp 0..2 = Ex, Ey, Ez),
    wave = array (nsrc, wave_len) of J^{n+1/2} for steps n0, n0 + 1, ... (Eq. 1 with J != 0)."""
    nx, ny, nz = _dims(f)
    ce = full_coef(ce, f[0].shape)
    ch = full_coef(ch, f[0].shape)
    src = np.asarray(sources, dtype=np.int32).reshape(-1, 4)
    w = np.ascontiguousarray(np.asarray(wave, dtype=np.float64).reshape(len(src), -1))
    cols = [np.ascontiguousarray(src[:, q]) for q in range(4)]
    PI = ctypes.POINTER(ctypes.c_int)
    _lib(omp).oracle_step_sources(nx, ny, nz, _pp(f), _pp(ce), _pp(ch), int(nsteps), int(n0), len(src),
                                  *[c.ctypes.data_as(PI) for c in cols], _ptr(w), w.shape[1], float(dx))
    return f


# Coefficients of the staggered fourth-order difference (exact for cubics)
C1_4 = 9.0 / 8.0
C2_4 = -1.0 / 24.0


def update_h4(f, ch, c1=C1_4, c2=C2_4):
    nx, ny, nz = _dims(f)
    ch = full_coef(ch, f[0].shape)
    _lib().oracle_update_h4(nx, ny, nz, *[_ptr(a) for a in (f[3], f[4], f[5], f[0], f[1], f[2])],
                            *[_ptr(a) for a in ch], float(c1), float(c2))


def update_e4(f, ce, c1=C1_4, c2=C2_4):
    nx, ny, nz = _dims(f)
    ce = full_coef(ce, f[0].shape)
    _lib().oracle_update_e4(nx, ny, nz, *[_ptr(a) for a in (f[0], f[1], f[2], f[3], f[4], f[5])],
                            *[_ptr(a) for a in ce], float(c1), float(c2))


def step4(f, ce, ch, nsteps: int, c1=C1_4, c2=C2_4, sources=(), wave=None, n0: int = 0, dx: float = 1.0,
          omp: bool = False):
    """Fourth-order (2,4) steps in place; optional point currents as in step_sources."""
    nx, ny, nz = _dims(f)
    ce = full_coef(ce, f[0].shape)
    ch = full_coef(ch, f[0].shape)
    src = np.asarray(sources, dtype=np.int32).reshape(-1, 4)
    w = np.zeros((max(len(src), 1), 1)) if wave is None else np.asarray(wave, dtype=np.float64)
    w = np.ascontiguousarray(w.reshape(max(len(src), 1), -1))
    cols = [np.ascontiguousarray(src[:, q]) for q in range(4)]
    PI = ctypes.POINTER(ctypes.c_int)
    _lib(omp).oracle_step4(nx, ny, nz, _pp(f), _pp(ce), _pp(ch), int(nsteps), float(c1), float(c2), int(n0),
                           len(src), *[c.ctypes.data_as(PI) for c in cols], _ptr(w), w.shape[1], float(dx))
    return f


def energy4(f, ce, ch, dt_over_dx: float, c1=C1_4, c2=C2_4) -> float:
    nx, ny, nz = _dims(f)
    ce = full_coef(ce, f[0].shape)
    ch = full_coef(ch, f[0].shape)
    return float(_lib().oracle_energy4(nx, ny, nz, _pp(f), _pp(ce), _pp(ch), float(dt_over_dx), float(c1),
                                       float(c2)))


def divergence4(f, ce, ch, c1=C1_4, c2=C2_4):
    """Fourth-order (divE at nodes, canonical shape; divH at cells, shape (nz, ny, nx))."""
    nx, ny, nz = _dims(f)
    de = np.zeros(f[0].shape, dtype=np.float64)
    dh = np.zeros((nz, ny, nx), dtype=np.float64)
    ce = full_coef(ce, f[0].shape)
    ch = full_coef(ch, f[0].shape)
    _lib().oracle_divergence4(nx, ny, nz, _pp(f), _pp(ce), _pp(ch), _ptr(de), _ptr(dh), float(c1), float(c2))
    return de, dh


def energy(f, ce, ch, dt_over_dx: float) -> float:
    nx, ny, nz = _dims(f)
    ce = full_coef(ce, f[0].shape)   # keep the arrays alive across the call
    ch = full_coef(ch, f[0].shape)
    return float(_lib().oracle_energy(nx, ny, nz, _pp(f), _pp(ce), _pp(ch), float(dt_over_dx)))


def divergence(f, ce, ch):
    """(divE at nodes, canonical shape; divH at cells, shape (nz, ny, nx))."""
    nx, ny, nz = _dims(f)
    de = np.zeros(f[0].shape, dtype=np.float64)
    dh = np.zeros((nz, ny, nx), dtype=np.float64)
    ce = full_coef(ce, f[0].shape)
    ch = full_coef(ch, f[0].shape)
    _lib().oracle_divergence(nx, ny, nz, _pp(f), _pp(ce), _pp(ch), _ptr(de), _ptr(dh))
    return de, dh


def as_f64(fields) -> list[np.ndarray]:
    return [np.ascontiguousarray(np.asarray(a, dtype=np.float64)) for a in fields]
