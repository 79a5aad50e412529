"""Plant plausible mistakes in the oracle's fourth-order scheme and check that its pins catch each one
(the same procedure as test_oracle_mutants.py: a textually edited copy of the C source, compiled on
the CPU and swapped in for the real library)."""
import ctypes
import shutil

import numpy as np
import pytest

import cavity_inputs as ci
from tests import yee_closed_forms as cf
from tests.test_oracle_mutants import _build_mutant
from tests.yee_matrix import YeeSpace, one_step_matrix

DT = ci.COURANT_HALF_DT

MUTANTS4 = {
    # odd image of tangential E read as even
    "e_image_even": ("        *q = 2 * n - *q;\n        s = -1.0;\n    }\n    return s * AT(a, i, j, k);",
                     "        *q = 2 * n - *q;\n        s = 1.0;\n    }\n    return s * AT(a, i, j, k);"),
    # even image of tangential H mirrored about a node instead of the wall
    "h_image_shift": ("*q = -1 - *q;\n    else if (*q > n - 1)\n        *q = 2 * n - 1 - *q;\n    return AT(a, i, j, k);",
                      "*q = -*q;\n    else if (*q > n - 1)\n        *q = 2 * n - 1 - *q;\n    return AT(a, i, j, k);"),
    "outer_tap_sign": ("const double m3 = tap_e(a, nx, ny, nz, axis, i - di, j - dj, k - dk);\n    return c1 * (p1 - m1) + c2 * (p3 - m3);",
                       "const double m3 = tap_e(a, nx, ny, nz, axis, i - di, j - dj, k - dk);\n    return c1 * (p1 - m1) + c2 * (p3 + m3);"),
    "outer_tap_reach": ("const double p3 = tap_h(a, nx, ny, nz, axis, i + di, j + dj, k + dk);",
                        "const double p3 = tap_h(a, nx, ny, nz, axis, i, j, k);"),
    "wrong_axis": ("double c = d4_h(hy, nx, ny, nz, 0, i, j, k, c1, c2) - d4_h(hx, nx, ny, nz, 1, i, j, k, c1, c2);",
                   "double c = d4_h(hy, nx, ny, nz, 0, i, j, k, c1, c2) - d4_h(hx, nx, ny, nz, 0, i, j, k, c1, c2);"),
    "energy_second_order_term": (
        "double c = d4_e(ez, nx, ny, nz, 1, i, j, k, c1, c2) - d4_e(ey, nx, ny, nz, 2, i, j, k, c1, c2);\n                    double h = AT(hx",
        "double c = d4_e(ez, nx, ny, nz, 1, i, j, k, c1, 0.0) - d4_e(ey, nx, ny, nz, 2, i, j, k, c1, c2);\n                    double h = AT(hx"),
    "div_e_image_odd": ("*q = -1 - *q;\n    else if (*q > n - 1)\n        *q = 2 * n - 1 - *q;\n    return AT(e, i, j, k) / AT(ce, i, j, k);",
                        "*q = -*q;\n    else if (*q > n - 1)\n        *q = 2 * n - 1 - *q;\n    return AT(e, i, j, k) / AT(ce, i, j, k);"),
    "e_update_range": ("    for (k = 0; k < nz; ++k)\n        for (j = 1; j < ny; ++j)\n            for (i = 1; i < nx; ++i) {\n                double c = d4_h(hy",
                       "    for (k = 1; k < nz; ++k)\n        for (j = 1; j < ny; ++j)\n            for (i = 1; i < nx; ++i) {\n                double c = d4_h(hy"),
}


def _pins4_pass(oracle):
    ok = True
    nx, ny, nz = 3, 4, 5
    sp = YeeSpace(nx, ny, nz, order=4)
    rng = np.random.default_rng(4)
    sh = (nz + 1, ny + 1, nx + 1)
    ce = [DT * rng.uniform(0.5, 1.0, sh) for _ in range(3)]
    ch = [DT * rng.uniform(0.5, 1.0, sh) for _ in range(3)]
    M, _, _ = one_step_matrix(sp, ce, ch)
    f = oracle.as_f64(ci.random_fields(5, nx, ny, nz))
    x = np.concatenate([sp.gather(f, sp.h_pts, 3), sp.gather(f, sp.e_pts, 0)])
    oracle.step4(f, ce, ch, 1)
    y = np.concatenate([sp.gather(f, sp.h_pts, 3), sp.gather(f, sp.e_pts, 0)])
    ok &= bool(np.max(np.abs(M @ x - y)) <= 1e-14)
    g, _ = cf.tm110(8, 6, 5, DT, 0, order=4)
    oracle.step4(g, DT, DT, 20)
    h, _ = cf.tm110(8, 6, 5, DT, 20, order=4)
    ok &= all(np.max(np.abs(g[c] - h[c])) <= 1e-12 for c in range(6))
    f = oracle.as_f64(ci.random_fields(6, nx + 2, ny + 1, nz))
    sh = f[0].shape
    ce = [DT * rng.uniform(0.5, 1.0, sh) for _ in range(3)]
    ch = [DT * rng.uniform(0.5, 1.0, sh) for _ in range(3)]
    w0 = oracle.energy4(f, ce, ch, DT)
    d0 = oracle.divergence4(f, ce, ch)
    oracle.step4(f, ce, ch, 20)
    ok &= abs(oracle.energy4(f, ce, ch, DT) - w0) <= 1e-12 * abs(w0)
    d1 = oracle.divergence4(f, ce, ch)
    ok &= all(np.max(np.abs(a - b)) <= 1e-12 for a, b in zip(d0, d1))
    return ok


def test_real_oracle_passes_quick_pins(oracle_mod):
    assert _pins4_pass(oracle_mod)


@pytest.mark.parametrize("name", sorted(MUTANTS4))
def test_mutant_is_caught(oracle_mod, tmp_path, name):
    if shutil.which("gcc") is None:
        pytest.skip("gcc missing")
    so = _build_mutant(tmp_path, name, MUTANTS4)
    real = oracle_mod._lib(False)
    lib = ctypes.CDLL(so)
    for fn in ("oracle_update_h4", "oracle_update_e4", "oracle_pec_e", "oracle_step4", "oracle_energy4",
               "oracle_divergence4"):
        getattr(lib, fn).argtypes = getattr(real, fn).argtypes
        getattr(lib, fn).restype = getattr(real, fn).restype
    saved = oracle_mod._LIBS[False]
    oracle_mod._LIBS[False] = lib
    try:
        assert not _pins4_pass(oracle_mod), f"mutant {name} slipped through the pins"
    finally:
        oracle_mod._LIBS[False] = saved
