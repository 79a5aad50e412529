"""Plant plausible mistakes in a copy of the oracle and check that the pins catch each one.

Each mutant is compiled from a textually edited copy of oracle/yee_oracle.c in a
temporary directory (CPU only), swapped in for the real library, and run
through the brute-force and closed-form checks.  A pin set that let any of
these through would not be strong enough to trust the oracle.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import cavity_inputs as ci
from tests import yee_closed_forms as cf
from tests.yee_matrix import YeeSpace, one_step_matrix

DT = ci.COURANT_HALF_DT

MUTANTS = {
    "h_sign_flip": ("AT(ez, i, j, k));\n                AT(hy, i, j, k) -= AT(chy, i, j, k) * c;",
                    "AT(ez, i, j, k));\n                AT(hy, i, j, k) += AT(chy, i, j, k) * c;"),
    "energy_wrong_index": ("- (AT(ex, i, j + 1, k) - AT(ex, i, j, k));\n                    double h = AT(hz",
                           "- (AT(ex, i + 1, j, k) - AT(ex, i, j, k));\n                    double h = AT(hz"),
    "wrong_index": ("- (AT(ex, i, j + 1, k) - AT(ex, i, j, k));\n                AT(hz",
                    "- (AT(ex, i + 1, j, k) - AT(ex, i, j, k));\n                AT(hz"),
    "div_wrong_coef": ("+ AT(ey, i, j, k) / AT(ce[1], i, j, k) - AT(ey, i, j - 1, k) / AT(ce[1], i, j - 1, k)",
                       "+ AT(ey, i, j, k) / AT(ce[1], i, j, k) - AT(ey, i, j - 1, k) / AT(ce[1], i, j, k)"),
    "dropped_term": ("double c = (AT(hy, i, j, k) - AT(hy, i - 1, j, k)) - (AT(hx, i, j, k) - AT(hx, i, j - 1, k));",
                     "double c = (AT(hy, i, j, k) - AT(hy, i - 1, j, k));"),
    "swapped_coef": ("AT(hy, i, j, k - 1));\n                AT(ex, i, j, k) += AT(cex, i, j, k) * c;",
                     "AT(hy, i, j, k - 1));\n                AT(ex, i, j, k) += AT(cey, i, j, k) * c;"),
    "transposed_stencil": ("- (AT(hz, i, j, k) - AT(hz, i - 1, j, k));", "- (AT(hz, i, j, k) - AT(hz, i, j - 1, k));"),
    # (skipping Hz's k = 0 plane would be an equivalent mutant: curl E vanishes on that face)
    "skipped_plane": ("for (k = 1; k < nz; ++k)\n        for (j = 1; j < ny; ++j)\n            for (i = 0; i < nx; ++i) {\n                /* (curl H)_x",
                      "for (k = 2; k < nz; ++k)\n        for (j = 1; j < ny; ++j)\n            for (i = 0; i < nx; ++i) {\n                /* (curl H)_x"),
    "wrong_sign_in_curl": ("double c = (AT(ex, i, j, k + 1) - AT(ex, i, j, k)) - (AT(ez, i + 1, j, k) - AT(ez, i, j, k));\n                AT(hy",
                           "double c = (AT(ex, i, j, k + 1) - AT(ex, i, j, k)) + (AT(ez, i + 1, j, k) - AT(ez, i, j, k));\n                AT(hy"),
}


def _build_mutant(tmp_path, name, table=MUTANTS):
    import oracle
    src = open(os.path.join(os.path.dirname(oracle.__file__), "yee_oracle.c")).read()
    old, new = table[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not unique/not found"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-ffp-contract=off", "-o", str(so), str(path), "-lm"],
                   check=True)
    return str(so)


def _pins_pass(oracle):
    """True when every quick pin passes."""
    ok = True
    # brute force on 3x4x5 with per-position coefficients
    nx, ny, nz = 3, 4, 5
    sp = YeeSpace(nx, ny, nz)
    rng = np.random.default_rng(1)
    sh = (nz + 1, ny + 1, nx + 1)
    ce = [DT * rng.uniform(0.5, 1.0, sh) for _ in range(3)]
    ch = [DT * rng.uniform(0.5, 1.0, sh) for _ in range(3)]
    M, _, _ = one_step_matrix(sp, ce, ch)
    f = oracle.as_f64(ci.random_fields(2, nx, ny, nz))
    x = np.concatenate([sp.gather(f, sp.h_pts, 3), sp.gather(f, sp.e_pts, 0)])
    oracle.step(f, ce, ch, 1)
    y = np.concatenate([sp.gather(f, sp.h_pts, 3), sp.gather(f, sp.e_pts, 0)])
    ok &= bool(np.max(np.abs(M @ x - y)) <= 1e-14)
    # closed-form TM110 and energy
    g, _ = cf.tm110(8, 6, 5, DT, 0)
    oracle.step(g, DT, DT, 20)
    h, _ = cf.tm110(8, 6, 5, DT, 20)
    ok &= all(np.max(np.abs(g[c] - h[c])) <= 1e-12 for c in range(6))
    # energy conservation and divergence invariance with per-position coefficients
    f = oracle.as_f64(ci.random_fields(3, nx + 2, ny + 1, nz))
    sh = f[0].shape
    ce = [DT * rng.uniform(0.5, 1.0, sh) for _ in range(3)]
    ch = [DT * rng.uniform(0.5, 1.0, sh) for _ in range(3)]
    w0 = oracle.energy(f, ce, ch, DT)
    d0 = oracle.divergence(f, ce, ch)
    oracle.step(f, ce, ch, 20)
    ok &= abs(oracle.energy(f, ce, ch, DT) - w0) <= 1e-12 * abs(w0)
    d1 = oracle.divergence(f, ce, ch)
    ok &= all(np.max(np.abs(a - b)) <= 1e-12 for a, b in zip(d0, d1))
    return ok


def test_real_oracle_passes_quick_pins(oracle_mod):
    assert _pins_pass(oracle_mod)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(oracle_mod, tmp_path, name):
    if shutil.which("gcc") is None:
        pytest.skip("gcc missing")
    so = _build_mutant(tmp_path, name)
    real = oracle_mod._lib(False)
    lib = ctypes.CDLL(so)
    for fn in ("oracle_update_h", "oracle_update_e", "oracle_pec_e", "oracle_step", "oracle_energy",
               "oracle_divergence"):
        getattr(lib, fn).argtypes = getattr(real, fn).argtypes
        getattr(lib, fn).restype = getattr(real, fn).restype
    saved = oracle_mod._LIBS[False]
    oracle_mod._LIBS[False] = lib
    try:
        assert not _pins_pass(oracle_mod), f"mutant {name} slipped through the pins"
    finally:
        oracle_mod._LIBS[False] = saved
