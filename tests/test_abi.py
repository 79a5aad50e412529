"""The C-ABI library builds, loads without a GPU, and exports every entry point of include/fdtd.h."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "fdtd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fdtd_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_expected_api():
    names = header_functions()
    for core in ("fdtd_create", "fdtd_set_fields", "fdtd_step", "fdtd_get_fields", "fdtd_energy",
                 "fdtd_divergence", "fdtd_destroy", "fdtd_last_error"):
        assert core in names


def test_library_exports_every_header_symbol():
    from paper_2504_09118_gb300 import binding
    lib = binding.lib()
    names = header_functions()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(binding.EXPORTS) == names
    assert lib.fdtd_version().decode().startswith("fdtd-gb300")


def test_exported_symbols_are_only_the_abi():
    from paper_2504_09118_gb300 import binding
    out = subprocess.run(["nm", "-D", "--defined-only", binding.library_path()], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("nm unavailable")
    fdtd_syms = sorted({l.split()[-1] for l in out.stdout.splitlines() if " T fdtd_" in l})
    assert fdtd_syms == header_functions()


def test_null_arguments_are_rejected_without_gpu():
    from paper_2504_09118_gb300 import binding
    lib = binding.lib()
    assert lib.fdtd_step(None, 1) == binding.FDTD_ERR_ARG
    assert lib.fdtd_steps_done(None) == -1
    assert lib.fdtd_batch_size(None) == -1
    lib.fdtd_destroy(None)
    assert lib.fdtd_create(None, 4, 4, 4, 0.1, 1.0, None, None, 0, None) == binding.FDTD_ERR_ARG


def test_create_rejects_bad_sizes_and_courant_without_gpu():
    from paper_2504_09118_gb300 import binding
    lib = binding.lib()
    out = ctypes.c_void_p()
    assert lib.fdtd_create(ctypes.byref(out), 0, 4, 4, 0.1, 1.0, None, None, 0, None) == binding.FDTD_ERR_ARG
    assert lib.fdtd_create(ctypes.byref(out), 4, 4, 4, -0.1, 1.0, None, None, 0, None) == binding.FDTD_ERR_ARG
    assert lib.fdtd_create(ctypes.byref(out), 4, 4, 4, 0.1, 1.0, None, None, 7, None) == binding.FDTD_ERR_ARG
    # sqrt(3) dt/dx = 1.04 > 1: unstable, rejected on the host before any device call
    assert lib.fdtd_create(ctypes.byref(out), 4, 4, 4, 0.6, 1.0, None, None, 0, None) == binding.FDTD_ERR_UNSTABLE
    assert "Courant" in binding.fdtd_last_error(None)
    assert out.value is None


def test_static_energy_size_guards_without_gpu():
    """fdtd_energy_static checks its sizes (widened to 64 bits before any addition) before touching a GPU:
    nz = INT_MAX, a plane of more than 2^31 points and nz beyond its fixed scratch are FDTD_ERR_ARG."""
    from paper_2504_09118_gb300 import binding
    lib = binding.lib()
    dummy = ctypes.c_float(0.0)
    f = (ctypes.c_void_p * 6)(*([ctypes.addressof(dummy)] * 6))
    w = ctypes.c_double(0.0)
    int_max = 2 ** 31 - 1
    for nx, ny, nz in ((4, 4, int_max), (int_max, 4, 4), (65536, 65536, 4), (4, 4, 8192)):
        rc = lib.fdtd_energy_static(nx, ny, nz, 0.1, 1.0, ctypes.cast(f, ctypes.c_void_p), None, None,
                                    ctypes.cast(ctypes.byref(w), ctypes.c_void_p), None)
        assert rc == binding.FDTD_ERR_ARG, (nx, ny, nz)
    assert "plane" in binding.fdtd_last_error(None)


def test_slab_arguments_are_checked_without_gpu():
    from paper_2504_09118_gb300 import binding
    lib = binding.lib()
    out = ctypes.c_void_p()
    for args in ((0, 0, 4), (5, 3, 2), (1, 10, 2), (0, 2, 3), (0, 10, 0), (0, 10, 65)):   # k0, k1, ghost
        rc = lib.fdtd_create_slab(ctypes.byref(out), 8, 8, 20, *args, 0.1, 1.0, None, None, 0, None)
        assert rc == binding.FDTD_ERR_ARG, args
    assert lib.fdtd_slab_halo_bytes(None) == -1
    assert lib.fdtd_storage_scale_of(ctypes.c_double(1.0)) == 256.0
