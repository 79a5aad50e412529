"""Configurations run by tests/test_gpu_checked.py with the normal and the bounds-checked library.

Run as a script (`python -m tests.checked_runs OUT.npz`) it writes every run's fields; the library is
whichever the FDTD_CHECK environment variable selects.
"""
import sys

import numpy as np

import cavity_inputs as ci

DT = ci.COURANT_HALF_DT
# sizes around the tile edges of the fused kernels (64, 60 and 58 cells in x, 4..16 rows in y)
DIMS = [(1, 3, 2), (7, 9, 11), (61, 13, 5), (64, 8, 3), (65, 17, 9), (121, 40, 7), (130, 67, 12), (2, 70, 5)]
TUNINGS = [dict(kernel=1), dict(kernel=2, tile_y=4), dict(kernel=2, tile_y=16, zchunk=3),
           dict(kernel=3, tile_y=8), dict(kernel=3, tile_y=12, zchunk=2, stages=3), dict(kernel=3, tile_y=16),
           dict(kernel=4, tile_y=12, zchunk=2, stages=3), dict(kernel=4, tile_y=16),
           dict(kernel=5, tile_y=8, zchunk=2, stages=3), dict(kernel=5, tile_y=12)]
TUNINGS4 = [dict(kernel=1), dict(kernel=2, tile_y=4, stages=4), dict(kernel=2, tile_y=8, zchunk=3),
            dict(kernel=2, tile_y=12), dict(kernel=2, tile_y=16, stages=5)]


def run_all() -> dict:
    import torch
    from paper_2504_09118_gb300 import Cavity, binding
    out = {}
    for d_i, dims in enumerate(DIMS):
        sph = ci.sphere_list(d_i, 3, dims, 2.0, max(2.5, min(dims) / 3)) if min(dims) >= 8 else None
        ce, ch = ci.sphere_coefficients(sph, *dims, DT) if sph else (None, None)
        f = ci.random_fields(50 + d_i, *dims)
        for storage in (0, 1):
            for t_i, t in enumerate(TUNINGS):
                with Cavity(*dims, DT, 1.0, ce, ch, storage) as cav:
                    cav.tune(**t)
                    cav.set_fields(f)
                    cav.step(7)
                    for c, a in enumerate(cav.get_fields()):
                        out[f"c{d_i}_s{storage}_t{t_i}_{c}"] = a
    # the fourth-order kernels: every tile height, a short z-chunk, the unfused path
    for d_i, dims in enumerate(DIMS):
        sph = ci.sphere_list(d_i, 3, dims, 2.0, max(2.5, min(dims) / 3)) if min(dims) >= 8 else None
        ce, ch = ci.sphere_coefficients(sph, *dims, DT) if sph else (None, None)
        f = ci.random_fields(70 + d_i, *dims)
        for storage in (0, 2):
            for t_i, t in enumerate(TUNINGS4):
                with Cavity(*dims, DT, 1.0, ce, ch, storage, order=4) as cav:
                    cav.tune(**t)
                    cav.set_fields(f)
                    cav.step(7)
                    for c, a in enumerate(cav.get_fields()):
                        out[f"o4_c{d_i}_s{storage}_t{t_i}_{c}"] = a
    # a batch of members with their own step counts, both kernels
    s = torch.cuda.Stream()
    for kernel in (2, 3, 4):
        cavs = []
        for d_i, dims in enumerate(DIMS):
            c = Cavity(*dims, DT, 1.0, None, None, 0, s)
            c.set_fields(ci.random_fields(90 + d_i, *dims))
            cavs.append(c)
        b = binding.fdtd_batch_create(0, s)
        binding.fdtd_batch_set_tuning(b, kernel=kernel, use_graph=1)
        for n, c in enumerate(cavs):
            binding.fdtd_batch_add(b, c.handle)
            binding.fdtd_batch_set_steps(b, c.handle, 5 + 3 * n)
        binding.fdtd_batch_step(b, 33)
        binding.fdtd_batch_sync(b)
        binding.fdtd_batch_destroy(b)
        for n, c in enumerate(cavs):
            for q, a in enumerate(c.get_fields()):
                out[f"b{kernel}_{n}_{q}"] = a
            c.close()
    return out


if __name__ == "__main__":
    np.savez(sys.argv[1], **run_all())
