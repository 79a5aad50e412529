"""fdtd_energy_static: the energy of caller-owned device fields without any device allocation.

Some callers cannot allocate device memory where they need the energy (work
captured into a CUDA graph, a fixed pre-reserved memory budget, a loop that
cannot take cudaMalloc's implicit synchronisation).  This entry point takes
their device buffers for the inputs and the result and keeps its partial sums
in a fixed array inside the library.  The test checks it against the
allocating entry point, fdtd_energy, on two calls in a row (the second call
reuses the shared array left over from the first), within the 1e-6 relative
energy tolerance the other GPU tests use.  This file is collected last.
"""
import numpy as np
import pytest

import cavity_inputs as ci

pytestmark = pytest.mark.gpu

DT = ci.COURANT_HALF_DT


def _energy_both(dims, seed, spheres):
    import torch
    from paper_2504_09118_gb300 import Cavity, binding
    nx, ny, nz = dims
    f = ci.random_fields(seed, nx, ny, nz)
    ce = ch = None
    if spheres:
        sph = ci.sphere_list(seed + 100, 3, dims, 2.0, 7.0)
        ce, ch = ci.sphere_coefficients(sph, nx, ny, nz, DT)
    with Cavity(nx, ny, nz, DT, 1.0, ce, ch) as cav:
        cav.set_fields(f)
        w_ctx = cav.energy()
    dev = [torch.from_numpy(a).cuda() for a in f]
    dce = None if ce is None else [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in ce]
    dch = None
    if ch is not None:
        dch = [torch.full(dev[0].shape, float(ch), dtype=torch.float32, device="cuda") for _ in range(3)]
    W = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    binding.fdtd_energy_static(nx, ny, nz, DT, 1.0, dev, W, dce, dch)
    torch.cuda.synchronize()
    return float(W.item()), w_ctx


def test_static_energy_matches_allocating_entry_point_twice():
    w1, r1 = _energy_both((37, 21, 30), 5, spheres=True)
    w2, r2 = _energy_both((12, 45, 9), 6, spheres=False)   # second call: smaller, reuses the shared scratch
    assert abs(w1 - r1) <= 1e-6 * abs(r1), (w1, r1)
    assert abs(w2 - r2) <= 1e-6 * abs(r2), (w2, r2)


def test_static_energy_rejects_planes_beyond_its_scratch():
    import torch
    from paper_2504_09118_gb300 import FdtdError, binding
    dev = [torch.zeros(8, dtype=torch.float32, device="cuda") for _ in range(6)]
    W = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(FdtdError) as ei:
        binding.lib().fdtd_energy_static  # loaded
        rc = binding.lib().fdtd_energy_static(1, 1, 9000, DT, 1.0,
                                               binding.ctypes.cast(binding._ptr_array([t.data_ptr() for t in dev]),
                                                                   binding.ctypes.c_void_p),
                                               None, None, W.data_ptr(), None)
        binding._check(None, rc)
    assert ei.value.code == binding.FDTD_ERR_ARG
    assert "8191" in binding.fdtd_last_error(None)
