"""Largest sizes: a cavity whose active arrays exceed 2^31 elements (so every global offset needs 64 bits),
in the two-step kernel's bench configuration.  Fields come from a seeded device generator (52 GB of
canonical FP32); after 4 steps the energy is conserved, tangential E on the faces is exactly zero, and
sub-boxes at both far corners and the centre match the FP64 oracle run on the sub-box alone (a value after
s steps depends only on inputs within s + 1 cells; real faces are exact)."""
import numpy as np
import pytest

import cavity_inputs as ci
from tests.gpu_util import DT, ENERGY_DRIFT_F32, REL_L2_F32

pytestmark = pytest.mark.gpu

DIMS = (1280, 1280, 1312)   # pitch * ny * nz = 2,149,580,800 > 2^31 elements per array
NEED_BYTES = 170e9          # two copies of the fields (103 GB) + canonical fields on the device (52 GB)


def test_active_arrays_beyond_2_31_elements():
    import torch
    import oracle
    from paper_2504_09118_gb300 import Cavity
    nx, ny, nz = DIMS
    free, _ = torch.cuda.mem_get_info()
    if free < NEED_BYTES:
        pytest.skip(f"needs {NEED_BYTES / 1e9:.0f} GB of free device memory, {free / 1e9:.0f} GB free")
    shape = (nz + 1, ny + 1, nx + 1)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(2024)
    f = [torch.rand(shape, generator=gen, device="cuda").mul_(2).sub_(1) for _ in range(6)]
    torch.cuda.empty_cache()
    s, R = 4, 16
    centres = [(0, 0, 0), (nx, ny, nz), (nx // 2, ny // 2, nz // 2), (nx, 0, nz)]
    boxes = []
    for (cx, cy, cz) in centres:
        a = [max(0, cx - R), max(0, cy - R), max(0, cz - R)]
        b = [min(nx, cx + R), min(ny, cy + R), min(nz, cz + R)]
        sub = [x[a[2]:b[2] + 1, a[1]:b[1] + 1, a[0]:b[0] + 1].cpu().numpy().astype(np.float64) for x in f]
        boxes.append((a, b, sub))
    try:
        with Cavity(nx, ny, nz, DT) as cav:
            cav.tune(kernel=3, tile_y=16, stages=4, use_graph=1)
            cav.set_fields(f, on_device=True)
            w0 = cav.energy()
            cav.step(s)
            w1 = cav.energy()
            cav.get_fields(f, on_device=True)   # the canonical tensors now hold the state after s steps
        assert abs(w1 - w0) / w0 <= ENERGY_DRIFT_F32, (w0, w1)
        # tangential E on the far faces (the offsets beyond 2^31) is exactly zero
        assert float(f[0][nz].abs().max()) == 0.0 and float(f[1][nz].abs().max()) == 0.0
        assert float(f[1][:, :, nx].abs().max()) == 0.0 and float(f[2][:, :, nx].abs().max()) == 0.0
        for a, b, sub in boxes:
            oracle.pec_e(sub)
            oracle.step(sub, DT, DT, s)
            m = s + 2
            sl = tuple(slice(m if lo > 0 else 0, (hi - lo + 1) - m if hi < n else hi - lo + 1)
                       for lo, hi, n in ((a[2], b[2], nz), (a[1], b[1], ny), (a[0], b[0], nx)))
            for c, name in enumerate(ci.COMPONENTS):
                got = f[c][a[2]:b[2] + 1, a[1]:b[1] + 1, a[0]:b[0] + 1].cpu().numpy().astype(np.float64)[sl]
                mask = ci.extent_mask(name, b[0] - a[0], b[1] - a[1], b[2] - a[2])[sl]
                ref = sub[c][sl]
                err = np.linalg.norm(got[mask] - ref[mask]) / max(np.linalg.norm(ref[mask]), 1e-30)
                assert err <= REL_L2_F32, (name, a, err)
    finally:
        del f
        torch.cuda.empty_cache()
