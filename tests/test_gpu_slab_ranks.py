"""One slab per process on the GPU: the product's rank path (CtxSlab + DistributedSlab) with real slab
contexts, exchanging ghost cells through gloo point-to-point messages in pinned host buffers.

Two and three processes share the one GPU here; each owns its own slab context and its kernels never wait
on another process (every exchange is a host-side send / receive between steps).  The gathered owned planes
must equal the undivided cavity stepped by the same kernel bit for bit.
"""
import os
import socket

import numpy as np
import pytest

import cavity_inputs as ci

pytestmark = pytest.mark.gpu

DT = ci.COURANT_HALF_DT
DIMS = (40, 30, 27)
STEPS = 13


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _setup():
    sph = ci.sphere_list(31, 3, DIMS, 3.0, 7.0)
    ce, ch = ci.sphere_coefficients(sph, *DIMS, DT)
    return ce, ch, ci.random_fields(32, *DIMS)


def _rank(rank, world, port, out_dir, order, ghost, tuning):
    import torch
    import torch.distributed as dist
    from paper_2504_09118_gb300 import binding as B
    from paper_2504_09118_gb300.slab import CtxSlab, DistributedSlab, local_planes, split_planes
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    h = None
    try:
        nx, ny, nz = DIMS
        ce, ch, f = _setup()
        k0, k1 = split_planes(nz, world)[rank]
        lo, hi, g_lo, g_hi = local_planes(k0, k1, nz, ghost)
        h = B.fdtd_create_slab(nx, ny, nz, k0, k1, ghost, DT, 1.0, [c[lo:hi + 1] for c in ce], ch)
        if order != 2:
            B.fdtd_set_order(h, order)
        B.fdtd_set_tuning(h, **tuning)
        B.fdtd_set_fields(h, [np.ascontiguousarray(a[lo:hi + 1]) for a in f], dims=(nx, ny, hi - lo))
        DistributedSlab(CtxSlab(h, order, host=True), rank, world).step(STEPS)
        loc = [np.empty((hi - lo + 1, ny + 1, nx + 1), np.float32) for _ in range(6)]
        B.fdtd_get_fields(h, loc, dims=(nx, ny, hi - lo))
        np.save(os.path.join(out_dir, f"own{rank}.npy"), np.stack([a[g_lo:g_lo + (k1 - k0)] for a in loc]))
        if k1 == nz:
            np.save(os.path.join(out_dir, "top.npy"), np.stack([a[hi - lo] for a in loc]))
        dist.barrier()
    finally:
        if h is not None:
            B.fdtd_destroy(h)
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("order,ghost,tuning", [(2, 2, {"kernel": 3, "tile_y": 16}), (4, 3, {"kernel": 2})])
def test_slab_per_process_equals_one_cavity(tmp_path, world, order, ghost, tuning):
    import torch.multiprocessing as mp
    from paper_2504_09118_gb300 import Cavity
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path), order, ghost, tuning), nprocs=world, join=True)
    nx, ny, nz = DIMS
    got = np.concatenate([np.load(tmp_path / f"own{r}.npy") for r in range(world)] +
                         [np.load(tmp_path / "top.npy")[:, None]], axis=1)
    ce, ch, f = _setup()
    with Cavity(*DIMS, DT, 1.0, ce, ch, 0, order=order) as cav:
        cav.tune(**tuning)
        cav.set_fields(f)
        cav.step(STEPS)
        ref = np.stack(cav.get_fields())
    assert got.shape == ref.shape
    for c, name in enumerate(ci.COMPONENTS):
        assert np.array_equal(got[c], ref[c]), name
