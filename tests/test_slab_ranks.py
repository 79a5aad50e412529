"""The z-slab schedule of paper_2504_09118_gb300.slab on CPU ranks (gloo, 127.0.0.1).

DistributedSlab (the product's orchestration: exchange the ghost cells with the neighbouring ranks, then
step at most ghost // reach steps) drives a test slab whose steps are the FP64 oracle's on the slab's own
planes.  The oracle treats each local boundary as a PEC wall, exactly as the GPU kernels treat a slab's,
so the gathered owned planes must equal one undivided oracle run bit for bit: for Eq. 2 with one and two
ghost cells, for the fourth-order differences with three and six, for two and three ranks (a middle rank
exchanges on both sides).  Skipping one exchange must change the result.
"""
import os
import socket

import numpy as np
import pytest

import cavity_inputs as ci

DT = ci.COURANT_HALF_DT


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _entry(rank, world, port, out_dir, case):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        _run_slab(rank, world, out_dir, **case)
    finally:
        dist.destroy_process_group()


class OracleSlab:
    """A slab in the shape DistributedSlab drives, stepped by the FP64 oracle on its local planes."""

    def __init__(self, fields, ce, ch, nz, k0, k1, ghost, order):
        import torch
        from paper_2504_09118_gb300 import slab
        lo, hi, g_lo, g_hi = slab.local_planes(k0, k1, nz, ghost)
        self.lo, self.hi, self.g_lo, self.g_hi, self.ghost = lo, hi, g_lo, g_hi, ghost
        self.loc = [np.ascontiguousarray(a[lo:hi + 1], dtype=np.float64) for a in fields]
        self.ce = [np.ascontiguousarray(c[lo:hi + 1], dtype=np.float64) for c in ce]
        self.ch = ch
        self.order = order
        self.has_lower, self.has_upper = g_lo > 0, g_hi > 0
        self.per_exchange = ghost // slab.reach(order)
        self.shape = (6, ghost) + self.loc[0].shape[1:]
        self.recv = [torch.zeros(self.shape, dtype=torch.float64) for _ in range(2)]
        self.intervals = 0   # step calls so far: the exchange before interval i is exchange i
        self.skip = -1       # test hook: drop the imports of this exchange

    def _planes(self, side, own):
        nzl = self.hi - self.lo
        if own:
            p0 = self.g_lo if side == 0 else nzl - self.g_hi - self.ghost
        else:
            p0 = 0 if side == 0 else nzl - self.g_hi
        return p0

    def export(self, side):
        import torch
        p0 = self._planes(side, True)
        return torch.from_numpy(np.ascontiguousarray(np.stack([a[p0:p0 + self.ghost] for a in self.loc])))

    def recv_buffer(self, side):
        return self.recv[side]

    def import_(self, side, buf):
        if self.intervals == self.skip:
            return
        p0 = self._planes(side, False)
        b = buf.numpy()
        for c in range(6):
            self.loc[c][p0:p0 + self.ghost] = b[c]

    def step(self, n):
        import oracle
        self.intervals += 1
        if self.order == 4:
            oracle.step4(self.loc, self.ce, self.ch, n)
        else:
            oracle.step(self.loc, self.ce, self.ch, n)


def _run_slab(rank, world, out_dir, dims, steps, ghost, order, skip=-1):
    import torch.distributed as dist
    from paper_2504_09118_gb300.slab import DistributedSlab, split_planes
    nx, ny, nz = dims
    sph = ci.sphere_list(3, 3, dims, 2.0, 5.0)
    ce, ch = ci.sphere_coefficients(sph, nx, ny, nz, DT)
    f = ci.random_fields(7, nx, ny, nz)
    k0, k1 = split_planes(nz, world)[rank]
    s = OracleSlab(f, ce, ch, nz, k0, k1, ghost, order)
    s.skip = skip
    d = DistributedSlab(s, rank, world)
    d.step(steps)
    own = np.stack([a[s.g_lo:s.g_lo + (k1 - k0)] for a in s.loc])
    np.save(os.path.join(out_dir, f"own{rank}.npy"), own)
    if k1 == nz:
        np.save(os.path.join(out_dir, "top.npy"), np.stack([a[-1] for a in s.loc]))
    dist.barrier()


def _gathered(tmp_path, world, dims):
    nx, ny, nz = dims
    parts = [np.load(tmp_path / f"own{r}.npy") for r in range(world)]
    full = np.concatenate(parts + [np.load(tmp_path / "top.npy")[:, None]], axis=1)
    assert full.shape == (6, nz + 1, ny + 1, nx + 1)
    return full


def _reference(dims, steps, order):
    import oracle
    nx, ny, nz = dims
    sph = ci.sphere_list(3, 3, dims, 2.0, 5.0)
    ce, ch = ci.sphere_coefficients(sph, nx, ny, nz, DT)
    ref = oracle.as_f64(ci.random_fields(7, nx, ny, nz))
    ce64 = [c.astype(np.float64) for c in ce]
    (oracle.step4 if order == 4 else oracle.step)(ref, ce64, ch, steps)
    return np.stack(ref)


def _spawn(world, tmp_path, case):
    import torch.multiprocessing as mp
    mp.spawn(_entry, args=(world, _free_port(), str(tmp_path), case), nprocs=world, join=True)


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("order,ghost", [(2, 1), (2, 2), (4, 3), (4, 6)])
def test_distributed_slabs_equal_one_domain(tmp_path, world, order, ghost):
    dims = (9, 8, 21)
    steps = 7
    _spawn(world, tmp_path, dict(dims=dims, steps=steps, ghost=ghost, order=order))
    got = _gathered(tmp_path, world, dims)
    ref = _reference(dims, steps, order)
    assert np.array_equal(got, ref)


def test_a_skipped_exchange_shows(tmp_path):
    dims = (9, 8, 21)
    _spawn(2, tmp_path, dict(dims=dims, steps=7, ghost=1, order=2, skip=3))
    got = _gathered(tmp_path, 2, dims)
    assert not np.array_equal(got, _reference(dims, 7, 2))
