"""z-slab decomposition of one cavity (host orchestration over the C ABI's slab calls).

A slab owns the cells of global planes [k0, k1) and keeps `ghost` cells of each neighbour; after the
ghost cells are refreshed, its owned cells stay exact for ghost // reach steps (reach: 1 plane per step
for Eq. 2, 3 for the fourth-order differences).  A run therefore alternates "exchange the ghost cells"
and "step every slab by at most ghost // reach".  With ghost = 2 and the two-step kernel that is one
launch per exchange, each exchange carrying two planes of the six fields per side.

* SlabDomain: every slab of one cavity in this process (one GPU; the exchange is a device-to-device
  copy between neighbouring slab contexts).
* DistributedSlab: one slab per rank of a torch.distributed group (NCCL between GPUs, gloo on CPUs);
  the exchange is export -> send / receive with the two neighbours -> import.  The slab it drives only
  needs export / import / step and the ghost geometry, so the schedule runs the same with any slab
  object of that shape.

Canonical arrays of a slab cover its local planes, global planes k0 - g_lo .. k1 + g_hi (g_lo = ghost
when k0 > 0, g_hi = ghost when k1 < nz); the global canonical index k along z is the cell index of every
component, so slab s contributes planes [k0, k1) to the gathered state (and the top slab also plane nz).
"""
from __future__ import annotations

import numpy as np

from . import binding as B


def split_planes(nz: int, nslabs: int) -> list[tuple[int, int]]:
    """nslabs contiguous plane ranges covering [0, nz), sizes differing by at most one."""
    if nslabs < 1 or nslabs > nz:
        raise ValueError("need 1 <= nslabs <= nz")
    out, k = [], 0
    for s in range(nslabs):
        n = nz // nslabs + (1 if s < nz % nslabs else 0)
        out.append((k, k + n))
        k += n
    return out


def local_planes(k0: int, k1: int, nz: int, ghost: int) -> tuple[int, int, int, int]:
    """(first global plane, last global plane, g_lo, g_hi) of a slab's local canonical arrays."""
    g_lo = ghost if k0 > 0 else 0
    g_hi = ghost if k1 < nz else 0
    return k0 - g_lo, k1 + g_hi, g_lo, g_hi


def reach(order: int) -> int:
    """Planes by which one leapfrog step's dependence spreads along z."""
    return 3 if order == 4 else 1


def _slice(arrs, lo: int, hi: int):
    return [np.ascontiguousarray(a[lo:hi + 1]) for a in arrs] if arrs is not None else None


def _slice_coef(c, lo, hi):
    if c is None or np.isscalar(c):
        return c
    return _slice(c, lo, hi)


class SlabDomain:
    """All z-slabs of one nx*ny*nz cavity in this process, stepped in lockstep with device-to-device
    ghost exchanges (fdtd_slab_exchange) between neighbours."""

    def __init__(self, nx, ny, nz, dt, dx=1.0, ce=None, ch=None, storage=B.FDTD_F32, nslabs=2, ghost=2,
                 order=2, tuning=None, streams=None):
        self.dims = (int(nx), int(ny), int(nz))
        self.ghost, self.order, self.storage = int(ghost), int(order), int(storage)
        self.ranges = split_planes(nz, nslabs)
        self.per_exchange = self.ghost // reach(order)
        if self.per_exchange < 1:
            raise ValueError(f"ghost {ghost} is below the reach {reach(order)} of one step")
        self.handles, self.locals = [], []
        try:
            for s, (k0, k1) in enumerate(self.ranges):
                lo, hi, g_lo, g_hi = local_planes(k0, k1, nz, ghost)
                stream = streams[s] if streams is not None else None
                h = B.fdtd_create_slab(nx, ny, nz, k0, k1, ghost, dt, dx, _slice_coef(ce, lo, hi),
                                       _slice_coef(ch, lo, hi), storage, stream)
                self.handles.append(h)
                self.locals.append((lo, hi, g_lo, g_hi))
                if order != 2:
                    B.fdtd_set_order(h, order)
                if tuning:
                    B.fdtd_set_tuning(h, **tuning)
        except Exception:
            self.close()
            raise
        self.fresh = False   # ghost cells current (no step since the last exchange)

    def close(self):
        for h in self.handles:
            B.fdtd_destroy(h)
        self.handles = []

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_fields(self, fields):
        """Load the global canonical state (host arrays); 16-bit slabs all store with the scales the whole
        cavity's maxima give, so that they round alike."""
        if self.storage != B.FDTD_F32:
            m_e = max(float(np.max(np.abs(a))) for a in fields[:3])
            m_h = max(float(np.max(np.abs(a))) for a in fields[3:])
            s_e, s_h = B.fdtd_storage_scale_of(m_e), B.fdtd_storage_scale_of(m_h)
            for h in self.handles:
                B.fdtd_set_storage_scales(h, s_e, s_h)
        nx, ny, _ = self.dims
        for h, (lo, hi, _, _) in zip(self.handles, self.locals):
            B.fdtd_set_fields(h, _slice(fields, lo, hi), dims=(nx, ny, hi - lo))
        self.fresh = False

    def exchange(self):
        for a, b in zip(self.handles[:-1], self.handles[1:]):
            B.fdtd_slab_exchange(a, b)
        self.fresh = True

    def step(self, n: int):
        left = int(n)
        while left > 0:
            if not self.fresh:
                self.exchange()
            m = min(left, self.per_exchange)
            for h in self.handles:
                B.fdtd_step(h, m)
            self.fresh = False
            left -= m

    def get_fields(self):
        """The global canonical state gathered from the owned planes of every slab."""
        nx, ny, nz = self.dims
        out = [np.zeros((nz + 1, ny + 1, nx + 1), np.float32) for _ in range(6)]
        for h, (k0, k1), (lo, hi, g_lo, g_hi) in zip(self.handles, self.ranges, self.locals):
            loc = [np.empty((hi - lo + 1, ny + 1, nx + 1), np.float32) for _ in range(6)]
            B.fdtd_get_fields(h, loc, dims=(nx, ny, hi - lo))
            for c in range(6):
                out[c][k0:k1] = loc[c][g_lo:g_lo + (k1 - k0)]
                if k1 == nz:
                    out[c][nz] = loc[c][hi - lo]
        return out

    def energy(self) -> float:
        """The cavity's energy: the sum of the slabs' owned parts (ghost cells refreshed first)."""
        if not self.fresh:
            self.exchange()
        return float(sum(B.fdtd_slab_energy(h) for h in self.handles))

    def divergence(self) -> tuple[float, float]:
        if not self.fresh:
            self.exchange()
        de = dh = 0.0
        for h in self.handles:
            a, b = B.fdtd_slab_divergence_sq(h)
            de += a
            dh += b
        return float(np.sqrt(de)), float(np.sqrt(dh))


class CtxSlab:
    """A slab context on this process's GPU in the shape DistributedSlab drives.  Halo buffers live in device
    memory (for NCCL) or, with host=True, in pinned host memory (for a CPU transport such as gloo)."""

    def __init__(self, handle, order: int, device=None, host: bool = False):
        import torch
        self.h = handle
        info = B.fdtd_slab_info(handle)
        self.has_lower, self.has_upper = info["g_lo"] > 0, info["g_hi"] > 0
        self.per_exchange = info["ghost"] // reach(order)
        n = B.fdtd_slab_halo_bytes(handle)
        self.nbytes = n
        self.device = device
        self.host = host

        def buf():
            if host:
                return torch.empty(n, dtype=torch.uint8, pin_memory=True)
            return torch.empty(n, dtype=torch.uint8, device=device or "cuda")
        self.send = [buf(), buf()]
        self.recv = [buf(), buf()]

    def export(self, side: int):
        B.fdtd_slab_export(self.h, side, self.send[side])   # a host export waits for its copy
        if not self.host:
            B.fdtd_sync(self.h)   # the send below reads the device buffer on another stream
        return self.send[side]

    def recv_buffer(self, side: int):
        return self.recv[side]

    def import_(self, side: int, buf):
        B.fdtd_slab_import(self.h, side, buf)

    def step(self, n: int):
        B.fdtd_step(self.h, n)


class DistributedSlab:
    """One slab per rank: slab r owns the r-th of split_planes(nz, world) and exchanges its ghost cells
    with ranks r - 1 and r + 1 through torch.distributed point-to-point messages."""

    def __init__(self, slab, rank: int, world: int, group=None):
        self.slab, self.rank, self.world, self.group = slab, rank, world, group
        self.fresh = False

    def exchange(self):
        import torch.distributed as dist
        reqs, recvs = [], []
        for side, peer, present in ((0, self.rank - 1, self.slab.has_lower), (1, self.rank + 1, self.slab.has_upper)):
            if not present:
                continue
            reqs.append(dist.isend(self.slab.export(side), peer, group=self.group))
            r = self.slab.recv_buffer(side)
            reqs.append(dist.irecv(r, peer, group=self.group))
            recvs.append((side, r))
        for q in reqs:
            q.wait()
        # a wait orders only torch's current stream after a device receive; the import runs on the slab's
        # own stream, so the received bytes must be complete on the device first
        if any(getattr(r, "is_cuda", False) for _, r in recvs):
            import torch
            torch.cuda.current_stream(recvs[0][1].device).synchronize()
        for side, r in recvs:
            self.slab.import_(side, r)
        self.fresh = True

    def step(self, n: int):
        left = int(n)
        while left > 0:
            if not self.fresh:
                self.exchange()
            m = min(left, self.slab.per_exchange)
            self.slab.step(m)
            self.fresh = False
            left -= m
