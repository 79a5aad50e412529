"""Cavity: an owning Python handle around one fdtd_ctx of the C ABI."""
from __future__ import annotations

import numpy as np

from . import binding as B


class Cavity:
    """A PEC box cavity of nx*ny*nz cells stepped on the GPU.

    ce/ch: None (vacuum), a scalar, or three canonical (nz+1, ny+1, nx+1) arrays of
    dt/(eps dx) at E positions and dt/(mu dx) at H positions.
    order: 2 (Eq. 2) or 4 (the staggered fourth-order (2,4) scheme, image-closed PEC walls).
    """

    def __init__(self, nx, ny, nz, dt, dx=1.0, ce=None, ch=None, storage=B.FDTD_F32, stream=None, order=2):
        self.dims = (int(nx), int(ny), int(nz))
        self.dt, self.dx, self.storage = float(dt), float(dx), int(storage)
        self.shape = (nz + 1, ny + 1, nx + 1)
        self.handle = B.fdtd_create(nx, ny, nz, dt, dx, ce, ch, storage, stream)
        if order != 2:
            try:
                B.fdtd_set_order(self.handle, order)
            except Exception:
                self.close()
                raise

    @property
    def order(self):
        return B.fdtd_get_order(self.handle)

    def set_fields(self, fields, on_device=False):
        B.fdtd_set_fields(self.handle, fields, int(on_device), dims=self.dims)

    def prefetch_fields(self, fields):
        """Start copying the next fields from host memory (pinned for overlap) while the cavity computes;
        load them with set_fields_prefetched.  The arrays are kept referenced until then."""
        self._prefetch_keep = B.fdtd_prefetch_fields(self.handle, fields, dims=self.dims)

    def set_fields_prefetched(self):
        B.fdtd_set_fields_prefetched(self.handle)
        self._prefetch_keep = None

    def get_fields(self, out=None, on_device=False):
        if out is None:
            out = [np.empty(self.shape, dtype=np.float32) for _ in range(6)]
        B.fdtd_get_fields(self.handle, out, int(on_device), dims=self.dims)
        return out

    def step(self, n=1):
        B.fdtd_step(self.handle, n)

    def energy(self):
        return B.fdtd_energy(self.handle)

    def divergence(self):
        return B.fdtd_divergence(self.handle)

    def sync(self):
        B.fdtd_sync(self.handle)

    def tune(self, **kw):
        B.fdtd_set_tuning(self.handle, **kw)

    def set_sources(self, sources, wave):
        """Point currents (Eq. 1's J): sources [(comp 0..2, i, j, k), ...], wave (nsrc, steps)."""
        B.fdtd_set_sources(self.handle, sources, wave)

    def set_probes(self, probes, capacity: int):
        """Record [(comp 0..5, i, j, k), ...] after every step, up to `capacity` steps."""
        self._probes = (len(probes), int(capacity))
        B.fdtd_set_probes(self.handle, probes, capacity)

    def get_probes(self):
        """(nprobe, recorded steps) array of the probed values (physical units)."""
        n, cap = getattr(self, "_probes", (0, 0))
        return B.fdtd_get_probes(self.handle, n, cap)

    def autotune(self, trial_steps: int = 16):
        """Pick the fastest kernel and launch shape on this cavity's state; returns (tuning, ms/step)."""
        return B.fdtd_autotune(self.handle, trial_steps)

    @property
    def steps_done(self):
        return B.fdtd_steps_done(self.handle)

    @property
    def device_bytes(self):
        return B.fdtd_device_bytes(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            B.fdtd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
