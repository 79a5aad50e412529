"""ctypes binding of libfdtd.so: the C ABI of include/fdtd.h under the same names.

Argument marshalling only.  Every computation happens in the CUDA library;
when the library cannot be built or loaded, importing a function raises.
PyTorch is optional here: device tensors are accepted wherever the C ABI takes
device pointers (on_device=1), and a torch.cuda.Stream (or a raw handle) may be
passed as the stream.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

FDTD_F32, FDTD_F16, FDTD_BF16 = 0, 1, 2
FDTD_OK, FDTD_ERR_ARG, FDTD_ERR_OOM, FDTD_ERR_CUDA, FDTD_ERR_TIMEOUT, FDTD_ERR_STATE, FDTD_ERR_UNSTABLE = (
    0, -1, -2, -3, -4, -5, -6)
(FDTD_KERNEL_AUTO, FDTD_KERNEL_SIMPLE, FDTD_KERNEL_FUSED, FDTD_KERNEL_TEMPORAL, FDTD_KERNEL_TEMPORAL2,
 FDTD_KERNEL_TEMPORAL3) = 0, 1, 2, 3, 4, 5
STATUS_NAMES = {0: "OK", -1: "ERR_ARG", -2: "ERR_OOM", -3: "ERR_CUDA", -4: "ERR_TIMEOUT", -5: "ERR_STATE",
                -6: "ERR_UNSTABLE"}

# Every entry point declared in include/fdtd.h (checked against the header by the tests).
EXPORTS = (
    "fdtd_create", "fdtd_set_fields", "fdtd_step", "fdtd_get_fields", "fdtd_energy", "fdtd_divergence",
    "fdtd_sync", "fdtd_set_tuning", "fdtd_steps_done", "fdtd_device_bytes", "fdtd_destroy", "fdtd_last_error",
    "fdtd_batch_create", "fdtd_batch_add", "fdtd_batch_remove", "fdtd_batch_step", "fdtd_batch_set_tuning",
    "fdtd_batch_size", "fdtd_batch_sync", "fdtd_batch_destroy", "fdtd_batch_last_error",
    "fdtd_debug_inject_timeout", "fdtd_version", "fdtd_energy_static", "fdtd_batch_set_steps",
    "fdtd_batch_steps_done", "fdtd_autotune", "fdtd_batch_autotune", "fdtd_set_sources", "fdtd_set_probes",
    "fdtd_get_probes", "fdtd_set_order", "fdtd_get_order", "fdtd_batch_retune", "fdtd_prefetch_fields",
    "fdtd_set_fields_prefetched", "fdtd_debug_fail_alloc", "fdtd_debug_tile_plan", "fdtd_debug_pec_code",
    "fdtd_debug_pec_table",
    "fdtd_create_slab", "fdtd_slab_info", "fdtd_slab_halo_bytes", "fdtd_slab_export", "fdtd_slab_import",
    "fdtd_slab_exchange", "fdtd_slab_energy", "fdtd_slab_divergence_sq", "fdtd_set_storage_scales",
    "fdtd_storage_scale_of",
)


class FdtdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class fdtd_tuning(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("tile_y", ctypes.c_int), ("zchunk", ctypes.c_int),
                ("ctas_per_sm", ctypes.c_int), ("stages", ctypes.c_int), ("use_graph", ctypes.c_int)]


_LIB = None
_LOCK = threading.Lock()


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Load libfdtd.so (building it first when the sources are newer and nvcc exists)."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            if not _build.up_to_date():
                try:
                    _build.build()
                except Exception as e:   # no silent fallback: the CUDA library is the only implementation
                    if not os.path.exists(_build.LIB):
                        raise ImportError(f"libfdtd.so is missing and could not be built: {e}") from e
            L = ctypes.CDLL(_build.LIB)
            vp, i, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
            L.fdtd_create.argtypes = [ctypes.POINTER(vp), i, i, i, d, d, vp, vp, i, vp]
            L.fdtd_set_fields.argtypes = [vp, vp, i]
            L.fdtd_step.argtypes = [vp, i]
            L.fdtd_get_fields.argtypes = [vp, vp, i]
            L.fdtd_energy.argtypes = [vp, ctypes.POINTER(d)]
            L.fdtd_divergence.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(d)]
            L.fdtd_sync.argtypes = [vp]
            L.fdtd_set_tuning.argtypes = [vp, ctypes.POINTER(fdtd_tuning)]
            L.fdtd_steps_done.argtypes = [vp]
            L.fdtd_steps_done.restype = ll
            L.fdtd_device_bytes.argtypes = [vp]
            L.fdtd_device_bytes.restype = ll
            L.fdtd_destroy.argtypes = [vp]
            L.fdtd_destroy.restype = None
            L.fdtd_last_error.argtypes = [vp]
            L.fdtd_last_error.restype = ctypes.c_char_p
            L.fdtd_batch_create.argtypes = [ctypes.POINTER(vp), i, vp]
            L.fdtd_batch_add.argtypes = [vp, vp]
            L.fdtd_batch_remove.argtypes = [vp, vp]
            L.fdtd_batch_step.argtypes = [vp, i]
            L.fdtd_batch_set_tuning.argtypes = [vp, ctypes.POINTER(fdtd_tuning)]
            L.fdtd_batch_size.argtypes = [vp]
            L.fdtd_batch_sync.argtypes = [vp]
            L.fdtd_batch_destroy.argtypes = [vp]
            L.fdtd_batch_destroy.restype = None
            L.fdtd_batch_last_error.argtypes = [vp]
            L.fdtd_batch_last_error.restype = ctypes.c_char_p
            L.fdtd_debug_inject_timeout.argtypes = [vp, i]
            L.fdtd_batch_set_steps.argtypes = [vp, vp, ll]
            L.fdtd_batch_steps_done.argtypes = [vp]
            L.fdtd_batch_steps_done.restype = ll
            L.fdtd_version.restype = ctypes.c_char_p
            L.fdtd_energy_static.argtypes = [i, i, i, d, d, vp, vp, vp, vp, vp]
            L.fdtd_autotune.argtypes = [vp, i, ctypes.POINTER(fdtd_tuning), ctypes.POINTER(d)]
            L.fdtd_batch_autotune.argtypes = [vp, i, ctypes.POINTER(fdtd_tuning), ctypes.POINTER(d)]
            L.fdtd_set_sources.argtypes = [vp, i, vp, vp, vp, i]
            L.fdtd_set_probes.argtypes = [vp, i, vp, vp, i]
            L.fdtd_get_probes.argtypes = [vp, vp, ctypes.POINTER(i)]
            L.fdtd_set_order.argtypes = [vp, i]
            L.fdtd_prefetch_fields.argtypes = [vp, vp]
            L.fdtd_debug_fail_alloc.argtypes = [i]
            L.fdtd_debug_tile_plan.argtypes = [ll, i, i, i, i, vp, i, ctypes.POINTER(i), ctypes.POINTER(ll), vp]
            L.fdtd_debug_pec_code.argtypes = [i, i, i, i, i, ctypes.POINTER(i)]
            L.fdtd_debug_pec_table.argtypes = [vp, i, vp]
            L.fdtd_set_fields_prefetched.argtypes = [vp]
            L.fdtd_batch_retune.argtypes = [vp, i, ctypes.POINTER(fdtd_tuning), ctypes.POINTER(d),
                                            ctypes.POINTER(i)]
            L.fdtd_get_order.argtypes = [vp]
            L.fdtd_create_slab.argtypes = [ctypes.POINTER(vp), i, i, i, i, i, i, d, d, vp, vp, i, vp]
            L.fdtd_slab_info.argtypes = [vp, vp]
            L.fdtd_slab_halo_bytes.argtypes = [vp]
            L.fdtd_slab_halo_bytes.restype = ll
            L.fdtd_slab_export.argtypes = [vp, i, vp, i]
            L.fdtd_slab_import.argtypes = [vp, i, vp, i]
            L.fdtd_slab_exchange.argtypes = [vp, vp]
            L.fdtd_slab_energy.argtypes = [vp, ctypes.POINTER(d)]
            L.fdtd_slab_divergence_sq.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(d)]
            L.fdtd_set_storage_scales.argtypes = [vp, d, d]
            L.fdtd_storage_scale_of.argtypes = [d]
            L.fdtd_storage_scale_of.restype = d
            _LIB = L
        return _LIB


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream or None
    h = getattr(stream, "cuda_stream", None)
    if h is None:
        raise TypeError("stream must be a torch.cuda.Stream or an int handle")
    return int(h) or None


def _check(ctx, rc: int) -> None:
    if rc != FDTD_OK:
        msg = lib().fdtd_last_error(ctx)
        raise FdtdError(rc, msg.decode() if msg else "")


def _host_f32(a, shape):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if a.shape != shape and a.size != int(np.prod(shape)):
        raise ValueError(f"array of shape {a.shape} does not match canonical shape {shape}")
    return a


def _ptr_array(ptrs):
    return (ctypes.c_void_p * len(ptrs))(*ptrs)


def fdtd_create(nx: int, ny: int, nz: int, dt: float, dx: float = 1.0, ce=None, ch=None,
                storage: int = FDTD_F32, stream=None):
    """Create a cavity; ce/ch are None or three canonical host arrays.  Returns the context handle."""
    L = lib()
    shape = (nz + 1, ny + 1, nx + 1)
    keep = []

    def arr3(c):
        if c is None:
            return None
        if np.isscalar(c):
            c = [c, c, c]
        vs = [np.ascontiguousarray(np.broadcast_to(np.asarray(v, dtype=np.float32), shape)) for v in c]
        keep.extend(vs)
        return _ptr_array([v.ctypes.data for v in vs])

    ce_p, ch_p = arr3(ce), arr3(ch)
    out = ctypes.c_void_p()
    rc = L.fdtd_create(ctypes.byref(out), int(nx), int(ny), int(nz), float(dt), float(dx),
                       ctypes.cast(ce_p, ctypes.c_void_p) if ce_p is not None else None,
                       ctypes.cast(ch_p, ctypes.c_void_p) if ch_p is not None else None,
                       int(storage), _stream_handle(stream))
    _check(None, rc)
    return out.value


def fdtd_create_slab(nx: int, ny: int, nz_global: int, k0: int, k1: int, ghost: int, dt: float, dx: float = 1.0,
                     ce=None, ch=None, storage: int = FDTD_F32, stream=None):
    """A z-slab [k0, k1) of an nx*ny*nz_global cavity with `ghost` cells on each side that has a neighbour;
    ce/ch are None or canonical host arrays of the slab's local planes (k0 - g_lo .. k1 + g_hi)."""
    L = lib()
    g_lo = ghost if k0 > 0 else 0
    g_hi = ghost if k1 < nz_global else 0
    shape = (k1 - k0 + g_lo + g_hi + 1, ny + 1, nx + 1)
    keep = []

    def arr3(c):
        if c is None:
            return None
        if np.isscalar(c):
            c = [c, c, c]
        vs = [np.ascontiguousarray(np.broadcast_to(np.asarray(v, dtype=np.float32), shape)) for v in c]
        keep.extend(vs)
        return _ptr_array([v.ctypes.data for v in vs])

    ce_p, ch_p = arr3(ce), arr3(ch)
    out = ctypes.c_void_p()
    rc = L.fdtd_create_slab(ctypes.byref(out), int(nx), int(ny), int(nz_global), int(k0), int(k1), int(ghost),
                            float(dt), float(dx),
                            ctypes.cast(ce_p, ctypes.c_void_p) if ce_p is not None else None,
                            ctypes.cast(ch_p, ctypes.c_void_p) if ch_p is not None else None,
                            int(storage), _stream_handle(stream))
    _check(None, rc)
    return out.value


def fdtd_slab_info(ctx) -> dict:
    info = (ctypes.c_int * 7)()
    _check(ctx, lib().fdtd_slab_info(ctx, info))
    return dict(zip(("nz_global", "k0", "k1", "g_lo", "g_hi", "ghost", "steps_left"), list(info)))


def fdtd_slab_halo_bytes(ctx) -> int:
    return int(lib().fdtd_slab_halo_bytes(ctx))


def _buffer(buf, writable: bool):
    """(pointer, on_device) of a halo buffer: a CUDA tensor, a CPU tensor or a numpy array (contiguous)."""
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("halo buffers must be contiguous")
        return buf.data_ptr(), bool(getattr(buf, "is_cuda", False))
    if not (isinstance(buf, np.ndarray) and buf.flags.c_contiguous and (buf.flags.writeable or not writable)):
        raise ValueError("halo buffers must be contiguous (and writable for an export)")
    return buf.ctypes.data, False


def fdtd_slab_export(ctx, side: int, buf) -> None:
    """Owned boundary cells of one side into buf: a device tensor (stream-ordered) or host memory (a CPU
    tensor or numpy array; the call waits for the copy)."""
    ptr, on_device = _buffer(buf, True)
    if buf.nbytes < fdtd_slab_halo_bytes(ctx):
        raise ValueError("halo buffer smaller than fdtd_slab_halo_bytes")
    _check(ctx, lib().fdtd_slab_export(ctx, int(side), ptr, int(on_device)))


def fdtd_slab_import(ctx, side: int, buf) -> None:
    ptr, on_device = _buffer(buf, False)
    if buf.nbytes < fdtd_slab_halo_bytes(ctx):
        raise ValueError("halo buffer smaller than fdtd_slab_halo_bytes")
    _check(ctx, lib().fdtd_slab_import(ctx, int(side), ptr, int(on_device)))


def fdtd_slab_exchange(lo, hi) -> None:
    _check(lo, lib().fdtd_slab_exchange(lo, hi))


def fdtd_slab_energy(ctx) -> float:
    w = ctypes.c_double()
    _check(ctx, lib().fdtd_slab_energy(ctx, ctypes.byref(w)))
    return w.value


def fdtd_slab_divergence_sq(ctx) -> tuple[float, float]:
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib().fdtd_slab_divergence_sq(ctx, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def fdtd_set_storage_scales(ctx, s_e: float, s_h: float) -> None:
    _check(ctx, lib().fdtd_set_storage_scales(ctx, float(s_e), float(s_h)))


def fdtd_storage_scale_of(maxabs: float) -> float:
    return float(lib().fdtd_storage_scale_of(float(maxabs)))


def _field_ptrs(fields, shape, on_device: bool, writable: bool):
    if len(fields) != 6:
        raise ValueError("need six fields Ex, Ey, Ez, Hx, Hy, Hz")
    if on_device:
        ptrs = []
        for t in fields:
            if str(t.dtype) != "torch.float32" or not t.is_contiguous() or t.numel() != int(np.prod(shape)):
                raise ValueError("device fields must be contiguous float32 tensors of the canonical size")
            ptrs.append(t.data_ptr())
        # the library reads / writes them on its own stream: torch's pending work on them must be done
        import torch
        torch.cuda.current_stream(fields[0].device).synchronize()
        return ptrs, fields
    arrs = []
    for a in fields:
        if writable:
            if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags.c_contiguous and a.size == int(np.prod(shape))):
                raise ValueError("host output fields must be C-contiguous float32 arrays of the canonical size")
            arrs.append(a)
        else:
            arrs.append(_host_f32(a, shape))
    return [a.ctypes.data for a in arrs], arrs


def fdtd_set_fields(ctx, fields, on_device: int = 0, dims=None) -> None:
    nx, ny, nz = dims if dims is not None else _dims_of(fields)
    ptrs, keep = _field_ptrs(fields, (nz + 1, ny + 1, nx + 1), bool(on_device), False)
    _check(ctx, lib().fdtd_set_fields(ctx, ctypes.cast(_ptr_array(ptrs), ctypes.c_void_p), int(on_device)))
    del keep


def fdtd_prefetch_fields(ctx, fields, dims=None):
    """Start the host-to-device copy of the next fields; returns the host arrays the copy reads, which
    the caller must keep alive and unchanged until fdtd_set_fields_prefetched."""
    nx, ny, nz = dims if dims is not None else _dims_of(fields)
    ptrs, keep = _field_ptrs(fields, (nz + 1, ny + 1, nx + 1), False, False)
    _check(ctx, lib().fdtd_prefetch_fields(ctx, ctypes.cast(_ptr_array(ptrs), ctypes.c_void_p)))
    return keep


def fdtd_debug_fail_alloc(after: int) -> None:
    """Make the library's device allocation after `after` more successes fail once (-1 disarms)."""
    lib().fdtd_debug_fail_alloc(int(after))


def fdtd_debug_tile_plan(cols: int, nz: int, ctas: int, prologue: int, zchunk: int = 0,
                         assignment: bool = True) -> tuple[list[int], int, np.ndarray | None]:
    """Host-only work split of one cavity: (chunk lengths, makespan in plane-times, CTA of each listed
    tile or None).  Needs no GPU."""
    cap = max(128, -(-int(nz) // int(zchunk))) if zchunk > 0 else 128   # the search tries at most 68 chunks
    chunks = np.zeros(cap, np.int32)
    n, ms = ctypes.c_int(0), ctypes.c_longlong(0)
    call = lambda out: lib().fdtd_debug_tile_plan(int(cols), int(nz), int(ctas), int(prologue), int(zchunk),
                                                  chunks.ctypes.data, cap, ctypes.byref(n), ctypes.byref(ms), out)
    rc = call(None)
    if rc != FDTD_OK:
        raise FdtdError(rc, "fdtd_debug_tile_plan: invalid arguments")
    cta = None
    if assignment:
        cta = np.full(n.value * int(cols), -1, np.int32)
        rc = call(cta.ctypes.data)
        if rc != FDTD_OK:
            raise FdtdError(rc, "fdtd_debug_tile_plan: invalid arguments")
    return [int(x) for x in chunks[:n.value]], int(ms.value), cta


def fdtd_debug_pec_code(ntab: int, mat: int, i: int, j: int, k: int) -> int:
    """Host-only: the PEC-coded id the two-step kernels read for a cell of material `mat` at (i, j, k)."""
    code = ctypes.c_int(0)
    rc = lib().fdtd_debug_pec_code(int(ntab), int(mat), int(i), int(j), int(k), ctypes.byref(code))
    if rc != FDTD_OK:
        raise FdtdError(rc, "fdtd_debug_pec_code: invalid arguments")
    return int(code.value)


def fdtd_debug_pec_table(tab) -> np.ndarray:
    """Host-only: the PEC-coded table built from tab (ntab x 8 floats), shape (1 + 8 ntab, 8)."""
    t = np.ascontiguousarray(np.asarray(tab, np.float32).reshape(-1, 8))
    out = np.zeros((1 + 8 * len(t), 8), np.float32)
    rc = lib().fdtd_debug_pec_table(t.ctypes.data, len(t), out.ctypes.data)
    if rc != FDTD_OK:
        raise FdtdError(rc, "fdtd_debug_pec_table: invalid arguments")
    return out


def fdtd_set_fields_prefetched(ctx) -> None:
    _check(ctx, lib().fdtd_set_fields_prefetched(ctx))


def fdtd_get_fields(ctx, fields, on_device: int = 0, dims=None) -> None:
    nx, ny, nz = dims if dims is not None else _dims_of(fields)
    ptrs, keep = _field_ptrs(fields, (nz + 1, ny + 1, nx + 1), bool(on_device), True)
    _check(ctx, lib().fdtd_get_fields(ctx, ctypes.cast(_ptr_array(ptrs), ctypes.c_void_p), int(on_device)))
    del keep


def _dims_of(fields):
    s = tuple(fields[0].shape)
    if len(s) != 3:
        raise ValueError("pass dims=(nx, ny, nz) for flat field arrays")
    return s[2] - 1, s[1] - 1, s[0] - 1


def fdtd_step(ctx, nsteps: int) -> None:
    _check(ctx, lib().fdtd_step(ctx, int(nsteps)))


def fdtd_energy(ctx) -> float:
    w = ctypes.c_double()
    _check(ctx, lib().fdtd_energy(ctx, ctypes.byref(w)))
    return w.value


def fdtd_divergence(ctx) -> tuple[float, float]:
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib().fdtd_divergence(ctx, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def fdtd_sync(ctx) -> None:
    _check(ctx, lib().fdtd_sync(ctx))


def fdtd_set_tuning(ctx, kernel=0, tile_y=0, zchunk=0, ctas_per_sm=0, stages=0, use_graph=0) -> None:
    t = fdtd_tuning(kernel, tile_y, zchunk, ctas_per_sm, stages, use_graph)
    _check(ctx, lib().fdtd_set_tuning(ctx, ctypes.byref(t)))


def fdtd_set_order(ctx, order: int) -> None:
    """Spatial order of the curl differences: 2 (Eq. 2) or 4 (the staggered (2,4) scheme)."""
    _check(ctx, lib().fdtd_set_order(ctx, int(order)))


def fdtd_get_order(ctx) -> int:
    return int(lib().fdtd_get_order(ctx))


def _tuning_dict(t) -> dict:
    return {k: int(getattr(t, k)) for k, _ in fdtd_tuning._fields_}


def fdtd_autotune(ctx, trial_steps: int = 16) -> tuple[dict, float]:
    """Time the candidate launch shapes on the context's state (restored afterwards), keep the
    fastest; returns (tuning, ms per step)."""
    t = fdtd_tuning()
    ms = ctypes.c_double()
    _check(ctx, lib().fdtd_autotune(ctx, int(trial_steps), ctypes.byref(t), ctypes.byref(ms)))
    return _tuning_dict(t), float(ms.value)


def fdtd_set_sources(ctx, sources, wave) -> None:
    """sources: [(comp, i, j, k), ...] with comp 0..2 (Ex, Ey, Ez); wave: (nsrc, wave_len) current J of
    each step (empty sources remove them)."""
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.int32).reshape(-1, 4))
    n = len(src)
    comp = np.ascontiguousarray(src[:, 0])
    ijk = np.ascontiguousarray(src[:, 1:])
    w = np.ascontiguousarray(np.asarray(wave, dtype=np.float32).reshape(n, -1)) if n else np.zeros((0, 1), np.float32)
    _check(ctx, lib().fdtd_set_sources(ctx, n, comp.ctypes.data if n else None, ijk.ctypes.data if n else None,
                                       w.ctypes.data if n else None, int(w.shape[1])))


def fdtd_set_probes(ctx, probes, capacity: int) -> None:
    """probes: [(comp, i, j, k), ...] with comp 0..5 (Ex..Hz); capacity: steps recorded."""
    pr = np.ascontiguousarray(np.asarray(probes, dtype=np.int32).reshape(-1, 4))
    n = len(pr)
    comp = np.ascontiguousarray(pr[:, 0])
    ijk = np.ascontiguousarray(pr[:, 1:])
    _check(ctx, lib().fdtd_set_probes(ctx, n, comp.ctypes.data if n else None, ijk.ctypes.data if n else None,
                                      int(capacity)))


def fdtd_get_probes(ctx, nprobe: int, capacity: int) -> np.ndarray:
    """(nprobe, recorded steps) float32 array of the probed values."""
    out = np.zeros((nprobe, capacity), dtype=np.float32)
    n = ctypes.c_int()
    _check(ctx, lib().fdtd_get_probes(ctx, out.ctypes.data, ctypes.byref(n)))
    return out[:, :n.value]


def fdtd_steps_done(ctx) -> int:
    return int(lib().fdtd_steps_done(ctx))


def fdtd_device_bytes(ctx) -> int:
    return int(lib().fdtd_device_bytes(ctx))


def fdtd_destroy(ctx) -> None:
    if ctx:
        lib().fdtd_destroy(ctx)


def fdtd_last_error(ctx=None) -> str:
    m = lib().fdtd_last_error(ctx)
    return m.decode() if m else ""


def fdtd_debug_inject_timeout(ctx, limit_us: int) -> None:
    _check(ctx, lib().fdtd_debug_inject_timeout(ctx, int(limit_us)))


def fdtd_energy_static(nx: int, ny: int, nz: int, dt: float, dx: float, fields, W, ce=None, ch=None,
                       stream=None) -> None:
    """Energy of canonical FP32 device tensors into the float64 device tensor W, allocating nothing.

    For callers that cannot allocate device memory where they need the energy.  The
    library's fixed scratch is shared by all calls: do not overlap calls on the GPU.
    """
    shape = (nz + 1, ny + 1, nx + 1)
    fptr, _ = _field_ptrs(fields, shape, True, False)
    if str(W.dtype) != "torch.float64" or not W.is_cuda:
        raise ValueError("W must be a float64 CUDA tensor")

    def coef(c):
        if c is None:
            return None
        if len(c) != 3:
            raise ValueError("coefficients are three device tensors")
        for t in c:
            if str(t.dtype) != "torch.float32" or not t.is_contiguous() or t.numel() != int(np.prod(shape)):
                raise ValueError("coefficients must be contiguous float32 tensors of the canonical size")
        return ctypes.cast(_ptr_array([t.data_ptr() for t in c]), ctypes.c_void_p)

    rc = lib().fdtd_energy_static(int(nx), int(ny), int(nz), float(dt), float(dx),
                                  ctypes.cast(_ptr_array(fptr), ctypes.c_void_p), coef(ce), coef(ch),
                                  W.data_ptr(), _stream_handle(stream))
    _check(None, rc)


def fdtd_version() -> str:
    return lib().fdtd_version().decode()


# ---------------------------------------------------------------- batches
def _bcheck(b, rc):
    if rc != FDTD_OK:
        m = lib().fdtd_batch_last_error(b)
        raise FdtdError(rc, m.decode() if m else "")


def fdtd_batch_create(storage: int = FDTD_F32, stream=None):
    out = ctypes.c_void_p()
    rc = lib().fdtd_batch_create(ctypes.byref(out), int(storage), _stream_handle(stream))
    if rc != FDTD_OK:
        raise FdtdError(rc, "fdtd_batch_create failed")
    return out.value


def fdtd_batch_add(b, ctx) -> None:
    _bcheck(b, lib().fdtd_batch_add(b, ctx))


def fdtd_batch_remove(b, ctx) -> None:
    _bcheck(b, lib().fdtd_batch_remove(b, ctx))


def fdtd_batch_step(b, nsteps: int) -> None:
    _bcheck(b, lib().fdtd_batch_step(b, int(nsteps)))


def fdtd_batch_set_tuning(b, kernel=0, tile_y=0, zchunk=0, ctas_per_sm=0, stages=0, use_graph=0) -> None:
    t = fdtd_tuning(kernel, tile_y, zchunk, ctas_per_sm, stages, use_graph)
    _bcheck(b, lib().fdtd_batch_set_tuning(b, ctypes.byref(t)))


def fdtd_batch_autotune(b, trial_steps: int = 16) -> tuple[dict, float]:
    """fdtd_autotune over a batch's current members (state and clock restored afterwards)."""
    t = fdtd_tuning()
    ms = ctypes.c_double()
    _bcheck(b, lib().fdtd_batch_autotune(b, int(trial_steps), ctypes.byref(t), ctypes.byref(ms)))
    return _tuning_dict(t), float(ms.value)


def fdtd_batch_retune(b, trial_steps: int = 16) -> tuple[dict, float, bool]:
    """Online re-tuning from the size-bucket model: (tuning, bucket ms per step, whether trials ran)."""
    t = fdtd_tuning()
    ms = ctypes.c_double()
    timed = ctypes.c_int()
    _bcheck(b, lib().fdtd_batch_retune(b, int(trial_steps), ctypes.byref(t), ctypes.byref(ms), ctypes.byref(timed)))
    return _tuning_dict(t), float(ms.value), bool(timed.value)


def fdtd_batch_set_steps(b, ctx, nsteps: int) -> None:
    _bcheck(b, lib().fdtd_batch_set_steps(b, ctx, int(nsteps)))


def fdtd_batch_steps_done(b) -> int:
    return int(lib().fdtd_batch_steps_done(b))


def fdtd_batch_size(b) -> int:
    return int(lib().fdtd_batch_size(b))


def fdtd_batch_sync(b) -> None:
    _bcheck(b, lib().fdtd_batch_sync(b))


def fdtd_batch_destroy(b) -> None:
    if b:
        lib().fdtd_batch_destroy(b)


def fdtd_batch_last_error(b) -> str:
    m = lib().fdtd_batch_last_error(b)
    return m.decode() if m else ""
