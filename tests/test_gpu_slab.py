"""z-slab decomposition on one GPU: slab contexts exchanging ghost cells device to device.

Each slab runs the ordinary kernels on its own planes; the exchange refreshes `ghost` cells of all six
fields per side, after which the owned cells stay exact for ghost // reach steps.  The gathered state must
equal the undivided cavity stepped by the same kernel bit for bit (FP32; and BF16 when every slab stores
with the whole cavity's scales), and the FP64 oracle to the contract bound; the owned energies and
squared divergences must add up to the cavity's.
"""
import numpy as np
import pytest

import cavity_inputs as ci
from tests.gpu_util import DT, ENERGY_DRIFT_F32, REL_L2_F32, compare_fields

pytestmark = pytest.mark.gpu

CASES = [
    # (order, kernel tuning, ghost): two-step kernel with 2 ghost cells (one launch per exchange), the same
    # with 4 (two launches), one-step kernel with 1, two rows per warp, the three-step kernel with 3 (one
    # launch per exchange), fourth order with 3 and 6
    (2, {"kernel": 3, "tile_y": 16}, 2),
    (2, {"kernel": 5, "tile_y": 10}, 3),
    (2, {"kernel": 3, "tile_y": 8, "use_graph": 1}, 4),
    (2, {"kernel": 2, "tile_y": 8}, 1),
    (2, {"kernel": 4, "tile_y": 16}, 2),
    (4, {"kernel": 2, "tile_y": 12}, 3),
    (4, {"kernel": 2, "tile_y": 8}, 6),
]


def _setup(dims, seed):
    sph = ci.sphere_list(seed, 4, dims, 3.0, 9.0)
    ce, ch = ci.sphere_coefficients(sph, *dims, DT)
    return ce, ch, ci.random_fields(seed + 1, *dims)


def _single(dims, ce, ch, f, steps, order, tuning, storage=0):
    from paper_2504_09118_gb300 import Cavity
    with Cavity(*dims, DT, 1.0, ce, ch, storage, order=order) as cav:
        cav.tune(**tuning)
        cav.set_fields(f)
        w0, d0 = cav.energy(), cav.divergence()
        cav.step(steps)
        return cav.get_fields(), w0, d0, cav.energy(), cav.divergence()


@pytest.mark.parametrize("nslabs", [2, 4])
@pytest.mark.parametrize("order,tuning,ghost", CASES)
def test_slabs_equal_one_cavity_bitwise(nslabs, order, tuning, ghost):
    import torch
    from paper_2504_09118_gb300.slab import SlabDomain
    dims = (67, 41, 53)
    steps = 23
    ce, ch, f = _setup(dims, 5)
    ref, w0, d0, w1, d1 = _single(dims, ce, ch, f, steps, order, tuning)
    streams = [torch.cuda.Stream() for _ in range(nslabs)]
    with SlabDomain(*dims, DT, 1.0, ce, ch, 0, nslabs, ghost, order, tuning, streams) as dom:
        dom.set_fields(f)
        ws0, ds0 = dom.energy(), dom.divergence()
        dom.step(steps)
        got = dom.get_fields()
        ws1, ds1 = dom.energy(), dom.divergence()
    for c, name in enumerate(ci.COMPONENTS):
        assert np.array_equal(got[c], ref[c]), name
    # owned parts add up to the cavity's invariants (summed in another order)
    for a, b in ((ws0, w0), (ws1, w1), (ds0[0], d0[0]), (ds0[1], d0[1]), (ds1[0], d1[0]), (ds1[1], d1[1])):
        assert abs(a - b) <= 1e-12 * abs(b), (a, b)


def test_slabs_vs_oracle():
    import oracle
    from paper_2504_09118_gb300.slab import SlabDomain
    dims = (70, 45, 61)
    steps = 40
    ce, ch, f = _setup(dims, 9)
    ref = oracle.as_f64(f)
    oracle.step(ref, [c.astype(np.float64) for c in ce], ch, steps, omp=True)
    with SlabDomain(*dims, DT, 1.0, ce, ch, 0, 3, 2, 2, {"kernel": 3}) as dom:
        dom.set_fields(f)
        w0 = dom.energy()
        dom.step(steps)
        got = dom.get_fields()
        w1 = dom.energy()
    compare_fields(got, ref, dims, REL_L2_F32)
    assert abs(w1 - w0) / w0 <= ENERGY_DRIFT_F32


def test_bf16_slabs_with_shared_scales_equal_one_cavity():
    from paper_2504_09118_gb300.slab import SlabDomain
    dims = (59, 33, 40)
    ce, ch, f = _setup(dims, 13)
    tuning = {"kernel": 3, "tile_y": 16}
    ref, *_ = _single(dims, ce, ch, f, 18, 2, tuning, storage=2)
    with SlabDomain(*dims, DT, 1.0, ce, ch, 2, 3, 2, 2, tuning) as dom:
        dom.set_fields(f)
        dom.step(18)
        got = dom.get_fields()
    for c, name in enumerate(ci.COMPONENTS):
        assert np.array_equal(got[c], ref[c]), name


def test_host_export_import_equals_device_exchange():
    """The buffer path (export to host memory, import from it: what a message-passing exchange carries)
    gives the same state as the direct device-to-device exchange."""
    from paper_2504_09118_gb300 import binding as B
    from paper_2504_09118_gb300.slab import SlabDomain
    dims = (40, 30, 24)
    ce, ch, f = _setup(dims, 17)
    out = []
    for mode in ("device", "host"):
        with SlabDomain(*dims, DT, 1.0, ce, ch, 0, 2, 2, 2, {"kernel": 3}) as dom:
            dom.set_fields(f)
            for _ in range(6):
                if mode == "device":
                    dom.exchange()
                else:
                    lo, hi = dom.handles
                    n = B.fdtd_slab_halo_bytes(lo)
                    up, down = np.empty(n, np.uint8), np.empty(n, np.uint8)
                    B.fdtd_slab_export(lo, 1, up)
                    B.fdtd_slab_export(hi, 0, down)
                    B.fdtd_slab_import(hi, 0, up)
                    B.fdtd_slab_import(lo, 1, down)
                for h in dom.handles:
                    B.fdtd_step(h, 2)
            out.append(dom.get_fields())
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_slab_rules():
    from paper_2504_09118_gb300 import FdtdError
    from paper_2504_09118_gb300 import binding as B
    nx, ny, nz = 16, 12, 20
    # ghosts outside the cavity, a slab owning fewer planes than the ghost depth, a bad ghost depth
    for k0, k1, g in ((1, 10, 2), (0, 2, 3), (0, 10, 0)):
        with pytest.raises(FdtdError) as e:
            B.fdtd_create_slab(nx, ny, nz, k0, k1, g, DT)
        assert e.value.code == B.FDTD_ERR_ARG
    lo = B.fdtd_create_slab(nx, ny, nz, 0, 10, 2, DT)
    hi = B.fdtd_create_slab(nx, ny, nz, 10, 20, 2, DT)
    try:
        assert B.fdtd_slab_info(lo) == dict(nz_global=nz, k0=0, k1=10, g_lo=0, g_hi=2, ghost=2, steps_left=0)
        f = ci.random_fields(1, nx, ny, 12)
        B.fdtd_set_fields(lo, f)
        B.fdtd_set_fields(hi, f)
        with pytest.raises(FdtdError) as e:       # ghosts untrusted after a load
            B.fdtd_step(lo, 1)
        assert e.value.code == B.FDTD_ERR_STATE
        B.fdtd_slab_exchange(lo, hi)
        assert B.fdtd_slab_info(hi)["steps_left"] == 2
        B.fdtd_step(lo, 2)
        with pytest.raises(FdtdError):            # the ghosts cover two steps
            B.fdtd_step(lo, 1)
        with pytest.raises(FdtdError):            # reductions need current ghosts
            B.fdtd_slab_energy(lo)
        with pytest.raises(FdtdError):            # the lower slab has no neighbour below
            B.fdtd_slab_export(lo, 0, np.empty(B.fdtd_slab_halo_bytes(lo), np.uint8))
        with pytest.raises(FdtdError):            # not neighbours in this order
            B.fdtd_slab_exchange(hi, lo)
        with pytest.raises(FdtdError):
            B.fdtd_set_storage_scales(lo, 3.0, 1.0)
        assert B.fdtd_storage_scale_of(1.0) == 256.0 and B.fdtd_storage_scale_of(0.3) == 512.0
        # a fixed FP16 scale that the loaded values would overflow is refused at the load
        h16 = B.fdtd_create(nx, ny, 12, DT, 1.0, None, None, B.FDTD_F16)
        try:
            B.fdtd_set_storage_scales(h16, 2.0 ** 20, 256.0)
            with pytest.raises(FdtdError) as e:
                B.fdtd_set_fields(h16, f)
            assert e.value.code == B.FDTD_ERR_ARG
            B.fdtd_set_storage_scales(h16, 256.0, 256.0)
            B.fdtd_set_fields(h16, f)
        finally:
            B.fdtd_destroy(h16)
    finally:
        B.fdtd_destroy(lo)
        B.fdtd_destroy(hi)
