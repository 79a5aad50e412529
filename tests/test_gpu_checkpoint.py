"""Checkpoint / resume: fdtd_get_fields is the checkpoint and fdtd_set_fields restores it.  A run split
into two halves through a checkpoint (into a fresh context) equals the unsplit run bit for bit (FP32
storage), for every fused kernel and both spatial orders; and an injected allocation failure leaves the
library usable."""
import numpy as np
import pytest

import cavity_inputs as ci
from tests.gpu_util import DT

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("order,tuning", [(2, dict(kernel=3, tile_y=16)), (2, dict(kernel=2, tile_y=8)),
                                          (2, dict(kernel=1)), (4, dict(kernel=2, tile_y=12)),
                                          (4, dict(kernel=1))])
def test_split_run_through_a_checkpoint_is_bitwise_equal(order, tuning):
    from paper_2504_09118_gb300 import Cavity
    dims = (97, 41, 36)
    sph = ci.sphere_list(60, 4, dims, 3.0, 10.0)
    ce, ch = ci.sphere_coefficients(sph, *dims, DT)
    f = ci.random_fields(61, *dims)
    with Cavity(*dims, DT, 1.0, ce, ch, order=order) as cav:
        cav.tune(**tuning)
        cav.set_fields(f)
        cav.step(100)
        whole = cav.get_fields()
    with Cavity(*dims, DT, 1.0, ce, ch, order=order) as a:
        a.tune(**tuning)
        a.set_fields(f)
        a.step(50)
        ckpt = a.get_fields()
    with Cavity(*dims, DT, 1.0, ce, ch, order=order) as b:
        b.tune(**tuning)
        b.set_fields(ckpt)
        b.step(50)
        resumed = b.get_fields()
    for x, y, name in zip(whole, resumed, ci.COMPONENTS):
        assert np.array_equal(x, y), name


def test_injected_allocation_failure_is_reported_and_recovered():
    from paper_2504_09118_gb300 import Cavity, FdtdError, binding
    dims = (40, 30, 20)
    binding.fdtd_debug_fail_alloc(0)
    try:
        with pytest.raises(FdtdError) as e:
            Cavity(*dims, DT)
        assert e.value.code == binding.FDTD_ERR_OOM
    finally:
        binding.fdtd_debug_fail_alloc(-1)
    with Cavity(*dims, DT) as cav:                 # the next context is made and steps normally
        cav.set_fields(ci.random_fields(62, *dims))
        cav.step(4)
        assert np.isfinite(cav.energy())
