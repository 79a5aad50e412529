"""GB300 (sm_103a) Yee FDTD: fused, TMA-pipelined CUDA stencil behind a C ABI.

The package holds the CUDA sources (csrc/), their build step (build.py), the
ctypes binding of the C ABI (binding.py, same names as include/fdtd.h), and
the host-side batching, autotuning and serving layers built on that ABI.
"""
from .binding import *  # noqa: F401,F403
from .binding import EXPORTS, FdtdError, lib  # noqa: F401
from .cavity import Cavity  # noqa: F401
