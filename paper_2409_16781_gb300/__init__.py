"""GB300-native D3Q19 lattice-Boltzmann update (arXiv 2409.16781, extended to 3D).

The compute path is liblbgb.so (hand-written sm_103a CUDA behind the C ABI of
include/lbgb.h); this package holds its ctypes binding, the batched serving
loop and the seeded workload generators.
"""
from ._lib import LbError, LbDiverged  # noqa: F401
from .lattice import Lattice, bytes_required, velocity_set  # noqa: F401

__all__ = ["Lattice", "LbError", "LbDiverged", "bytes_required", "velocity_set"]
