"""GB300-native AMG-DD solve phase (algebraic multigrid domain decomposition).

The library is libamgdd.so (C ABI in include/amgdd.h): host setup of the AMG
hierarchy and composite grids, and sm_103a CUDA kernels for every step of the
solve phase. `capi` is its ctypes binding with the same function names;
`Solver` wraps a handle with torch device tensors.
"""
from . import capi  # noqa: F401
from .solver import Solver  # noqa: F401
