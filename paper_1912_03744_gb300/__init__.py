"""GB300-native (sm_103a) ADI heat solver for layered axisymmetric cylinders.

The compute path is libheat.so (CUDA kernels behind the C ABI in
include/heat.h); this package is its thin Python binding.
"""
from .heat import HeatBatch, HeatError, HeatNl, HeatSolver, load, LIB_PATH, SYMBOLS  # noqa: F401
from .surrogate import Surrogate, SURR_SYMBOLS  # noqa: F401
