"""GB300 (sm_103a) Position-Based Nonlinear Gauss-Seidel (arXiv 2306.09021).

The solver is the C ABI in include/pbng.h, implemented by the CUDA kernels and
host runtime under csrc/ and built in-tree by ``build.build()``.  This package
only marshals arguments to it.
"""

from ._lib import ACCEL, PRECISION, PbngError, PbngParams, load
from .mesh import Mesh, default_params, measure_fp32_peak
from .autograd import EquilibriumModel

__all__ = ["ACCEL", "PRECISION", "PbngError", "PbngParams", "load", "Mesh", "default_params",
           "EquilibriumModel", "measure_fp32_peak"]
