"""GB300-native macromodel + AIM solver for scattering from large arrays of PEC elements.

The compute path is the C-ABI library libmacroaim (include/macroaim.h): host
FP64 set-up (macromodel build, AIM grid, precorrected near field) and sm_103a
CUDA kernels for the GMRES matrix-vector product of eq. (MV_product1) of
Patel, Triverio and Hum (arXiv 1712.02443).  This package is its thin ctypes
binding (``_binding``), a builder (``build``) and the seeded synthetic
workloads (``workloads``).  There is no CPU fallback: the binding raises if the
library is not built.
"""
from . import workloads  # noqa: F401
from ._binding import *  # noqa: F401,F403
from ._binding import load, exported_symbols, MacroAIMError  # noqa: F401
