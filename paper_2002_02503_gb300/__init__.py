"""GB300 (sm_103a) lattice Boltzmann library with the Galilean-invariant filtered
collision of Chen, Zhang & Gopalakrishnan (arXiv 2002.02503).

``lbm`` is the ctypes binding of the C-ABI (``include/lbm.h``); ``fields``
generates seeded synthetic initial conditions; ``build`` compiles the CUDA
library in-tree.  The CUDA library is loaded lazily on the first call.
"""
from . import fields  # noqa: F401

__all__ = ["fields", "lbm", "build"]
