"""GB300 (sm_103a) DA-based fast multipole method for the Coulomb potential and field.

The compute path is libdafmm.so (CUDA C++, include/dafmm.h); this package holds its
build script (``_build``), the symbolic-DA code generator (``gen``), the ctypes
binding (``binding``) and the seeded synthetic workloads (``workloads``).
"""
from . import binding  # noqa: F401
from .binding import Context, Tree  # noqa: F401
