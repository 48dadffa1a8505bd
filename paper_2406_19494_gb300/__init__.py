"""GB300 (sm_103a) finite-volume compressible Navier-Stokes solver: WENO5 + HLLC + fourth-order
central dissipative fluxes in an explicit TVD-RK3 step, behind the C ABI of include/fluid.h.

Submodules
----------
workloads  seeded synthetic cases and initial fields (numpy only)
native     ctypes declarations of the C ABI and the library loader
solver     torch binding (Solver) -- imports torch and loads libfluid.so on first use
build      in-tree nvcc build of libfluid.so
"""
from . import workloads  # noqa: F401


def Solver(*args, **kwargs):
    from .solver import Solver as _S
    return _S(*args, **kwargs)
