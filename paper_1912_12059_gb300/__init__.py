"""GB300 (sm_103a) DGSEM hot path of the parabolic relaxation model of the
Navier-Stokes-Korteweg equations (arXiv:1912.12059): the C-ABI library
libnsk.so (include/nsk.h), its ctypes binding and the seeded workloads."""
from .nsk import Solver, NskError, load_library  # noqa: F401

__all__ = ["Solver", "NskError", "load_library"]
