"""B300-native (sm_103a) 1D viscous Burgers solvers of arXiv 2601.12204.

Explicit forward-Euler upwind/central steps (Eq. 21) and lagged-coefficient
upwind BTCS steps (Sec. 2.4, Eq. 23; Thomas-type partitioned solves, cyclic
systems through Sherman-Morrison) run in hand-written CUDA kernels behind the
C ABI of include/burgers.h (libburgers.so). Importing this package loads
nothing; ``Context`` loads the library on first use and raises if it is
missing (there is no CPU fallback).
"""
from ._lib import (BURGERS_BTCS, BURGERS_DIRICHLET, BURGERS_EXPLICIT, BURGERS_F32,  # noqa: F401
                   BURGERS_F64, BURGERS_PERIODIC, BurgersError)


def __getattr__(name):
    if name in ("Batch", "Context"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
