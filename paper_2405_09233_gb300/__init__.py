"""GB300-native tensor Krylov solvers for the Sylvester tensor equation A*X - X*B = C.

The compute path is libtstar.so (hand-written CUDA for sm_103a behind the C ABI of
include/tstar.h); `binding` is its thin ctypes wrapper and `inputs` holds the
seeded synthetic workloads.  See include/tstar.h for the entry points.
"""
from .binding import Context, Operator, SolveResult, TstarError, lib, LIB_PATH  # noqa: F401

__all__ = ["Context", "Operator", "SolveResult", "TstarError", "lib", "LIB_PATH"]
