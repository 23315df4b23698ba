"""B300-native alternating-minimisation multi-agent trajectory optimiser.

The solver lives in libamto.so (CUDA, sm_103a) behind the C ABI of
include/amto.h; `amto` is its ctypes binding.
"""
from . import amto  # noqa: F401
from .amto import AmtoError, Mixed, Planner, Server  # noqa: F401
