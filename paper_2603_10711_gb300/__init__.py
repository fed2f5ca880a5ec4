"""GPU-native sequential convex programming with a consensus-ADMM inner
solver (arXiv 2603.10711) for NVIDIA GB300 (sm_103a).

The compute path is the CUDA library ``libucn.so`` (sources in ``csrc/``,
C ABI in ``include/ucn.h``); ``ucn`` is its ctypes binding.
"""
from . import ucn  # noqa: F401
from .ucn import Solver, UcnError  # noqa: F401
