"""GB300-native PCG solver for layered 3D-IC thermal systems (CUTh-Solver's method).

The compute path is libthermal.so (hand-written sm_103a CUDA behind a C ABI,
``include/thermal.h``); this package is its Python binding.
"""
from ._lib import ThermalError, load  # noqa: F401
from .api import (HotspotLSE, SteadyAdjoint, ThermalGrid, make_opts,  # noqa: F401
                  solve_batched)

__all__ = ["ThermalGrid", "ThermalError", "make_opts", "solve_batched", "SteadyAdjoint", "HotspotLSE", "load"]
