"""GB300-native ensemble Gillespie SSA with on-device time-aligned mean/variance.

The compute path is libssa (CUDA kernels for sm_103a behind the C ABI in
``include/ssa.h``); this package holds its sources (``csrc/``), the in-tree
build (``build.py``) and the ctypes binding (``binding.py``).
"""
from .binding import (EXPORTS, Batch, EnsembleResult, Model, RunOpts, RunStats, SSAError, ensemble_avg_xy,
                      ensemble_grad, ensemble_run, lib, library_path, make_opts, release_cached_memory,
                      workspace_bytes)

__all__ = ["EXPORTS", "Batch", "EnsembleResult", "Model", "RunOpts", "RunStats", "SSAError", "ensemble_avg_xy",
           "ensemble_grad",
           "ensemble_run", "lib", "library_path", "make_opts", "release_cached_memory", "workspace_bytes"]
