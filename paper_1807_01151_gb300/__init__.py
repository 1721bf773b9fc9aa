"""GB300 (sm_103a) exponential p-multigrid solver for steady Euler flow with modal DG.

The compute path is the CUDA library ``libemg.so`` (C ABI in ``include/emg.h``); this
package only marshals arguments to it (``Solver``) and builds it (``build``).
"""
from ._lib import EmgError, Server, Solver, build_info, estimate_device_bytes, load  # noqa: F401

__all__ = ["Solver", "Server", "EmgError", "build_info", "estimate_device_bytes", "load"]
