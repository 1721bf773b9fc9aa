"""GB300 (sm_103a) exponential p-multigrid solver for steady Euler flow with modal DG.

The compute path is the CUDA library ``libemg.so`` (C ABI in ``include/emg.h``); this
package only marshals arguments to it (``Solver``) and builds it (``build``).
"""
from ._lib import EmgError, Solver, build_info, load  # noqa: F401

__all__ = ["Solver", "EmgError", "build_info", "load"]
