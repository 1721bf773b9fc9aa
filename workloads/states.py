"""Seeded random draws used to build non-trivial test states.

Only raw draws live here; turning them into modal coefficients (which needs
element volumes and the basis ordering) is done by the caller.
"""
import numpy as np


def standard_normal_modes(n_elems, n_vars, n_modes, seed=1807):
    """float64 [n_elems][n_vars][n_modes] standard normal draws (numpy PCG64)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n_elems, n_vars, n_modes))
