"""Shared test helpers: seeded non-trivial states built from the oracle's geometry."""
import numpy as np

from oracle.basis import degrees
from workloads import standard_normal_modes


def perturbed_state(dg, p=None, seed=1807, amp=1e-2):
    """U_inf + amp * U_inf-scaled seeded draws decaying as 1/(1+deg)^2 on every mode.

    Returned as modal coefficients (coefficient = element mean * sqrt|E| for mode 0).
    """
    p = dg.p_max if p is None else p
    n = dg.N(p)
    xi = standard_normal_modes(dg.E, 5, n, seed)
    deg = degrees(dg.dim, p)
    scale = np.abs(dg.Uinf).copy()
    scale[1:4] = max(scale[1:3].max(), 1e-1)
    if dg.dim == 2:
        scale[3] = 0.0
    w = amp * scale[None, :, None] * xi / (1.0 + deg[None, None, :]) ** 2
    w[:, :, 0] += dg.Uinf[None, :]
    return w * np.sqrt(dg.mesh.vol)[:, None, None]


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    den = max(np.abs(b).max(), 1e-300)
    return float(np.abs(a - b).max() / den)
