"""Seeded stream of steady-solve requests for the request loop (served cylinder solves).

Arrivals are a Poisson process (exponential gaps, mean 0.25 s = 4 requests/s); each
request draws its O-grid uniformly from 32x16, 64x32, 128x64 and 256x128, its order p
uniformly from 1..4 and its Mach number uniformly from [0.1, 0.5] (angle of attack 0).
Only random draws live here, none of the method's arithmetic.
"""
from dataclasses import dataclass

import numpy as np

GRIDS = ((32, 16), (64, 32), (128, 64), (256, 128))
ORDERS = (1, 2, 3, 4)


@dataclass(frozen=True)
class SolveRequest:
    arrival: float     # seconds after the start of the stream
    n_theta: int
    n_r: int
    p: int
    mach: float


def request_stream(n=64, seed=1807, mean_gap=0.25, grids=GRIDS, orders=ORDERS, mach=(0.1, 0.5)):
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(mean_gap, size=n)
    gi = rng.integers(0, len(grids), size=n)
    pi = rng.integers(0, len(orders), size=n)
    ma = rng.uniform(mach[0], mach[1], size=n)
    t = np.cumsum(gaps) - gaps[0]   # the first request arrives at t = 0
    return [SolveRequest(float(t[k]), grids[gi[k]][0], grids[gi[k]][1], orders[pi[k]], float(ma[k]))
            for k in range(n)]
