"""Write tests/golden/cyl32x16_p2_steady.npz with the oracle only.

The cylinder stand-in (O-grid 32 x 16, r in [0.5, 20], Ma = 0.3, alpha = 0, p = 2) is
solved by the oracle's FAS V-cycle from the free stream until the density residual of
Eq. cfl has dropped by 1e-10; the converged modal state and the residual history are
stored.  Run:  python tests/golden/make_golden.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import emg  # noqa: E402
from oracle.dg import DG  # noqa: E402
from workloads import ogrid  # noqa: E402


def main():
    dg = DG(ogrid(32, 16), 2, mach=0.3)
    u = dg.freestream_state()
    hist = []
    t = time.time()
    u, cycles, ok = emg.solve_steady(dg, u, drop=1e-10, max_cycles=2000, history=hist)
    print(f"converged={ok} cycles={cycles} time={time.time() - t:.0f}s final drop={hist[-1] / hist[0]:.3e}")
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cyl32x16_p2_steady.npz")
    np.savez_compressed(out, u=u, history=np.array(hist), cycles=cycles, converged=ok)


if __name__ == "__main__":
    main()
