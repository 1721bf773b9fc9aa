"""The EXP1 step that allocates nothing (emg_exp1_step_noalloc) against emg_exp1_step.

The no-allocation variant serves callers that may not call cudaMalloc while they run
(their device memory comes from their own pool, or they issue work during stream
capture); it keeps its Krylov work arrays in one fixed device array.  It must give the
same result as the context-based step, call after call, although every call reuses the
array the previous call left behind.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from oracle import emg as oemg
from oracle.dg import DG
from tests.helpers import perturbed_state, rel_err
from workloads import ogrid

pytestmark = pytest.mark.gpu

TOL = 1e-12


def test_noalloc_exp1_matches_context_exp1_twice():
    import torch

    import paper_1807_01151_gb300 as pkg
    from paper_1807_01151_gb300._lib import exp1_step_noalloc

    torch.cuda.set_device(0)
    desc = ogrid(32, 16)
    s = pkg.Solver(desc, p_max=2)
    dg = DG(desc, 2)
    dev = torch.device("cuda", 0)
    for call, seed in enumerate((11, 12)):
        u = perturbed_state(dg, seed=seed, amp=0.02)
        u0 = np.ascontiguousarray(u[:, :, :1])
        dt = np.ascontiguousarray(oemg.dtau(dg, 2, u, 100.0) * 3.0)
        ref, k_ref = s.exp1_step(u0, dt)                          # context entry point
        diag, off, nbr = s.jacobian_p0(u0)
        r0 = s.residual(0, u0)
        t = {name: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
             for name, a in dict(diag=diag, off=off, nbr=nbr, r0=r0, dt=dt, u0=u0).items()}
        out = torch.full_like(t["u0"], float("nan"))
        k = exp1_step_noalloc(2, t["diag"], t["off"], t["nbr"], t["r0"], t["dt"], t["u0"], out, krylov_m=30)
        got = out.cpu().numpy()
        assert k == k_ref, (call, k, k_ref)
        assert np.isfinite(got).all()
        assert rel_err(got - u0, ref - u0) < TOL, (call, rel_err(got - u0, ref - u0))
    s.close()


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch

    from paper_1807_01151_gb300._lib import EmgError, exp1_step_noalloc

    dev = torch.device("cuda", 0)
    E = 8193
    z = lambda *shape: torch.zeros(shape, dtype=torch.float64, device=dev)   # noqa: E731
    nbr = torch.zeros((E, 4), dtype=torch.int64, device=dev)
    with pytest.raises(EmgError) as ei:
        exp1_step_noalloc(2, z(E, 5, 5), z(E, 4, 5, 5), nbr, z(E, 5, 1), z(E), z(E, 5, 1), z(E, 5, 1))
    assert ei.value.status == 1
