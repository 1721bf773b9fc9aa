"""The EXP1 step that allocates nothing (emg_exp1_step_noalloc) against emg_exp1_step.

The no-allocation variant serves callers that may not call cudaMalloc once they are running:
their device memory comes from their own pool (a caching allocator that already holds the
free memory), or their loop may not take the device-wide synchronisation that cudaMalloc and
cudaFree can cause.  It keeps its Krylov work arrays in one fixed device array.  It must give
the same result as the context-based step, call after call, although every call reuses the
array the previous call left behind; it must reject sizes beyond the array and neighbour
indices out of range before anything reads through them.  This file is collected last on
purpose.
"""
import numpy as np
import pytest

from oracle import emg as oemg
from oracle.dg import DG
from tests.helpers import perturbed_state, rel_err
from workloads import cubed_sphere_shell, ogrid

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _inputs(s, dg, seed, dev, torch):
    p = dg.p_max
    u = perturbed_state(dg, seed=seed, amp=0.02)
    u0 = np.ascontiguousarray(u[:, :, :1])
    dt = np.ascontiguousarray(oemg.dtau(dg, p, u, 100.0) * 3.0)
    diag, off, nbr = s.jacobian_p0(u0)
    r0 = s.residual(0, u0)
    t = {name: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
         for name, a in dict(diag=diag, off=off, nbr=nbr, r0=r0, dt=dt, u0=u0).items()}
    return u0, dt, t


@pytest.mark.parametrize("mk,p,m,on_stream", [
    (lambda: ogrid(32, 16), 2, 30, False),            # 2-D, legacy default stream
    (lambda: cubed_sphere_shell(4, 3), 1, 40, True),  # 3-D (six faces), a torch stream, m at its limit
])
def test_noalloc_exp1_matches_context_exp1_twice(mk, p, m, on_stream):
    import torch

    import paper_1807_01151_gb300 as pkg
    from paper_1807_01151_gb300._lib import exp1_step_noalloc

    torch.cuda.set_device(0)
    desc = mk()
    s = pkg.Solver(desc, p_max=p, krylov_m=m)
    dg = DG(desc, p)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream() if on_stream else None
    for call, seed in enumerate((11, 12)):
        u0, dt, t = _inputs(s, dg, seed, dev, torch)
        ref, k_ref = s.exp1_step(u0, dt)                          # context entry point
        out = torch.full_like(t["u0"], float("nan"))
        torch.cuda.synchronize()
        k = exp1_step_noalloc(dg.dim, t["diag"], t["off"], t["nbr"], t["r0"], t["dt"], t["u0"], out,
                              krylov_m=m, stream=stream.cuda_stream if stream else None)
        torch.cuda.synchronize()
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
    with pytest.raises(EmgError) as ei:
        exp1_step_noalloc(2, z(8, 5, 5), z(8, 4, 5, 5), nbr[:8], z(8, 5, 1), z(8), z(8, 5, 1), z(8, 5, 1),
                          krylov_m=41)
    assert ei.value.status == 1


def test_noalloc_rejects_neighbour_indices_out_of_range():
    """A neighbour index outside [-1, n_elems) is caught by the packing kernel (which
    substitutes -1 so that nothing out of range is read) and the call returns EMG_ERR_ARG
    before the Krylov step; the next valid call is unaffected."""
    import torch

    import paper_1807_01151_gb300 as pkg
    from paper_1807_01151_gb300._lib import EmgError, exp1_step_noalloc

    desc = ogrid(16, 8)
    s = pkg.Solver(desc, p_max=1)
    dg = DG(desc, 1)
    dev = torch.device("cuda", 0)
    u0, dt, t = _inputs(s, dg, 5, dev, torch)
    out = torch.zeros_like(t["u0"])
    for bad in (dg.E, -2, 1 << 40):
        nb = t["nbr"].clone()
        nb[3, 1] = bad
        with pytest.raises(EmgError) as ei:
            exp1_step_noalloc(2, t["diag"], t["off"], nb, t["r0"], t["dt"], t["u0"], out)
        assert ei.value.status == 1, bad
    ref, k_ref = s.exp1_step(u0, dt)
    k = exp1_step_noalloc(2, t["diag"], t["off"], t["nbr"], t["r0"], t["dt"], t["u0"], out)
    assert k == k_ref
    assert rel_err(out.cpu().numpy() - u0, ref - u0) < TOL
    s.close()


def test_noalloc_alternating_krylov_dimensions():
    """Calls with different m reuse the array with a different row stride of the Hessenberg
    matrix; each must still equal the context step of the same m."""
    import torch

    import paper_1807_01151_gb300 as pkg
    from paper_1807_01151_gb300._lib import exp1_step_noalloc

    desc = ogrid(16, 8)
    dg = DG(desc, 1)
    dev = torch.device("cuda", 0)
    solvers = {m: pkg.Solver(desc, p_max=1, krylov_m=m) for m in (40, 30, 12)}
    for call, m in enumerate((40, 30, 12, 40)):
        s = solvers[m]
        u0, dt, t = _inputs(s, dg, 20 + call, dev, torch)
        ref, k_ref = s.exp1_step(u0, dt)
        out = torch.full_like(t["u0"], float("nan"))
        k = exp1_step_noalloc(2, t["diag"], t["off"], t["nbr"], t["r0"], t["dt"], t["u0"], out, krylov_m=m)
        assert k == k_ref, (m, k, k_ref)
        assert rel_err(out.cpu().numpy() - u0, ref - u0) < TOL, (m, rel_err(out.cpu().numpy() - u0, ref - u0))
    for s in solvers.values():
        s.close()
