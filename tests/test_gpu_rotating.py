"""The rotating frame (Eq. euler with omega != 0) on the GPU against the oracle: residuals at every
level, the element-diagonal and p = 0 Jacobian blocks, the float32 block operator and V-cycles,
in 2-D (rotation about z) and 3-D."""
import numpy as np
import pytest

from oracle import emg as oemg
from oracle.dg import DG
from tests.helpers import perturbed_state, rel_err
from workloads import cubed_sphere_shell, ogrid

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
CASES = [
    ("cyl8x4_p3", lambda: ogrid(8, 4), 3, (0.0, 0.0, 0.2)),
    ("sphere6x2x2x2_p2", lambda: cubed_sphere_shell(2, 2), 2, (0.05, -0.08, 0.1)),
]


def make(desc, p, omega, **kw):
    import paper_1807_01151_gb300 as pkg
    return pkg.Solver(desc, p_max=p, omega=omega, **kw), DG(desc, p, omega=omega)


@pytest.mark.parametrize("name,mk,p,om", CASES)
def test_rotating_residual_and_blocks(name, mk, p, om):
    desc = mk()
    s, dg = make(desc, p, om)
    u = perturbed_state(dg, amp=0.05)
    for lev in range(p + 1):
        ul = np.ascontiguousarray(u[:, :, :dg.N(lev)])
        Rg, Ro = s.residual(lev, ul), dg.residual(lev, ul)
        assert rel_err(Rg, Ro) < 1e-12, (lev, rel_err(Rg, Ro))
        Dg, Do = s.jacobian_diag(lev, ul), dg.diag_blocks(lev, ul)
        assert rel_err(Dg, Do) < 1e-11, (lev, rel_err(Dg, Do))
    u0 = np.ascontiguousarray(u[:, :, :1])
    dgg, og, ng = s.jacobian_p0(u0)
    do, oo, no = dg.p0_blocks(u0)
    assert np.array_equal(ng, no)
    assert rel_err(dgg, do) < 1e-12 and rel_err(og, oo) < 1e-12
    s.close()
    # the same residual without rotation differs (the frame terms are exercised)
    s0 = make(desc, p, (0.0, 0.0, 0.0))[0]
    assert rel_err(s0.residual(p, np.ascontiguousarray(u)), Ro) > 1e-4
    s0.close()


@pytest.mark.parametrize("name,mk,p,om", CASES)
@pytest.mark.parametrize("kernels", [1, 2, 3])
def test_rotating_float32_block_operator(name, mk, p, om, kernels):
    """The float32 block forms (tensor-core, SIMT and earlier SIMT) assemble the rotating frame's
    P_e = I/dtau - D_e within the float32 bound of the other block tests, 16 K u32 |P_e|_max
    (K = Q + 2d QF terms per entry)."""
    desc = mk()
    s, dg = make(desc, p, om, prec=1, block_kernels=kernels)
    u = perturbed_state(dg, amp=0.002)
    cfl = 3.0
    D = dg.diag_blocks(p, u)
    dt = oemg.dtau(dg, p, u, cfl)
    P = np.eye(D.shape[-1])[None] / dt[:, None, None] - D
    Pg = s.block_operator(p, u, cfl=cfl, which=0)
    s.close()
    q = p + 2
    K = q ** dg.dim + 2 * dg.dim * q ** (dg.dim - 1)
    err = np.abs(Pg - P).max(axis=(1, 2))
    assert np.all(err <= 16 * K * U32 * np.abs(P).max(axis=(1, 2))), err.max()


@pytest.mark.parametrize("name,mk,p,om", CASES)
def test_rotating_vcycles(name, mk, p, om):
    """Two V-cycles (FP64 form) from identical inputs, Sec. 2.3, against the oracle."""
    desc = mk()
    s, dg = make(desc, p, om)
    u = perturbed_state(dg, amp=0.02)
    s.set_state(np.ascontiguousarray(u))
    opts = oemg.Options()
    uo = u
    for n in (1, 2):
        info = s.vcycle()
        uo, oi = oemg.vcycle(dg, uo, n, opts)
        assert info["krylov_dim"] == oi.krylov_dim
        assert rel_err(s.get_state(), uo) < 1e-11, (n, rel_err(s.get_state(), uo))
        s.set_state(np.ascontiguousarray(uo))
        s.set_cycle(n + 1, opts.res_ref)
    s.close()


def test_rotation_axis_must_be_z_in_2d():
    import paper_1807_01151_gb300 as pkg
    with pytest.raises(pkg.EmgError) as ei:
        pkg.Solver(ogrid(8, 2), p_max=1, omega=(0.0, 0.1, 0.0))
    assert ei.value.status == 1
