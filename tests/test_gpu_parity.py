"""GPU path (C ABI, libemg.so) against the CPU oracle, element by element.

Tolerances: the oracle and the kernels evaluate the same FP64 formulas in different
orders, so single-kernel results agree to a few ulps times the condition of the step;
the target tolerances are 1e-11 (relative) per V-cycle and 1e-9 on the converged state.
"""
import os

import numpy as np
import pytest

from oracle import emg as oemg
from oracle.basis import exponents
from oracle.dg import DG
from tests.helpers import perturbed_state, rel_err
from workloads import BC_FARFIELD, cubed_sphere_shell, ogrid

pytestmark = pytest.mark.gpu

TOL_KERNEL = 1e-12
GOLDEN_PATH = os.path.join(os.path.dirname(__file__), "golden", "cyl32x16_p2_steady.npz")
TOL_CYCLE = 1e-11


@pytest.fixture(scope="module")
def lib():
    import paper_1807_01151_gb300 as pkg
    return pkg


def make(lib, desc, p, **kw):
    return lib.Solver(desc, p_max=p, **kw), DG(desc, p, mach=kw.get("mach", 0.3),
                                               alpha_deg=kw.get("alpha_deg", 0.0))


CASES = [
    ("cyl32x16_p2", lambda: ogrid(32, 16), 2),          # the cylinder stand-in of the 32 x 16 case
    ("ogrid5x3_p4_ragged", lambda: ogrid(5, 3), 4),     # E = 15: ragged element tiles
    ("sphere6x2x2x2_p3", lambda: cubed_sphere_shell(2, 2), 3),
]


@pytest.mark.parametrize("name,mk,p", CASES)
def test_geometry_and_residual_all_levels(lib, name, mk, p):
    desc = mk()
    s, dg = make(lib, desc, p)
    vol, h = s.element_geometry()
    assert rel_err(vol, dg.mesh.vol) < 1e-13
    assert rel_err(h, dg.mesh.h) < 1e-13
    u = perturbed_state(dg, amp=0.05)
    for lev in range(p + 1):
        ul = np.ascontiguousarray(u[:, :, :dg.N(lev)])
        Rg = s.residual(lev, ul)
        Ro = dg.residual(lev, ul)
        assert rel_err(Rg, Ro) < TOL_KERNEL, (name, lev, rel_err(Rg, Ro))
    s.close()


def test_freestream_residual_is_zero_on_farfield_annulus(lib):
    desc = ogrid(12, 4, inner_bc=BC_FARFIELD)
    s = lib.Solver(desc, p_max=3, mach=0.4, alpha_deg=20.0)
    u = s.get_state()
    for lev in range(4):
        R = s.residual(lev, np.ascontiguousarray(u[:, :, :s.n_modes(lev)]))
        assert np.abs(R).max() < 1e-13 * np.abs(u).max()
    s.close()


@pytest.mark.parametrize("name,mk,p", CASES)
def test_diag_blocks(lib, name, mk, p):
    desc = mk()
    s, dg = make(lib, desc, p)
    u = perturbed_state(dg, amp=0.05)
    for lev in range(p, -1, -1):
        ul = np.ascontiguousarray(u[:, :, :dg.N(lev)])
        Dg = s.jacobian_diag(lev, ul)
        Do = dg.diag_blocks(lev, ul)
        assert rel_err(Dg, Do) < 1e-11, (name, lev, rel_err(Dg, Do))
    s.close()


@pytest.mark.parametrize("name,mk,p", CASES[:2])
def test_prk_step(lib, name, mk, p):
    desc = mk()
    s, dg = make(lib, desc, p)
    # a random state is far from any flow: keep the step moderate so that both sides stay
    # physical (CFL 10 already drives the 5 x 3 p = 4 case to negative pressures)
    u = perturbed_state(dg, amp=0.002)
    rng = np.random.default_rng(5)
    for lev in range(p, 0, -1):
        ul = np.ascontiguousarray(u[:, :, :dg.N(lev)])
        tau = 1e-6 * rng.standard_normal(ul.shape) * np.sqrt(dg.mesh.vol)[:, None, None]
        for cfl, tu in ((1.0, None), (3.0, tau)):
            ug = s.prk_step(lev, ul, tau=tu, cfl=cfl)
            D = dg.diag_blocks(lev, ul)
            dt = oemg.dtau(dg, lev, ul, cfl)
            P = np.eye(D.shape[-1])[None] / dt[:, None, None] - D
            tt = tu if tu is not None else 0.0
            uo = oemg.prk_step(lambda w: dg.residual(lev, w) + tt, P, ul)
            assert np.isfinite(uo).all() and np.isfinite(ug).all()
            assert rel_err(ug - ul, uo - ul) < TOL_CYCLE, (lev, cfl, rel_err(ug - ul, uo - ul))
    s.close()


@pytest.mark.parametrize("name,mk,p", CASES)
def test_p0_block_jacobian(lib, name, mk, p):
    desc = mk()
    s, dg = make(lib, desc, p)
    u0 = np.ascontiguousarray(perturbed_state(dg, amp=0.05)[:, :, :1])
    dgg, og, ng = s.jacobian_p0(u0)
    do, oo, no = dg.p0_blocks(u0)
    assert np.array_equal(ng, no)
    assert rel_err(dgg, do) < TOL_KERNEL
    assert rel_err(og, oo) < TOL_KERNEL
    s.close()


def test_exp1_step_fixed_dimension(lib):
    desc = ogrid(16, 8)
    s, dg = make(lib, desc, 1)
    u0 = np.ascontiguousarray(perturbed_state(dg, amp=0.05)[:, :, :1])
    rng = np.random.default_rng(3)
    tau0 = 1e-4 * rng.standard_normal(u0.shape)
    dt = oemg.dtau(dg, 1, perturbed_state(dg, amp=0.05), 100.0) * 2.0
    ug, kg = s.exp1_step(u0, dt, tau0)
    uo, ko = oemg.exp1_step(dg, u0, tau0, dt, oemg.Options())
    assert kg == ko == 30
    assert rel_err(ug - u0, uo - u0) < TOL_CYCLE, rel_err(ug - u0, uo - u0)


def test_exp1_step_with_float32_krylov(lib):
    """The Arnoldi process in float32 arithmetic (krylov_f32): the same EXP1 step as the FP64
    oracle to float32 accuracy.  Every basis vector carries rounding of order u32 = 2^-24 per
    operation, compounded over m = 30 Gram-Schmidt steps with reorthogonalisation; the step
    (a combination of the basis with phi_1 coefficients) is asserted within 1e-4 relative, and
    above FP64 error (it is float32 arithmetic)."""
    desc = ogrid(16, 8)
    s = lib.Solver(desc, p_max=1, krylov_f32=1)
    dg = DG(desc, 1)
    u0 = np.ascontiguousarray(perturbed_state(dg, amp=0.05)[:, :, :1])
    rng = np.random.default_rng(3)
    tau0 = 1e-4 * rng.standard_normal(u0.shape)
    dt = oemg.dtau(dg, 1, perturbed_state(dg, amp=0.05), 100.0) * 2.0
    ug, kg = s.exp1_step(u0, dt, tau0)
    uo, ko = oemg.exp1_step(dg, u0, tau0, dt, oemg.Options())
    assert kg == ko == 30
    e = rel_err(ug - u0, uo - u0)
    assert 1e-12 < e < 1e-4, e
    s.close()


@pytest.mark.skipif(not os.path.exists(GOLDEN_PATH), reason="golden file not generated")
def test_float32_krylov_converged_state_matches_fp64_oracle(lib):
    """float32 block factors and a float32 Krylov basis change only the smoother and the
    coarse correction: the converged state is the FP64 fixed point R = 0."""
    g = np.load(GOLDEN_PATH)
    s = lib.Solver(ogrid(32, 16), p_max=2, prec=1, krylov_f32=1)
    rep = s.solve_steady(drop=1e-10, max_cycles=int(g["cycles"]) + 400)
    assert rep["converged"]
    assert rel_err(s.get_state(), g["u"]) < 1e-9, rel_err(s.get_state(), g["u"])
    s.close()


def test_exp1_happy_breakdown_matches_dense(lib):
    """Tiny mesh, K0 = 20 < m: the Krylov space is exhausted and EXP1 equals the dense
    phi_1(DT J) DT R."""
    import scipy.linalg
    desc = ogrid(4, 1)
    s, dg = make(lib, desc, 0)
    u0 = np.ascontiguousarray(perturbed_state(dg, amp=0.05))
    dt = oemg.dtau(dg, 0, u0, 50.0)
    ug, kg = s.exp1_step(u0, dt)
    J = dg.full_jacobian(0, u0)
    A = np.repeat(dt, 5)[:, None] * J
    N = np.repeat(dt, 5) * dg.residual(0, u0).ravel()
    ref = np.linalg.solve(A, (scipy.linalg.expm(A) - np.eye(len(N))) @ N)
    assert kg <= 20
    assert rel_err((ug - u0).ravel(), ref) < 1e-10


@pytest.mark.parametrize("p", [1, 2])
def test_vcycle_parity(lib, p):
    desc = ogrid(32, 16)
    s, dg = make(lib, desc, p)
    u = perturbed_state(dg, amp=0.02)
    s.set_state(np.ascontiguousarray(u))
    opts = oemg.Options()
    uo = u
    for n in (1, 2):
        info = s.vcycle()
        uo, oi = oemg.vcycle(dg, uo, n, opts)
        ug = s.get_state()
        assert abs(info["res_rho"] - oi.res) <= 1e-12 * oi.res
        assert abs(info["cfl"] - oi.cfl) <= 1e-12 * oi.cfl
        assert info["krylov_dim"] == oi.krylov_dim
        assert rel_err(ug, uo) < TOL_CYCLE, (n, rel_err(ug, uo))
        s.set_state(np.ascontiguousarray(uo))     # next cycle from the identical state
        s.set_cycle(n + 1, opts.res_ref)
    s.close()


def test_vcycle_3d_parity(lib):
    desc = cubed_sphere_shell(2, 2)
    s, dg = make(lib, desc, 2)
    u = perturbed_state(dg, amp=0.02)
    s.set_state(np.ascontiguousarray(u))
    s.vcycle()
    uo, _ = oemg.vcycle(dg, u, 1)
    assert rel_err(s.get_state(), uo) < TOL_CYCLE


def test_p0_only_vcycle(lib):
    desc = ogrid(8, 4)
    s, dg = make(lib, desc, 0)
    u = perturbed_state(dg, amp=0.02)
    s.set_state(np.ascontiguousarray(u))
    s.vcycle()
    uo, _ = oemg.vcycle(dg, u, 1)
    assert rel_err(s.get_state(), uo) < TOL_CYCLE


GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cyl32x16_p2_steady.npz")


@pytest.mark.skipif(not os.path.exists(GOLDEN), reason="golden file not generated")
def test_converged_state_matches_oracle(lib):
    g = np.load(GOLDEN)
    s = lib.Solver(ogrid(32, 16), p_max=2)
    rep = s.solve_steady(drop=1e-10, max_cycles=int(g["cycles"]) + 200)
    assert rep["converged"]
    u = s.get_state()
    assert rel_err(u, g["u"]) < 1e-9, rel_err(u, g["u"])


def test_bounded_wait_times_out_and_context_survives(lib):
    desc = ogrid(8, 2)
    s = lib.Solver(desc, p_max=1)
    u = s.get_state()
    R0 = s.residual(1, u)
    with pytest.raises(lib.EmgError) as ei:
        s._check(s.lib.emg_selftest_wait_timeout(s.h))
    assert ei.value.status == 7
    # the context is still usable and the flag was cleared
    assert np.array_equal(s.residual(1, u), R0)
    info = s.vcycle()
    assert np.isfinite(info["res_rho"])
    s.close()


def test_fp32_block_prk_step_close_to_oracle(lib):
    """FP32 blocks change only the preconditioner: the PRK update agrees with the FP64
    oracle to float accuracy."""
    desc = ogrid(32, 16)
    s = lib.Solver(desc, p_max=2, prec=1)
    dg = DG(desc, 2)
    u = np.ascontiguousarray(perturbed_state(dg, amp=0.002))
    ug = s.prk_step(2, u, cfl=3.0)
    D = dg.diag_blocks(2, u)
    dt = oemg.dtau(dg, 2, u, 3.0)
    P = np.eye(D.shape[-1])[None] / dt[:, None, None] - D
    uo = oemg.prk_step(lambda w: dg.residual(2, w), P, u)
    e = rel_err(ug - u, uo - u)
    assert 1e-12 < e < 1e-4, e
    s.close()


@pytest.mark.skipif(not os.path.exists(GOLDEN), reason="golden file not generated")
def test_fp32_block_converged_state_matches_fp64_oracle(lib):
    """The fixed point R = 0 does not depend on the preconditioner (Eq. prk_scalar)."""
    g = np.load(GOLDEN)
    s = lib.Solver(ogrid(32, 16), p_max=2, prec=1)
    rep = s.solve_steady(drop=1e-10, max_cycles=int(g["cycles"]) + 300)
    assert rep["converged"]
    assert rel_err(s.get_state(), g["u"]) < 1e-9, rel_err(s.get_state(), g["u"])
    s.close()


def test_error_paths(lib):
    desc = ogrid(8, 2)
    s = lib.Solver(desc, p_max=1)
    u = s.get_state()
    bad = u.copy()
    bad[3, 0, 0] = np.nan
    with pytest.raises(lib.EmgError) as ei:
        s.set_state(bad)
    assert ei.value.status == 4
    with pytest.raises(lib.EmgError):
        s.residual(5, u)
    s.close()
    with pytest.raises(lib.EmgError) as ei:
        lib.Solver(desc, p_max=7)
    assert ei.value.status == 1


# ---- full-size cylinder workload (128 x 64, p = 4): the configuration bench.py times ----

@pytest.fixture(scope="module")
def c2(lib):
    desc = ogrid(128, 64)
    s = lib.Solver(desc, p_max=4)
    dg = DG(desc, 4)
    return s, dg


def test_fullsize_residual(c2):
    s, dg = c2
    u = perturbed_state(dg, amp=0.02)
    for lev in (4, 2, 0):
        ul = np.ascontiguousarray(u[:, :, :dg.N(lev)])
        assert rel_err(s.residual(lev, ul), dg.residual(lev, ul)) < TOL_KERNEL


def test_fullsize_diag_block_sampled_columns(c2):
    """Sampled columns of every block of one colour class (one complex-step residual each)."""
    s, dg = c2
    u = perturbed_state(dg, amp=0.02)
    Dg = s.jacobian_diag(4, np.ascontiguousarray(u))
    col = dg.mesh.coloring(1)
    mask = col == 0
    n = dg.N(4)
    for (a, j) in ((0, 0), (1, 3), (4, 14), (2, 7)):
        uc = u.astype(complex)
        uc[mask, a, j] += 1e-30j
        Ri = dg.residual(4, uc).imag / 1e-30
        ref = Ri[mask].reshape(mask.sum(), -1)
        got = Dg[mask][:, :, a * n + j]
        assert rel_err(got, ref) < 1e-11


def test_fullsize_exp1(c2):
    s, dg = c2
    u0 = np.ascontiguousarray(perturbed_state(dg, amp=0.02)[:, :, :1])
    dt = oemg.dtau(dg, 4, perturbed_state(dg, amp=0.02), 100.0) * 5.0
    ug, kg = s.exp1_step(u0, dt)
    uo, ko = oemg.exp1_step(dg, u0, np.zeros_like(u0), dt, oemg.Options())
    assert kg == ko
    assert rel_err(ug - u0, uo - u0) < TOL_CYCLE


def test_fullsize_vcycles_keep_mirror_symmetry(c2):
    """Property at any size: the O-grid and the flow (alpha = 0) are symmetric about y = 0."""
    s, dg = c2
    s.set_state(None)
    for _ in range(3):
        info = s.vcycle()
        assert np.isfinite(info["res_rho"])
    u = s.get_state()
    nt, nr = 128, 64
    perm = np.array([l * nt + (nt - 1 - k) % nt for l in range(nr) for k in range(nt)])
    sgn = np.array([1.0, 1.0, -1.0, 1.0, 1.0])[:, None] * ((-1.0) ** exponents(2, 4)[:, 1])[None, :]
    assert np.abs(u[perm] * sgn[None] - u).max() < 1e-11 * np.abs(u).max()


@pytest.mark.gpu
def test_graph_replayed_cycles_are_bitwise_the_kernel_by_kernel_cycles():
    """The V-cycle body captured as a CUDA graph runs the same kernels as the direct
    launches: the states after several cycles are identical bit for bit, and so are the
    launch counts."""
    from paper_1807_01151_gb300 import Solver
    from workloads import ogrid
    out = {}
    for g in (0, 1):
        for prec in (0, 1):
            s = Solver(ogrid(16, 8), p_max=3, prec=prec, use_graph=g)
            l0 = s.launch_count
            infos = [s.vcycle() for _ in range(6)]
            out[g, prec] = (s.get_state(), [i["cfl"] for i in infos], s.launch_count - l0, s.graph_kernels)
            s.close()
    for prec in (0, 1):
        np.testing.assert_array_equal(out[0, prec][0], out[1, prec][0])
        assert out[0, prec][1] == out[1, prec][1]            # CFL_n from the device cycle counter
        assert out[0, prec][2] == out[1, prec][2]
        assert out[0, prec][3] == 0 and out[1, prec][3] > 50


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 1])
def test_side_stream_overlap_is_bitwise_the_serial_order(prec):
    """The residuals and forcings run on a second stream beside each block build (graph branches
    or direct launches) give the same bits as the one-stream order the event profiler keeps."""
    from paper_1807_01151_gb300 import Solver
    from workloads import ogrid
    out = []
    for serial, g in ((1, 0), (0, 0), (0, 1)):
        s = Solver(ogrid(16, 8), p_max=4, prec=prec, use_graph=g, pre_smooth=2)
        if serial:
            s.profile(True)
        for _ in range(5):
            s.vcycle(info=False)
        out.append(s.get_state())
        s.close()
    np.testing.assert_array_equal(out[0], out[1])
    np.testing.assert_array_equal(out[0], out[2])


@pytest.mark.gpu
def test_tuned_kernel_variants_give_bitwise_the_same_cycles():
    """The tuner only picks among variants that compute identically."""
    from paper_1807_01151_gb300 import Solver
    from workloads import ogrid
    out, notes = [], []
    for at in (0, 1):
        s = Solver(ogrid(16, 8), p_max=4, prec=1, autotune=at)
        for _ in range(4):
            s.vcycle(info=False)
        out.append(s.get_state())
        notes.append(s.tuning)
        s.close()
    np.testing.assert_array_equal(out[0], out[1])
    assert notes[0] == "" and "gj B=75" in notes[1] and "gj B=15" in notes[1]


@pytest.mark.gpu
def test_barrier_free_arnoldi_is_bitwise_the_persistent_kernel():
    """The Arnoldi process as plain kernels (no grid barrier) and as one cooperative
    persistent kernel: same blocks, same arithmetic, bitwise the same cycles; also when
    the process stops early at happy breakdown (4x1 O-grid at p = 0, K0 = 20 < m), and with
    the float32 Krylov basis."""
    from paper_1807_01151_gb300 import Solver
    from workloads import ogrid
    for desc, p, prec, kf in ((ogrid(16, 8), 3, 1, 0), (ogrid(16, 8), 2, 0, 0), (ogrid(4, 1), 0, 0, 0),
                              (ogrid(16, 8), 3, 1, 1), (ogrid(4, 1), 0, 0, 1)):
        out = []
        for coop in (1, 0):
            s = Solver(desc, p_max=p, prec=prec, coop_krylov=coop, krylov_f32=kf)
            infos = [s.vcycle() for _ in range(5)]
            out.append((s.get_state(), [(i["krylov_dim"], i["cfl"], i["res_rho"]) for i in infos]))
            s.close()
        np.testing.assert_array_equal(out[0][0], out[1][0])
        assert out[0][1] == out[1][1]
        if p == 0:
            assert out[0][1][0][0] <= 20         # breakdown: the space is exhausted
