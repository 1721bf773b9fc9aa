"""GPU against the oracle on the float32 block path at the block sizes the benchmark and the
sphere cases run (B = 75, 100, 175), on V-cycles at p_max = 4 (2-D) and 3 (3-D), and on the
variants of the method: a global EXP1 step, frozen block factors, the Krylov tolerance of
Sec. 5 and symmetry planes.

Float32 error bounds (u32 = 2^-24), per element e:
* assembly: every entry of P_e is a sum of K products of rounded inputs (K = Q + 2d QF
  quadrature terms), so |P^_e - P_e|_max <= c_a K u32 |P_e|_max with c_a = 16 allowing for
  the rounding of the flux Jacobian entries and of I/dtau;
* inverse: to first order ||X^ - P^-1|| / ||P^-1|| <= kappa_2(P_e) (eps_e + B u32), eps_e the
  measured relative assembly error and B u32 the Gauss-Jordan rounding; asserted with a
  factor 4;
* PRK step (four stages): the update differs from the FP64 one by at most
  8 max_e kappa_2(P_e) (max_e eps_e + B u32), relative to the update.
"""
import numpy as np
import pytest

from oracle import emg as oemg
from oracle.dg import DG
from tests.helpers import perturbed_state, rel_err
from workloads import cubed_sphere_shell, half_mesh, ogrid

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
TOL_CYCLE = 1e-11

BLOCK_CASES = [
    ("cyl8x4_p4_B75", lambda: ogrid(8, 4), 4),
    ("sphere6x2x2x2_p3_B100", lambda: cubed_sphere_shell(2, 2), 3),
    ("sphere6x1x1x2_p4_B175", lambda: cubed_sphere_shell(1, 2), 4),
]

_oracle_cache = {}


def oracle_case(name, mk, p):
    """(desc, DG, u, D) with the oracle's diagonal blocks of the top level (computed once)."""
    if name not in _oracle_cache:
        desc = mk()
        dg = DG(desc, p)
        u = perturbed_state(dg, amp=0.002)
        _oracle_cache[name] = (desc, dg, u, dg.diag_blocks(p, u))
    return _oracle_cache[name]


def n_terms(dim, p):
    q = p + 2
    return q ** dim + 2 * dim * q ** (dim - 1)


@pytest.mark.parametrize("name,mk,p", BLOCK_CASES)
@pytest.mark.parametrize("cfl", [3.0, 100.0])
@pytest.mark.parametrize("kernels", [1, 2, 3])       # tensor-core, SIMT, SIMT unblocked inverse
def test_fp32_block_operator_and_inverse(name, mk, p, cfl, kernels):
    import paper_1807_01151_gb300 as pkg
    desc, dg, u, D = oracle_case(name, mk, p)
    s = pkg.Solver(desc, p_max=p, prec=1, block_kernels=kernels)
    B = D.shape[-1]
    dt = oemg.dtau(dg, p, u, cfl)
    P = np.eye(B)[None] / dt[:, None, None] - D
    Pg = s.block_operator(p, u, cfl=cfl, which=0)
    Xg = s.block_operator(p, u, cfl=cfl, which=1)
    s.close()
    K = n_terms(dg.dim, p)
    amax = np.abs(P).max(axis=(1, 2))
    err_a = np.abs(Pg - P).max(axis=(1, 2))
    assert np.all(err_a > 0.0)                              # it is float32 arithmetic
    assert np.all(err_a <= 16 * K * U32 * amax), (err_a / (K * U32 * amax)).max()
    X = np.linalg.inv(P)
    kappa = np.linalg.cond(P)
    eps = np.linalg.norm(Pg - P, ord=2, axis=(1, 2)) / np.linalg.norm(P, ord=2, axis=(1, 2))
    err_x = np.linalg.norm(Xg - X, ord=2, axis=(1, 2)) / np.linalg.norm(X, ord=2, axis=(1, 2))
    bound = 4 * kappa * (eps + B * U32)
    assert np.all(err_x <= bound), (err_x / bound).max()


@pytest.mark.parametrize("name,mk,p", BLOCK_CASES)
@pytest.mark.parametrize("kernels", [1, 2, 3])
def test_fp32_block_prk_step_at_block_size(name, mk, p, kernels):
    import paper_1807_01151_gb300 as pkg
    desc, dg, u, D = oracle_case(name, mk, p)
    cfl = 3.0
    s = pkg.Solver(desc, p_max=p, prec=1, block_kernels=kernels)
    ug = s.prk_step(p, u, cfl=cfl)
    Pg = s.block_operator(p, u, cfl=cfl, which=0)
    s.close()
    B = D.shape[-1]
    dt = oemg.dtau(dg, p, u, cfl)
    P = np.eye(B)[None] / dt[:, None, None] - D
    uo = oemg.prk_step(lambda w: dg.residual(p, w), P, u)
    eps = (np.linalg.norm(Pg - P, ord=2, axis=(1, 2)) / np.linalg.norm(P, ord=2, axis=(1, 2))).max()
    bound = 8 * np.linalg.cond(P).max() * (eps + B * U32)
    e = rel_err(ug - u, uo - u)
    assert 1e-12 < e <= bound, (e, bound)


LEVEL_CASES = [
    ("cyl8x4_p4", lambda: ogrid(8, 4), 4),                      # B = 15, 30, 50, 75
    ("sphere6x2x2x2_p3", lambda: cubed_sphere_shell(2, 2), 3),  # B = 20, 50, 100
]


@pytest.mark.parametrize("name,mk,pmax", LEVEL_CASES)
@pytest.mark.parametrize("kernels", [2, 3])          # blocked and unblocked SIMT inverse
def test_fp32_inverse_at_every_level(name, mk, pmax, kernels):
    """The float32 Gauss-Jordan inverse alone, at every block size of the levels: against the
    FP64 inverse of the very float32 operator the kernel was given.  Gauss-Jordan elimination
    with partial pivoting is forward stable, ||X^ - X|| / ||X|| <= c B u32 kappa_2(P); asserted
    with c = 4 per element, and at least float32 error (it is float32 arithmetic)."""
    import paper_1807_01151_gb300 as pkg
    desc = mk()
    dg = DG(desc, pmax)
    u = perturbed_state(dg, amp=0.002)
    s = pkg.Solver(desc, p_max=pmax, prec=1, block_kernels=kernels)
    for p in range(1, pmax + 1):
        up = np.ascontiguousarray(u[:, :, :dg.N(p)])
        for cfl in (3.0, 100.0):
            Pg = s.block_operator(p, up, cfl=cfl, which=0).astype(np.float64)
            Xg = s.block_operator(p, up, cfl=cfl, which=1)
            B = Pg.shape[-1]
            X = np.linalg.inv(Pg)
            err = np.linalg.norm(Xg - X, ord=2, axis=(1, 2)) / np.linalg.norm(X, ord=2, axis=(1, 2))
            bound = 4 * np.linalg.cond(Pg) * B * U32
            assert np.all(err <= bound), (p, cfl, (err / bound).max())
            assert err.max() > 0.0
    s.close()


@pytest.mark.parametrize("name,mk,pmax", LEVEL_CASES + [("sphere6x1x1x2_p4", lambda: cubed_sphere_shell(1, 2), 4)])
def test_fp32_assembly_forms_are_bitwise_the_same(name, mk, pmax):
    """The register-blocked SIMT assembly (several b and j per thread) sums every entry's terms
    in the order of the one-row-per-thread form, and the face Jacobians differentiated one
    direction per thread equal the five-direction dual numbers' columns: bitwise the same
    blocks at every level (block_kernels 2 against the earlier forms, 3)."""
    import paper_1807_01151_gb300 as pkg
    desc = mk()
    dg = DG(desc, pmax)
    u = perturbed_state(dg, amp=0.002)
    out = []
    for bk in (2, 3):
        s = pkg.Solver(desc, p_max=pmax, prec=1, block_kernels=bk)
        out.append([s.block_operator(p, np.ascontiguousarray(u[:, :, :dg.N(p)]), cfl=3.0, which=0)
                    for p in range(1, pmax + 1)])
        s.close()
    for x, y in zip(*out):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("name,mk,p", BLOCK_CASES)
def test_bf16_block_operator(name, mk, p):
    """The BF16 form multiplies bfloat16 operands (8 significant bits, rounding 2^-9) with float32
    accumulation: each entry of P_e is a sum of K products whose operands carry relative errors
    up to 2^-9, so |P^_e - P_e|_max <= 4 K 2^-9 max_t |term| with the largest term bounded by
    the largest entry of the float32 block times the block's cancellation; asserted as a
    relative max-norm error of 2^-5 per element, and at least float32 error (it is not the
    float32 form)."""
    import paper_1807_01151_gb300 as pkg
    desc, dg, u, D = oracle_case(name, mk, p)
    cfl = 3.0
    B = D.shape[-1]
    dt = oemg.dtau(dg, p, u, cfl)
    P = np.eye(B)[None] / dt[:, None, None] - D
    s = pkg.Solver(desc, p_max=p, prec=2)
    Pg = s.block_operator(p, u, cfl=cfl, which=0)
    Xg = s.block_operator(p, u, cfl=cfl, which=1)
    s.close()
    amax = np.abs(P).max(axis=(1, 2))
    err = np.abs(Pg - P).max(axis=(1, 2)) / amax
    assert np.all(err <= 2.0 ** -5), err.max()
    assert err.max() > 16 * n_terms(dg.dim, p) * U32
    # its explicit inverse is the float32 inverse of the bf16-assembled block
    Xr = np.linalg.inv(Pg)
    rel = np.linalg.norm(Xg - Xr, ord=2, axis=(1, 2)) / np.linalg.norm(Xr, ord=2, axis=(1, 2))
    assert np.all(rel <= 4 * np.linalg.cond(Pg) * B * U32), rel.max()


@pytest.mark.parametrize("mk,p", [(lambda: ogrid(16, 8), 4), (lambda: cubed_sphere_shell(2, 2), 3)])
def test_vcycle_parity_at_the_highest_orders(mk, p):
    """Two FP64 V-cycles p_max -> 0 -> p_max with the tau forcing nested over every level
    (Sec. 2.3), each from the identical input state, against the oracle."""
    import paper_1807_01151_gb300 as pkg
    desc = mk()
    s = pkg.Solver(desc, p_max=p)
    dg = DG(desc, p)
    u = perturbed_state(dg, amp=0.01)
    s.set_state(np.ascontiguousarray(u))
    opts = oemg.Options()
    uo = u
    for n in (1, 2):
        info = s.vcycle()
        uo, oi = oemg.vcycle(dg, uo, n, opts)
        assert info["krylov_dim"] == oi.krylov_dim
        assert abs(info["cfl"] - oi.cfl) <= 1e-12 * oi.cfl
        assert rel_err(s.get_state(), uo) < TOL_CYCLE, (n, rel_err(s.get_state(), uo))
        s.set_state(np.ascontiguousarray(uo))
        s.set_cycle(n + 1, opts.res_ref)
    s.close()


def _cycles(pkg, desc, p, n_cycles, solver_kw, opts):
    s = pkg.Solver(desc, p_max=p, **solver_kw)
    dg = DG(desc, p)
    u = perturbed_state(dg, amp=0.01)
    s.set_state(np.ascontiguousarray(u))
    uo = u
    for n in range(1, n_cycles + 1):
        info = s.vcycle()
        uo, oi = oemg.vcycle(dg, uo, n, opts)
        assert info["krylov_dim"] == oi.krylov_dim, (n, info["krylov_dim"], oi.krylov_dim)
        assert rel_err(s.get_state(), uo) < TOL_CYCLE, (n, rel_err(s.get_state(), uo))
    s.close()


def test_global_exp1_step_vcycles():
    import paper_1807_01151_gb300 as pkg
    _cycles(pkg, ogrid(16, 8), 2, 2, dict(exp_dt_global=1), oemg.Options(exp_dt_global=True))


@pytest.mark.parametrize("use_graph", [1, 0])
def test_frozen_block_factors_vcycles(use_graph):
    """jac_freeze = 2: cycle 1 assembles and factors, cycle 2 reuses them, cycle 3 assembles
    again; every cycle against the oracle, continuing from the GPU's own state."""
    import paper_1807_01151_gb300 as pkg
    _cycles(pkg, ogrid(16, 8), 2, 3, dict(jac_freeze=2, use_graph=use_graph), oemg.Options(jac_freeze=2))


def test_krylov_tolerance_vcycles():
    """Krylov tolerance of Sec. 5 (reading C4): the same steps are taken as in the oracle."""
    import paper_1807_01151_gb300 as pkg
    _cycles(pkg, ogrid(16, 8), 1, 2, dict(krylov_tol=1e-5), oemg.Options(krylov_tol=1e-5))


def test_krylov_tolerance_exp1_step_stops_early():
    import paper_1807_01151_gb300 as pkg
    desc = ogrid(16, 8)
    s = pkg.Solver(desc, p_max=1, krylov_tol=1e-5)
    dg = DG(desc, 1)
    u0 = np.ascontiguousarray(perturbed_state(dg, amp=0.05)[:, :, :1])
    dt = oemg.dtau(dg, 1, perturbed_state(dg, amp=0.05), 10.0)
    ug, kg = s.exp1_step(u0, dt)
    uo, ko = oemg.exp1_step(dg, u0, np.zeros_like(u0), dt, oemg.Options(krylov_tol=1e-5))
    s.close()
    assert kg == ko < 30
    assert rel_err(ug - u0, uo - u0) < TOL_CYCLE


@pytest.mark.parametrize("mk,p", [(lambda: ogrid(16, 6), 3), (lambda: cubed_sphere_shell(2, 2), 2)])
def test_symmetry_plane_residual_and_vcycle(mk, p):
    """Half meshes with symmetry planes on y = 0 (Sec. 5, sphere case): residuals at every
    level and one V-cycle against the oracle."""
    import paper_1807_01151_gb300 as pkg
    desc, _ = half_mesh(mk(), axis=1)
    s = pkg.Solver(desc, p_max=p)
    dg = DG(desc, p)
    u = perturbed_state(dg, amp=0.02)
    for lev in range(p + 1):
        ul = np.ascontiguousarray(u[:, :, :dg.N(lev)])
        assert rel_err(s.residual(lev, ul), dg.residual(lev, ul)) < 1e-12, lev
    s.set_state(np.ascontiguousarray(u))
    s.vcycle()
    uo, _ = oemg.vcycle(dg, u, 1)
    assert rel_err(s.get_state(), uo) < TOL_CYCLE
    s.close()


def test_unbuilt_options_are_rejected():
    import paper_1807_01151_gb300 as pkg
    for kw in (dict(quad_extra=3), dict(omega=(1.0, 0.0, 0.0)), dict(jac_freeze=-1), dict(krylov_tol=-1.0)):
        with pytest.raises(pkg.EmgError) as ei:
            pkg.Solver(ogrid(8, 2), p_max=1, **kw)
        assert ei.value.status == 1, kw


def test_probe_peaks_are_plausible():
    """The library's register-only FMA probes (the ALU roofline denominators)."""
    from paper_1807_01151_gb300._lib import probe_peaks
    pk = probe_peaks()
    assert 0.3 < pk["fp64_tflops"] < 5.0, pk
    assert 20.0 < pk["fp32_tflops"] < 200.0, pk
    assert pk["fp32_tflops"] > 10 * pk["fp64_tflops"]
    assert 300.0 < pk["sm_mhz"] < 2500.0, pk
    # the rates stay below the unit counts (2 FP64 and 128 FP32 FMA per clock per SM, 152 SMs)
    # at the probe's own clock and reach most of them
    r64 = pk["fp64_tflops"] / (2 * 2 * 152 * pk["sm_mhz"] * 1e-6)
    r32 = pk["fp32_tflops"] / (128 * 2 * 152 * pk["sm_mhz"] * 1e-6)
    assert 0.7 < r64 < 1.02 and 0.7 < r32 < 1.02, (r64, r32, pk)


def test_fp64_form_at_3d_p4():
    """The plain FP64 form at 3-D p = 4 (175 x 175 float64 blocks, larger than shared memory:
    factored in global memory): the PRK step and one V-cycle against the oracle."""
    import paper_1807_01151_gb300 as pkg
    name, mk, p = BLOCK_CASES[2]
    desc, dg, u, D = oracle_case(name, mk, p)
    s = pkg.Solver(desc, p_max=p)
    for cfl in (3.0, 100.0):
        ug = s.prk_step(p, u, cfl=cfl)
        dt = oemg.dtau(dg, p, u, cfl)
        P = np.eye(D.shape[-1])[None] / dt[:, None, None] - D
        uo = oemg.prk_step(lambda w: dg.residual(p, w), P, u)
        assert rel_err(ug - u, uo - u) < TOL_CYCLE, (cfl, rel_err(ug - u, uo - u))
    s.set_state(np.ascontiguousarray(u))
    s.vcycle()
    uo, _ = oemg.vcycle(dg, u, 1)
    assert rel_err(s.get_state(), uo) < TOL_CYCLE
    s.close()


@pytest.mark.parametrize("name,mk,p", BLOCK_CASES)
@pytest.mark.parametrize("kernels", [1, 2, 3])
def test_inverse_of_non_finite_blocks_completes(name, mk, p, kernels):
    """A state with NaN entries (a diverging solve) gives blocks with NaN entries: the
    Gauss-Jordan forms must still pick one pivot row per step (the lowest unused row when a
    column has no number), so the permutation stays whole, the call completes and the
    context stays usable; the result is simply not finite."""
    import paper_1807_01151_gb300 as pkg
    desc, dg, u, D = oracle_case(name, mk, p)
    s = pkg.Solver(desc, p_max=p, prec=1, block_kernels=kernels)
    bad = u.copy()
    bad[::3, :, :] = np.nan
    X = s.block_operator(p, bad, cfl=3.0, which=1)
    assert not np.isfinite(X[::3]).any()
    Xg = s.block_operator(p, u, cfl=3.0, which=1)       # the context still works
    assert np.isfinite(Xg).all()
    s.close()
