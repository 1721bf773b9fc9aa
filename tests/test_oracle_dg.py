"""Pins of the oracle's DG residual and Jacobians (Eqs. euler3, jac1, jac2)."""
import numpy as np
import pytest

from oracle import euler
from oracle.dg import DG
from tests.helpers import perturbed_state
from workloads import BC_EXACT, BC_FARFIELD, BC_SYMMETRY, BC_WALL, box, cubed_sphere_shell, ogrid


@pytest.mark.parametrize("desc,p", [(ogrid(8, 3, inner_bc=BC_FARFIELD), 3),
                                    (cubed_sphere_shell(2, 1, inner_bc=BC_FARFIELD), 2)])
def test_freestream_preserved(desc, p):
    dg = DG(desc, p, mach=0.4, alpha_deg=17.0)
    u = dg.freestream_state()
    for lev in range(p + 1):
        R = dg.residual(lev, u[:, :, :dg.N(lev)])
        assert np.abs(R).max() < 1e-13 * np.abs(u).max()


def test_freestream_preserved_distorted_box_exact_bc():
    Uinf = euler.freestream(0.3, 30.0)
    dg = DG(box(4, 3, jitter=0.2, seed=2, bc=BC_EXACT), 3, mach=0.3, alpha_deg=30.0,
            exact_state=lambda x: np.broadcast_to(Uinf, x.shape[:-1] + (5,)).copy())
    R = dg.residual(3, dg.freestream_state())
    assert np.abs(R).max() < 1e-13


def test_closed_slip_box_conserves_mass_and_energy():
    """With slip walls only, mass and energy fluxes through the boundary vanish, so the
    cell-mean residuals sum to zero for any state (interior Roe fluxes cancel)."""
    dg = DG(box(4, 3, jitter=0.2, seed=4, bc=BC_WALL), 2)
    u = perturbed_state(dg, amp=0.1)
    R = dg.residual(2, u)
    total = np.einsum('e,ea->a', np.sqrt(dg.mesh.vol), R[:, :, 0])
    scale = np.abs(R).max()
    assert abs(total[0]) < 1e-13 * scale
    assert abs(total[4]) < 1e-13 * scale


def test_residual_conservation_split():
    """sum_e int_E R_h = -(sum of boundary fluxes): interior fluxes telescope."""
    dg = DG(ogrid(6, 3), 2)
    u = perturbed_state(dg, amp=0.05)
    R = dg.residual(2, u)
    total = np.einsum('e,ea->a', np.sqrt(dg.mesh.vol), R[:, :, 0])
    L = dg.levels[2]
    m = dg.mesh
    UL = np.einsum('fai,fqi->fqa', u[m.bnd_L], L.bnd_psi)
    code = np.broadcast_to(L.bnd_code[:, None], UL.shape[:2])
    Gs = dg.ghost(UL, L.bnd_n, L.bnd_x, code, L.bnd_wn)
    bflux = np.einsum('fq,fqa->a', L.bnd_amag, euler.roe(UL, Gs, L.bnd_n))
    assert np.allclose(total, -bflux, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("desc", [ogrid(7, 2), cubed_sphere_shell(2, 1)])
def test_wall_reflection_normal_is_the_body_normal(desc):
    """Interpolated node normals at wall face points equal the radial direction of the
    point (circle / sphere centred at the origin), in closed form."""
    dg = DG(desc, 2)
    L = dg.levels[2]
    wall = L.bnd_code == BC_WALL
    x = L.bnd_x[wall]
    radial = x / np.linalg.norm(x, axis=-1, keepdims=True)
    wn = L.bnd_wn[wall][..., :dg.dim]
    assert np.abs(np.abs(np.sum(wn * radial, axis=-1)) - 1.0).max() < 1e-14
    # the facet normal differs from it (the walls are faceted)
    assert np.abs(np.abs(np.sum(L.bnd_n[wall][..., :dg.dim] * radial, axis=-1)) - 1.0).max() > 1e-4


def test_jvp_and_blocks_against_finite_differences():
    dg = DG(ogrid(5, 2), 2)
    u = perturbed_state(dg, amp=0.05)
    rng = np.random.default_rng(0)
    for p in (2, 1, 0):
        up = u[:, :, :dg.N(p)]
        x = rng.standard_normal(up.shape)
        eps = 1e-6
        fd = (dg.residual(p, up + eps * x) - dg.residual(p, up - eps * x)) / (2 * eps)
        jv = dg.jvp(p, up, x)
        assert np.abs(fd - jv).max() < 1e-7 * np.abs(jv).max()
        D = dg.diag_blocks(p, up)
        b = 5 * dg.N(p)
        # FD column of the element-diagonal block
        for (e, col) in [(0, 0), (3, b - 1), (7, b // 2)]:
            a, j = divmod(col, dg.N(p))
            du = np.zeros_like(up)
            du[e, a, j] = 1.0
            fdc = (dg.residual(p, up + eps * du) - dg.residual(p, up - eps * du))[e].ravel() / (2 * eps)
            assert np.abs(fdc - D[e, :, col]).max() < 1e-7 * np.abs(D[e]).max()


def test_blocks_equal_brute_force_dense_jacobian():
    dg = DG(ogrid(4, 2), 1)
    u = perturbed_state(dg, amp=0.05)
    for p in (1, 0):
        up = u[:, :, :dg.N(p)]
        b = 5 * dg.N(p)
        K = dg.E * b
        # dense Jacobian, one residual evaluation per column (central differences)
        Jfd = np.zeros((K, K))
        eps = 1e-6
        for k in range(K):
            du = np.zeros(K)
            du[k] = eps
            du = du.reshape(up.shape)
            Jfd[:, k] = (dg.residual(p, up + du) - dg.residual(p, up - du)).ravel() / (2 * eps)
        J = dg.full_jacobian(p, up)
        assert np.abs(J - Jfd).max() < 1e-6 * np.abs(J).max()
        D = dg.diag_blocks(p, up)
        for e in range(dg.E):
            assert np.allclose(D[e], J[e * b:(e + 1) * b, e * b:(e + 1) * b], rtol=1e-12, atol=1e-14)
    diag, off, nb = dg.p0_blocks(u[:, :, :1])
    J0 = dg.full_jacobian(0, u[:, :, :1])
    for e in range(dg.E):
        assert np.allclose(diag[e], J0[5 * e:5 * e + 5, 5 * e:5 * e + 5], atol=1e-14)
        for f in range(4):
            if nb[e, f] >= 0:
                n_ = nb[e, f]
                assert np.allclose(off[e, f], J0[5 * e:5 * e + 5, 5 * n_:5 * n_ + 5], atol=1e-14)


def mms_setup(n, p):
    g = 1.4

    def prim(x):
        X, Y = x[..., 0], x[..., 1]
        rho = 1.0 + 0.2 * np.sin(np.pi * X) * np.sin(np.pi * Y)
        v = np.zeros(x.shape[:-1] + (3,), dtype=x.dtype)
        v[..., 0] = 0.3 + 0.1 * np.cos(np.pi * X) * np.sin(np.pi * Y)
        v[..., 1] = 0.1 * np.sin(np.pi * X) * np.cos(np.pi * Y)
        pr = 1.0 / g + 0.1 * np.cos(np.pi * X) * np.cos(np.pi * Y)
        return rho, v, pr

    def exact(x):
        return euler.conservative(*prim(x))

    def source(x):
        S = np.zeros(x.shape[:-1] + (5,))
        for k in range(2):
            xc = x.astype(complex)
            xc[..., k] += 1e-30j
            S += euler.flux(exact(xc))[..., k, :].imag / 1e-30
        return S

    dg = DG(box(n, n, jitter=0.15, seed=11, bc=BC_EXACT), p, exact_state=exact, source=source)
    return dg, exact


def mms_error(n, p):
    dg, exact = mms_setup(n, p)
    L = dg.levels[p]
    u = np.einsum('eq,eqi,eqa->eai', L.W, L.psi, exact(L.x))     # L2 projection
    for _ in range(8):
        R = dg.residual(p, u)
        if np.abs(R).max() < 1e-12:
            break
        J = dg.full_jacobian(p, u)
        u = u - np.linalg.solve(J, R.ravel()).reshape(u.shape)
    assert np.abs(dg.residual(p, u)).max() < 1e-11
    Uh = np.einsum('eai,eqi->eqa', u, L.psi)
    err = np.sqrt(np.sum(L.W * (Uh[..., 0] - exact(L.x)[..., 0]) ** 2))
    return err, dg, u


@pytest.mark.slow
def test_manufactured_solution_order_p_plus_1():
    for p, sizes in ((1, (4, 8, 16)), (2, (4, 8))):
        errs = [mms_error(n, p)[0] for n in sizes]
        rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
        assert rates[-1] > p + 1 - 0.35, (p, errs, rates)


def test_residual_conservation_split_3d():
    """The telescoping of interior fluxes in 3-D (cubed-sphere shell, wall and far field)."""
    dg = DG(cubed_sphere_shell(2, 2), 1)
    u = perturbed_state(dg, amp=0.05)
    R = dg.residual(1, u)
    total = np.einsum('e,ea->a', np.sqrt(dg.mesh.vol), R[:, :, 0])
    L = dg.levels[1]
    m = dg.mesh
    UL = np.einsum('fai,fqi->fqa', u[m.bnd_L], L.bnd_psi)
    code = np.broadcast_to(L.bnd_code[:, None], UL.shape[:2])
    Gs = dg.ghost(UL, L.bnd_n, L.bnd_x, code, L.bnd_wn)
    bflux = np.einsum('fq,fqa->a', L.bnd_amag, euler.roe(UL, Gs, L.bnd_n))
    assert np.allclose(total, -bflux, rtol=1e-12, atol=1e-13 * np.abs(bflux).max())


def test_jvp_and_blocks_against_finite_differences_3d():
    dg = DG(cubed_sphere_shell(2, 1), 2)
    u = perturbed_state(dg, amp=0.05)
    rng = np.random.default_rng(1)
    eps = 1e-6
    for p in (2, 1):
        up = np.ascontiguousarray(u[:, :, :dg.N(p)])
        x = rng.standard_normal(up.shape)
        fd = (dg.residual(p, up + eps * x) - dg.residual(p, up - eps * x)) / (2 * eps)
        jv = dg.jvp(p, up, x)
        assert np.abs(fd - jv).max() < 1e-7 * np.abs(jv).max()
        D = dg.diag_blocks(p, up)
        b = 5 * dg.N(p)
        for (e, col) in [(0, 0), (5, b - 1), (17, b // 2)]:
            a, j = divmod(col, dg.N(p))
            du = np.zeros_like(up)
            du[e, a, j] = 1.0
            fdc = (dg.residual(p, up + eps * du) - dg.residual(p, up - eps * du))[e].ravel() / (2 * eps)
            assert np.abs(fdc - D[e, :, col]).max() < 1e-7 * np.abs(D[e]).max()


def _mirror_y_state(dg, u):
    """(u + M u)/2 for the reflection y -> -y of a mesh that is symmetric about y = 0: the
    element map pairs mirrored centroids; the orthonormal basis of a mirrored element is the
    mirrored basis with sign (-1)^(y exponent) per mode, and rho v changes sign."""
    from oracle.basis import exponents
    xc = dg.mesh.xc
    mir = xc.copy()
    mir[:, 1] *= -1.0
    d = np.linalg.norm(xc[None, :, :] - mir[:, None, :], axis=-1)
    perm = np.argmin(d, axis=1)
    assert np.allclose(xc[perm], mir, atol=1e-12)
    n = u.shape[2]
    sgn_mode = (-1.0) ** exponents(dg.dim, dg.p_max)[:n, 1]
    sgn_var = np.array([1.0, 1.0, -1.0, 1.0, 1.0])
    Mu = u[perm] * sgn_var[None, :, None] * sgn_mode[None, None, :]
    return 0.5 * (u + Mu)


@pytest.mark.parametrize("mk,p", [(lambda: ogrid(8, 3), 3), (lambda: cubed_sphere_shell(2, 1), 2)])
def test_symmetry_plane_equals_the_mirrored_full_domain(mk, p):
    """Symmetry boundary condition (Sec. 5, sphere case): for a state symmetric about y = 0,
    the residual of the half mesh with symmetry planes on y = 0 equals the full mesh's
    residual restricted to the same elements (across y = 0 the Roe flux sees the mirrored
    state, which is exactly the symmetry ghost)."""
    from workloads import half_mesh
    full = mk()
    half, keep = half_mesh(full, axis=1)
    assert (half.face_bc == BC_SYMMETRY).sum() > 0
    dgf = DG(full, p, mach=0.3)
    dgh = DG(half, p, mach=0.3)
    assert np.allclose(dgh.mesh.vol, dgf.mesh.vol[keep], rtol=1e-13)
    us = _mirror_y_state(dgf, perturbed_state(dgf, amp=0.05))
    for lev in range(p + 1):
        ul = us[:, :, :dgf.N(lev)]
        Rf = dgf.residual(lev, ul)[keep]
        Rh = dgh.residual(lev, np.ascontiguousarray(ul[keep]))
        assert np.abs(Rh - Rf).max() <= 1e-12 * np.abs(Rf).max(), (lev, np.abs(Rh - Rf).max())
    # the pin is not vacuous: the same faces as far-field boundaries give another residual
    from workloads import MeshDesc
    fb = half.face_bc.copy()
    fb[fb == BC_SYMMETRY] = BC_FARFIELD
    dgx = DG(MeshDesc(half.dim, half.xyz, half.elem_nodes, fb, wall_normal=half.wall_normal), p, mach=0.3)
    Rx = dgx.residual(p, np.ascontiguousarray(us[keep]))
    assert np.abs(Rx - dgf.residual(p, us)[keep]).max() > 1e-6 * np.abs(Rx).max()
