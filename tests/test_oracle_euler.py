"""Pins of the oracle's flux, Roe solver and ghost states (Eq. euler, Sec. 3.1, 3.3, Appendix)."""
import numpy as np

from oracle import euler

G = 1.4


def random_states(n, seed=0):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.5, 2.0, n)
    v = rng.uniform(-0.6, 0.6, (n, 3))
    p = rng.uniform(0.4, 1.5, n)
    return euler.conservative(rho, v, p)


def unit(n, seed=1):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, 3))
    return x / np.linalg.norm(x, axis=1, keepdims=True)


def appendix_jacobian(U, n):
    """grad(psi) . dF/dU of the Appendix (Eq. dfdu) with omega = 0 and grad psi -> n.

    Reading: a_1 := gamma*E - a_0 with E the specific total energy (then a_1 = H).
    """
    rho = U[0]
    u, v, w = U[1:4] / rho
    E = U[4] / rho
    px, py, pz = n
    a0 = 0.5 * (G - 1) * (u * u + v * v + w * w)
    a1 = G * E - a0
    a2 = G - 1
    a3 = G - 2
    B1 = u * px + v * py + w * pz
    B2 = 0.0
    return np.array([
        [-B2, px, py, pz, 0],
        [a0 * px - B1 * u, B1 - B2 - a3 * u * px, u * py - a2 * v * px, u * pz - a2 * w * px, a2 * px],
        [a0 * py - B1 * v, v * px - a2 * u * py, B1 - B2 - a3 * v * py, v * pz - a2 * w * py, a2 * py],
        [a0 * pz - B1 * w, w * px - a2 * u * pz, w * py - a2 * v * pz, B1 - B2 - a3 * w * pz, a2 * pz],
        [(a0 - a1) * B1, a1 * px - a2 * B1 * u, a1 * py - a2 * v * B1, a1 * pz - a2 * B1 * w, G * B1 - B2],
    ])


def test_flux_jacobian_matches_appendix():
    U = random_states(20)
    n = unit(20)
    for k in range(20):
        J = np.zeros((5, 5))
        for b in range(5):
            Uc = U[k].astype(complex)
            Uc[b] += 1e-30j
            J[:, b] = euler.flux_n(Uc, n[k]).imag / 1e-30
        assert np.allclose(J, appendix_jacobian(U[k], n[k]), rtol=1e-13, atol=1e-13)


def test_roe_consistency_and_antisymmetry():
    UL, UR = random_states(50, 1), random_states(50, 2)
    n = unit(50)
    assert np.allclose(euler.roe(UL, UL, n), euler.flux_n(UL, n), rtol=1e-14, atol=1e-14)
    assert np.allclose(euler.roe(UL, UR, n), -euler.roe(UR, UL, -n), rtol=1e-13, atol=1e-14)


def roe_state(UL, UR):
    rL, vL, pL = euler.primitives(UL)
    rR, vR, pR = euler.primitives(UR)
    HL = (UL[4] + pL) / rL
    HR = (UR[4] + pR) / rR
    sL, sR = np.sqrt(rL), np.sqrt(rR)
    u = (sL * vL + sR * vR) / (sL + sR)
    H = (sL * HL + sR * HR) / (sL + sR)
    return u, H


def roe_matrix(u, H, n):
    """Appendix matrix evaluated at the Roe average, written with a_1 = H."""
    px, py, pz = n
    uu, vv, ww = u
    a0 = 0.5 * (G - 1) * (u @ u)
    a1 = H
    a2, a3 = G - 1, G - 2
    B1 = u @ n
    return np.array([
        [0, px, py, pz, 0],
        [a0 * px - B1 * uu, B1 - a3 * uu * px, uu * py - a2 * vv * px, uu * pz - a2 * ww * px, a2 * px],
        [a0 * py - B1 * vv, vv * px - a2 * uu * py, B1 - a3 * vv * py, vv * pz - a2 * ww * py, a2 * py],
        [a0 * pz - B1 * ww, ww * px - a2 * uu * pz, ww * py - a2 * vv * pz, B1 - a3 * ww * pz, a2 * pz],
        [(a0 - a1) * B1, a1 * px - a2 * B1 * uu, a1 * py - a2 * vv * B1, a1 * pz - a2 * B1 * ww, G * B1],
    ])


def test_roe_matrix_property_and_abs_matrix():
    """A^(U_R-U_L) = F_n(U_R)-F_n(U_L), and F~ = mean flux - |A^| dU / 2 with |A^| the
    Lagrange-interpolation matrix function on the three distinct eigenvalues."""
    UL, UR = random_states(30, 3), random_states(30, 4)
    n = unit(30, 5)
    for k in range(30):
        u, H = roe_state(UL[k], UR[k])
        A = roe_matrix(u, H, n[k])
        dU = UR[k] - UL[k]
        dF = euler.flux_n(UR[k], n[k]) - euler.flux_n(UL[k], n[k])
        assert np.allclose(A @ dU, dF, rtol=1e-12, atol=1e-13)
        c = np.sqrt((G - 1) * (H - 0.5 * u @ u))
        qn = u @ n[k]
        lam = [qn - c, qn, qn + c]
        I = np.eye(5)
        absA = np.zeros((5, 5))
        for i, li in enumerate(lam):
            term = abs(li) * I
            for j, lj in enumerate(lam):
                if j != i:
                    term = term @ (A - lj * I) / (li - lj)
            absA += term
        ref = 0.5 * (euler.flux_n(UL[k], n[k]) + euler.flux_n(UR[k], n[k])) - 0.5 * absA @ dU
        assert np.allclose(euler.roe(UL[k], UR[k], n[k]), ref, rtol=1e-11, atol=1e-12)


def test_roe_upwinds_supersonic():
    UL = euler.conservative(np.array([1.0]), np.array([[3.0, 0.1, 0.0]]), np.array([0.7]))
    UR = euler.conservative(np.array([1.2]), np.array([[2.8, 0.0, 0.1]]), np.array([0.8]))
    n = np.array([[1.0, 0.0, 0.0]])
    assert np.allclose(euler.roe(UL, UR, n), euler.flux_n(UL, n), rtol=1e-13)


def test_wall_flux_has_no_mass_or_energy_flux():
    U = random_states(40, 6)
    n = unit(40, 7)
    F = euler.roe(U, euler.wall_ghost(U, n), n)
    assert np.abs(F[:, 0]).max() < 1e-14
    assert np.abs(F[:, 4]).max() < 1e-13
    # momentum flux is the wall pressure (+ Roe correction) along n only
    tang = F[:, 1:4] - np.sum(F[:, 1:4] * n, axis=1, keepdims=True) * n
    assert np.abs(tang).max() < 1e-13


def test_farfield_ghost_of_freestream_is_freestream():
    Uinf = euler.freestream(0.3, 10.0)
    U = np.broadcast_to(Uinf, (25, 5)).copy()
    n = unit(25, 8)
    g = euler.farfield_ghost(U, n, Uinf)
    assert np.allclose(g, U, rtol=1e-14, atol=1e-14)


def test_farfield_uses_riemann_invariants():
    Uinf = euler.freestream(0.3)
    U = random_states(10, 9)
    n = unit(10, 10)
    g = euler.farfield_ghost(U, n, Uinf)
    r, v, p = euler.primitives(U)
    rg, vg, pg = euler.primitives(g)
    ri, vi, pi = euler.primitives(Uinf[None])
    c = np.sqrt(G * p / r)
    cg = np.sqrt(G * pg / rg)
    ci = np.sqrt(G * pi / ri)
    qn, qg, qi = np.sum(v * n, 1), np.sum(vg * n, 1), np.sum(vi * n, 1)
    assert np.allclose(qg + 2 * cg / (G - 1), qn + 2 * c / (G - 1), rtol=1e-13)
    assert np.allclose(qg - 2 * cg / (G - 1), qi - 2 * ci / (G - 1), rtol=1e-13)
    inflow = qg < 0
    s_g = pg / rg ** G
    assert np.allclose(s_g[inflow], (pi / ri ** G)[0], rtol=1e-12)
    assert np.allclose(s_g[~inflow], (p / r ** G)[~inflow], rtol=1e-12)
