"""Pins of the oracle's PRK, EXP1/Krylov, transfer operators and control (Secs. 2, 4)."""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

from oracle import emg
from oracle.basis import exponents
from oracle.dg import DG
from tests.helpers import perturbed_state
from workloads import BC_FARFIELD, ogrid


def test_prk_amplification_polynomial():
    """Linear scalar R(u) = lam (u - u*): one PRK step with P = 1/dtau - lam multiplies
    the error by sum_{j<=4} z^j/j!, z = lam/(1/dtau - lam) (from beta_k = 1/(s-k+1))."""
    for lam, dt in [(-2.0, 0.3), (-50.0, 10.0), (-0.1 + 0.0, 100.0)]:
        ustar = 0.7
        u0 = np.array([[[1.9]]])
        P = np.array([[[1.0 / dt - lam]]])
        u1 = emg.prk_step(lambda u: lam * (u - ustar), P, u0, stages=4)
        z = lam / (1.0 / dt - lam)
        g = sum(z ** j / math.factorial(j) for j in range(5))
        assert abs((u1[0, 0, 0] - ustar) - g * (1.9 - ustar)) < 1e-14


def rand_stable(K, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((K, K)) / np.sqrt(K)
    return A - 2.5 * np.eye(K)


def test_krylov_phi1_equals_dense_when_space_is_exhausted():
    for K, seed in [(6, 0), (15, 1)]:
        A = rand_stable(K, seed) * 7.0
        b = np.random.default_rng(seed + 10).standard_normal(K)
        y, k = emg.krylov_phi1(lambda x: A @ x, b, m=30)
        assert K <= k <= K + 1       # MGS may need one extra step to see the breakdown
        dense = np.linalg.solve(A, (scipy.linalg.expm(A) - np.eye(K)) @ b)
        assert np.allclose(y, dense, rtol=1e-11, atol=1e-12)


def test_phi1_of_diagonal_matrix_closed_form():
    d = np.array([-30.0, -1.0, -1e-3, 0.0, 0.5])
    b = np.ones(5)
    y, k = emg.krylov_phi1(lambda x: d * x, b, m=30)
    ref = np.where(d == 0, 1.0, np.expm1(d) / np.where(d == 0, 1.0, d))
    assert np.allclose(y, ref, rtol=1e-12)


def test_exp1_is_exact_flow_of_linear_ode():
    """For du/dt = A u + c, u + dt phi_1(dt A)(A u + c) is the exact solution at dt."""
    K = 8
    A = rand_stable(K, 3)
    c = np.random.default_rng(4).standard_normal(K)
    u0 = np.random.default_rng(5).standard_normal(K)
    dt = 0.8
    step, _ = emg.krylov_phi1(lambda x: dt * (A @ x), dt * (A @ u0 + c), m=30)
    sol = scipy.integrate.solve_ivp(lambda t, u: A @ u + c, (0, dt), u0, rtol=1e-12, atol=1e-13,
                                    method='DOP853')
    assert np.allclose(u0 + step, sol.y[:, -1], rtol=1e-9, atol=1e-10)


def test_exp1_time_step_limits():
    K = 6
    A = rand_stable(K, 7)
    R = np.random.default_rng(8).standard_normal(K)
    small, _ = emg.krylov_phi1(lambda x: 1e-8 * (A @ x), 1e-8 * R, m=30)
    assert np.allclose(small, 1e-8 * R, rtol=1e-7)
    big, _ = emg.krylov_phi1(lambda x: 1e3 * (A @ x), 1e3 * R, m=30)
    assert np.allclose(big, -np.linalg.solve(A, R), rtol=1e-9)      # Newton step


def test_restriction_prolongation_identities():
    dg = DG(ogrid(6, 2), 3)
    u = perturbed_state(dg, amp=0.05)
    for p in (3, 2, 1):
        n0 = dg.N(p - 1)
        e = u[:, :, :n0] * 0.3
        # R o P = I
        assert np.array_equal(emg.restrict(emg.prolong_add(np.zeros_like(u[:, :, :dg.N(p)]), e), n0), e)
    # the restriction of a degree <= p-1 field is exact: its level-(p-1) expansion
    # reproduces the field at the level-p points
    L2, L1 = dg.levels[2], dg.levels[1]
    coeff = np.random.default_rng(1).standard_normal((dg.E, 5, dg.N(1)))
    fine = np.zeros((dg.E, 5, dg.N(2)))
    fine[:, :, :dg.N(1)] = coeff
    coarse = emg.restrict(fine, dg.N(1))
    f_at = np.einsum('eai,eqi->eqa', fine, L2.psi)
    c_at = np.einsum('eai,eqi->eqa', coarse, L2.psi[:, :, :dg.N(1)])
    assert np.allclose(f_at, c_at, atol=1e-13)


def test_cfl_sequence():
    assert emg.cfl_n(1.0, 1, 2, 100.0, 1.0) == 1.0
    assert emg.cfl_n(1.0, 6, 2, 100.0, 1.0) == 2.0               # 1 + 5/5
    assert emg.cfl_n(1e-3, 2, 2, 100.0, 1.0) == 100.0            # capped
    assert emg.cfl_n(0.05, 2, 3, 100.0, 1.0) == 20.0             # residual branch
    assert emg.cfl_n(0.0, 2, 3, 100.0, 1.0) == 100.0


def test_dtau_freestream_closed_form():
    dg = DG(ogrid(8, 3), 2, mach=0.3)
    u = dg.freestream_state()
    for p in (2, 1, 0):
        dt = emg.dtau(dg, p, u[:, :, :dg.N(p)], 50.0)
        assert np.allclose(dt, 50.0 * dg.mesh.h / ((2 * p + 1) * 1.3), rtol=1e-13)


def test_vcycle_keeps_a_steady_state():
    dg = DG(ogrid(8, 3, inner_bc=BC_FARFIELD), 2)
    u = dg.freestream_state()
    u1, info = emg.vcycle(dg, u, 1)
    assert np.abs(u1 - u).max() < 1e-13
    assert info.res < 1e-15


def mirror_map(dg, nt, nr):
    """Element and sign maps of the reflection y -> -y of the O-grid (theta -> -theta)."""
    perm = np.empty(dg.E, dtype=np.int64)
    for l in range(nr):
        for k in range(nt):
            perm[l * nt + k] = l * nt + (nt - 1 - k) % nt
    ex = exponents(2, dg.p_max)
    sgn_mode = (-1.0) ** ex[:, 1]
    sgn_var = np.array([1.0, 1.0, -1.0, 1.0, 1.0])
    return perm, sgn_var[:, None] * sgn_mode[None, :]


def test_cylinder_vcycles_preserve_mirror_symmetry():
    nt, nr = 8, 3
    dg = DG(ogrid(nt, nr), 1)
    u = dg.freestream_state()
    perm, sgn = mirror_map(dg, nt, nr)
    opts = emg.Options()
    for n in (1, 2, 3):
        u, info = emg.vcycle(dg, u, n, opts)
        if n == 1:
            opts.res_ref = info.res
    assert np.abs(u[perm] * sgn[None] - u).max() < 1e-12 * np.abs(u).max()


@pytest.mark.slow
def test_emg_converges_to_the_newton_steady_state():
    """Path independence: the eMG fixed point is the discrete steady state R_p(U) = 0."""
    from tests.test_oracle_dg import mms_error
    _, dg, u_newton = mms_error(4, 1)
    u0 = np.einsum('eq,eqi,eqa->eai', dg.levels[1].W, dg.levels[1].psi,
                   dg.exact_state(dg.levels[1].x))
    u, cycles, ok = emg.solve_steady(dg, u0, drop=1e-11, max_cycles=300)
    assert ok, cycles
    assert np.abs(u - u_newton).max() < 1e-9 * np.abs(u_newton).max()


def _phi1_taylor(A, N, terms=80):
    """phi_1(A) N = sum_k A^k N / (k+1)! (the series definition; no matrix exponential)."""
    out = np.zeros_like(N)
    t = N.copy()
    for k in range(terms):
        out += t
        t = A @ t / (k + 2)
    return out


@pytest.mark.parametrize("mk", [lambda: ogrid(4, 1), lambda: ogrid(3, 2),
                                lambda: __import__("workloads").cubed_sphere_shell(1, 1)])
def test_exp1_step_equals_dense_phi1_on_exhausted_krylov_space(mk):
    """EXP1 on level 0 (Eq. EXP1 with local steps, du/dtau = DT R): on a tiny p = 0 mesh
    (K0 = 5E <= m) the Krylov space is the whole space, so the oracle's step must equal the
    dense u0 + phi_1(A) N with A = DT J_0 and N = DT (R_0(u0) + tau0), DT = diag(dt_e)
    repeated over the five variables.  The local steps differ between elements, so A = J DT
    or N = R (no DT) would fail; tau0 != 0 checks that the forcing enters N.  phi_1 is taken
    from its Taylor series at a moderate step and from A^-1 (e^A - I) N at a large one."""
    dg = DG(mk(), 0)
    assert 5 * dg.E <= 30
    u0 = perturbed_state(dg, amp=0.05)
    tau0 = 1e-3 * np.random.default_rng(21).standard_normal(u0.shape)
    J = dg.full_jacobian(0, u0)
    R = (dg.residual(0, u0) + tau0).ravel()
    base = emg.dtau(dg, 0, u0, 1.0)
    assert base.max() > 1.05 * base.min()            # genuinely local steps
    for scale, kind in ((0.5, "taylor"), (50.0, "dense")):
        dt = scale * base
        DT = np.repeat(dt, 5)
        A = DT[:, None] * J
        Nv = DT * R
        if kind == "taylor":
            assert np.linalg.norm(A, 2) < 4.0        # the series converges fast
            ref = _phi1_taylor(A, Nv)
        else:
            ref = np.linalg.solve(A, (scipy.linalg.expm(A) - np.eye(len(Nv))) @ Nv)
        u1, k = emg.exp1_step(dg, u0, tau0, dt, emg.Options(krylov_m=30))
        assert k <= 5 * dg.E + 1
        du = (u1 - u0).ravel()
        assert np.abs(du - ref).max() <= 1e-10 * np.abs(ref).max(), (kind, np.abs(du - ref).max())
        # the same step without the forcing differs: tau0 is really part of N
        u1b, _ = emg.exp1_step(dg, u0, np.zeros_like(u0), dt, emg.Options(krylov_m=30))
        assert np.abs((u1b - u1).ravel()).max() > 1e-6 * np.abs(ref).max()


def test_phi12_of_augmented_matrix_equals_series():
    """phi_1(H) e_1 and phi_2(H) e_1 from one exponential of the (k+2)-augmented matrix equal
    their series sum_j H^j e_1 / (j+1)! and sum_j H^j e_1 / (j+2)! (Hessenberg H)."""
    rng = np.random.default_rng(3)
    k = 7
    H = np.triu(rng.standard_normal((k, k)), -1) * 0.6
    p1, p2 = emg.phi12_small(H)
    e1 = np.zeros(k)
    e1[0] = 1.0
    s1, s2, t = np.zeros(k), np.zeros(k), e1.copy()
    f = 1.0
    for j in range(60):
        f1 = math.factorial(j + 1)
        s1 += t / f1
        s2 += t / (f1 * (j + 2))
        t = H @ t
    assert np.allclose(p1, s1, rtol=1e-13, atol=1e-15)
    assert np.allclose(p2, s2, rtol=1e-13, atol=1e-15)


def test_krylov_tolerance_mode_stops_early_within_tolerance():
    """Sec. 5 Krylov tolerance (reading C4): on a p = 0 mesh small enough for a dense
    reference (K0 = 60 > m), the tolerance-mode step stops before m steps, its distance to
    the exact phi_1(A) N is within a small multiple of the tolerance, and it is within the
    tolerance of the fixed-m step."""
    import scipy.linalg
    dg = DG(ogrid(6, 2), 0)
    u0 = perturbed_state(dg, amp=0.05)
    tau0 = np.zeros_like(u0)
    dt = emg.dtau(dg, 0, u0, 5.0)
    J = dg.full_jacobian(0, u0)
    DT = np.repeat(dt, 5)
    A = DT[:, None] * J
    Nv = DT * dg.residual(0, u0).ravel()
    exact = np.linalg.solve(A, (scipy.linalg.expm(A) - np.eye(len(Nv))) @ Nv)
    tol = 1e-5
    ut, kt = emg.exp1_step(dg, u0, tau0, dt, emg.Options(krylov_m=30, krylov_tol=tol))
    uf, kf = emg.exp1_step(dg, u0, tau0, dt, emg.Options(krylov_m=30))
    assert kt < kf == 30, (kt, kf)
    scale = np.linalg.norm(exact)
    # the estimate bounds the true error: within the tolerance of the exact step and of the
    # fixed-m step (which is exact to rounding here)
    assert np.linalg.norm((ut - u0).ravel() - exact) <= tol * scale
    assert np.linalg.norm((ut - uf).ravel()) <= tol * scale
    # and the tolerance is not idle: the same test at 1e-10 takes more steps
    _, kt2 = emg.exp1_step(dg, u0, tau0, dt, emg.Options(krylov_m=30, krylov_tol=1e-10))
    assert kt < kt2


@pytest.mark.slow
def test_frozen_blocks_converge_to_the_same_steady_state():
    """A preconditioner frozen for three V-cycles changes the path, not the fixed point R = 0
    (Eq. prk_scalar): the same Newton steady state as the default cycle."""
    from tests.test_oracle_dg import mms_error
    _, dg, u_newton = mms_error(4, 1)
    u0 = np.einsum('eq,eqi,eqa->eai', dg.levels[1].W, dg.levels[1].psi,
                   dg.exact_state(dg.levels[1].x))
    u, cycles, ok = emg.solve_steady(dg, u0, drop=1e-11, max_cycles=400,
                                     opts=emg.Options(jac_freeze=3, exp_dt_global=True))
    assert ok, cycles
    assert np.abs(u - u_newton).max() < 1e-9 * np.abs(u_newton).max()


def test_arnoldi_orthonormal_basis_and_hessenberg_projection():
    """Eq. vm: the Arnoldi vectors are orthonormal with v_1 = b/|b|, span the Krylov space
    {b, Ab, A^2 b, ...}, and H_k = V_k A V_k^T is upper Hessenberg; an invariant subspace of
    dimension 3 that contains b ends the process after three steps (happy breakdown)."""
    rng = np.random.default_rng(11)
    K, m = 40, 12
    A = rng.standard_normal((K, K))
    b = rng.standard_normal(K)
    V, H, beta, k = emg.arnoldi(lambda x: A @ x, b, m)
    assert k == m and beta == pytest.approx(np.linalg.norm(b), rel=1e-15)
    assert np.abs(V @ V.T - np.eye(k)).max() < 1e-13
    assert np.abs(V[0] - b / np.linalg.norm(b)).max() < 1e-15
    assert np.abs(V @ A @ V.T - H).max() < 1e-12 * np.abs(A).max() * K
    assert np.abs(np.tril(H, -2)).max() == 0.0
    kr = np.stack([np.linalg.matrix_power(A, j) @ b for j in range(4)])
    assert np.abs(kr - (kr @ V.T) @ V).max() < 1e-9 * np.abs(kr).max()
    # invariant subspace span(q1, q2, q3) with eigenvalues 1, -2, 4 and b its sum: the Krylov
    # space has dimension 3, the subdiagonal (sqrt 6, sqrt 3) stays well away from rounding
    Q, _ = np.linalg.qr(rng.standard_normal((K, K)))
    M = np.zeros((K, K))
    M[:3, :3] = np.diag([1.0, -2.0, 4.0])
    M[3:, 3:] = rng.standard_normal((K - 3, K - 3))
    A2 = Q @ M @ Q.T
    b2 = Q[:, :3] @ np.ones(3)
    _, H2, _, k2 = emg.arnoldi(lambda x: A2 @ x, b2, m)
    assert k2 == 3
    assert np.allclose(np.diag(H2, -1), [np.sqrt(6.0), np.sqrt(3.0)], rtol=1e-12)


def test_residual_norm_is_the_l2_norm_of_the_density_residual_field():
    """The norm of Eq. cfl: with the orthonormal basis the sum of the squared density
    coefficients equals the quadrature of R_h(rho)^2 over the mesh (on the rule the basis was
    orthonormalised with, p = p_max); the norm divides its square root by |Omega|, itself the
    quadrature of 1."""
    dg = DG(ogrid(6, 3), 2)
    L = dg.levels[2]
    R = np.random.default_rng(5).standard_normal((dg.E, 5, dg.N(2)))
    Rh = np.einsum('eqi,ei->eq', L.psi, R[:, 0, :])
    vol = L.W.sum()
    assert vol == pytest.approx(dg.mesh.domain_volume, rel=1e-13)
    assert emg.residual_norm(dg, R) == pytest.approx(np.sqrt(np.sum(L.W * Rh ** 2)) / vol, rel=1e-12)
    R2 = R.copy()
    R2[:, 1:, :] = 0.0
    assert emg.residual_norm(dg, R2) == emg.residual_norm(dg, R)
