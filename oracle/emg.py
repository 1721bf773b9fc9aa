"""PRK smoother, EXP1 / Krylov phi_1 step and the FAS V-cycle (oracle; test infrastructure).

Passages followed:
* Eq. prk_scalar: u^(k) = u^n + beta_k P^{-1}(u^n) R(u^(k-1)), beta_k = 1/(s-k+1), s = 4.
  Reading of the preconditioner's sign: R is the right-hand side of du/dt = R
  (Eq. starteq), so P_e = I/dtau_e - dR_e/du_e, the block-Jacobi backward-Euler
  operator (Sec. 2.3 recommends the I/dtau shift).
* Eqs. EXP1, Phi1, vm, final: u_{n+1} = u_n + dt phi_1(dt J) R with the Arnoldi
  decomposition J V_m = V_{m+1} H~_m, v_1 = N/||N||; phi_1(H_m) e_1 is taken from
  the exponential of the augmented matrix [[H_m, e_1], [0, 0]] (scipy's expm, a
  Pade scaling-and-squaring routine, replaces the Chebyshev rational approximation).
  With per-element steps the scheme is applied to du/dtau = DT R(u), DT = diag(dt_e).
* Sec. 2.3 steps 1-6: FAS V-cycle with `pre_smooth` PRK steps per level p >= 1 on the
  down leg (the paper does not fix the count; reading: 2, see Options), one EXP1 step
  on p = 0, no post-smoothing; restriction = truncation to the first N_{p-1}
  modes of the hierarchical orthonormal basis, prolongation = zero padding,
  tau_{p-1} = restrict(R~_p(v_p)) - R_{p-1}(restrict(v_p)), R~_p = R_p + tau_p.
* Eq. x3d: dtau = CFL h / ((2p+1)(|v|+c)) with v, c at the cell centre;
  EXP1 step dt_e = (p_max+1) dtau_e at p = p_max (Sec. 4).
* Krylov tolerance (Sec. 5: m = 30, tolerance 1e-5; the criterion is not stated).
  Reading: after k Arnoldi steps the process ends when the leading term of the error
  series of the phi_1 approximation, beta h_{k+1,k} |(phi_2(H_k) e_1)_k|, is at most
  tol * beta ||phi_1(H_k) e_1||; phi_1(H_k) e_1 and phi_2(H_k) e_1 are the last two
  columns of exp([[H_k, e_1, 0], [0, 0, 1], [0, 0, 0]]).  tol = 0: fixed m.
* Variants (Sec. 2.3, Sec. 4): a global EXP1 step min_e dt_e (Eq. EXP1 with one dt) and
  block factors frozen for k V-cycles (re-evaluated in cycles n with (n-1) mod k = 0).
* Eq. cfl: CFL_n = min{CFL_max, max[||R(rho_n)||^-1, 1 + (n-1)/(2p+1)]},
  ||R(rho)|| = (1/|Omega|) (sum_e sum_i R_{e,rho,i}^2)^(1/2), p = p_max.  Reading:
  the inverse-residual branch uses the residual relative to the first cycle's,
  ||R(rho_1)||/||R(rho_n)||, so that the start-up ramp does not depend on the
  units and domain size (taken literally on these meshes the branch is ~400 at
  n = 1 and the first cycle at CFL 100 produces negative densities).
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg

from . import euler


@dataclass
class Options:
    rk_stages: int = 4
    krylov_m: int = 30
    cfl_max: float = 100.0
    exp_dt_factor: float = 0.0      # <= 0 -> p_max + 1
    breakdown_rel: float = 1e-12
    res_ref: float = 0.0            # ||R(rho_1)|| of the first cycle (set by the solve loop)
    pre_smooth: int = 2             # PRK steps per level on the down leg
    krylov_tol: float = 0.0         # > 0: stop the Arnoldi process by the error estimate
    exp_dt_global: bool = False     # one EXP1 step min_e dt_e for the whole mesh
    jac_freeze: int = 1             # block factors re-evaluated every jac_freeze cycles
    frozen: dict = field(default_factory=dict)   # level -> last P (jac_freeze > 1)


def prk_step(resid, P, u_n, stages=4):
    """Eq. prk_scalar with P [E][b][b]; resid(u) -> R~(u) of the same shape as u."""
    E = u_n.shape[0]
    b = P.shape[-1]
    u = u_n
    for k in range(1, stages + 1):
        beta = 1.0 / (stages - k + 1)
        r = resid(u).reshape(E, b, 1)
        du = np.linalg.solve(P, r)[..., 0]
        u = u_n + beta * du.reshape(u_n.shape)
    return u


def phi12_small(H):
    """(phi_1(H) e_1, phi_2(H) e_1) from exp([[H, e_1, 0], [0, 0, 1], [0, 0, 0]])."""
    k = H.shape[0]
    A = np.zeros((k + 2, k + 2))
    A[:k, :k] = H
    A[0, k] = 1.0
    A[k, k + 1] = 1.0
    X = scipy.linalg.expm(A)
    return X[:k, k], X[:k, k + 1]


def krylov_converged(H, k, tol):
    """The Krylov tolerance test after k steps (H [k+1][k] with the subdiagonal h_{k+1,k})."""
    phi1, phi2 = phi12_small(H[:k, :k])
    return H[k, k - 1] * abs(phi2[k - 1]) <= tol * np.linalg.norm(phi1)


def arnoldi(matvec, b, m, breakdown_rel=1e-12, tol=0.0):
    """Arnoldi with modified Gram-Schmidt (Eq. vm).  Returns V [k][K], H [k][k], beta, k."""
    beta = np.linalg.norm(b)
    K = b.size
    V = np.zeros((m + 1, K))
    H = np.zeros((m + 1, m))
    if beta == 0.0:
        return V[:0], H[:0, :0], 0.0, 0
    V[0] = b / beta
    k = m
    for j in range(m):
        w = matvec(V[j])
        w0 = np.linalg.norm(w)
        for i in range(j + 1):
            H[i, j] = np.dot(V[i], w)
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] <= breakdown_rel * w0:
            k = j + 1
            break
        if tol > 0.0 and j + 1 < m and krylov_converged(H, j + 1, tol):
            k = j + 1
            break
        V[j + 1] = w / H[j + 1, j]
    return V[:k], H[:k, :k], beta, k


def phi1_small(H):
    """phi_1(H) e_1 from exp([[H, e_1], [0, 0]])."""
    k = H.shape[0]
    A = np.zeros((k + 1, k + 1))
    A[:k, :k] = H
    A[0, k] = 1.0
    return scipy.linalg.expm(A)[:k, k]


def krylov_phi1(matvec, b, m, breakdown_rel=1e-12, tol=0.0):
    """phi_1(A) b ~= beta V_k phi_1(H_k) e_1 (Eq. final with dt absorbed in A)."""
    V, H, beta, k = arnoldi(matvec, b, m, breakdown_rel, tol)
    if k == 0:
        return np.zeros_like(b), 0
    y = beta * phi1_small(H)
    return V.T @ y, k


def dtau(dg, p, u, cfl):
    """Eq. x3d per element at level p from the state at the cell centre."""
    Uc = dg.centroid_state(p, u)
    rho, v, pr = euler.primitives(Uc, dg.gamma)
    c = np.sqrt(dg.gamma * pr / rho)
    return cfl * dg.mesh.h / ((2 * p + 1) * (np.linalg.norm(v, axis=-1) + c))


def residual_norm(dg, R):
    """||R(rho)||_2 of Eq. cfl (orthonormal basis: int R^2 = sum of squared coefficients)."""
    return np.sqrt(np.sum(R[:, 0, :] ** 2)) / dg.mesh.domain_volume


def cfl_n(res, n, p_max, cfl_max, res_ref):
    """Eq. cfl with the residual measured relative to the first cycle's (res_ref)."""
    inv = np.inf if res == 0.0 else res_ref / res
    return min(cfl_max, max(inv, 1.0 + (n - 1) / (2 * p_max + 1)))


def exp1_step(dg, u0, tau0, dt, opts):
    """EXP1 on level 0: u0 + phi_1(DT J_0) DT R~_0(u0) (Eq. EXP1)."""
    R = dg.residual(0, u0) + tau0
    Nv = (dt[:, None, None] * R).ravel()

    def matvec(x):
        return (dt[:, None, None] * dg.jvp(0, u0, x.reshape(u0.shape))).ravel()

    du, k = krylov_phi1(matvec, Nv, opts.krylov_m, opts.breakdown_rel, opts.krylov_tol)
    return u0 + du.reshape(u0.shape), k


def restrict(v, n):
    return v[:, :, :n].copy()


def prolong_add(v, e):
    out = v.copy()
    out[:, :, :e.shape[2]] += e
    return out


@dataclass
class CycleInfo:
    n: int
    res: float
    cfl: float
    krylov_dim: int
    res5: np.ndarray = field(default_factory=lambda: np.zeros(5))


def vcycle_entry(dg, u, n, opts):
    """Residual, its norm and CFL_n at the state entering V-cycle n."""
    R0 = dg.residual(dg.p_max, u)
    res = residual_norm(dg, R0)
    if not opts.res_ref > 0.0:
        opts.res_ref = res          # the first cycle fixes the reference residual
    return R0, res, cfl_n(res, n, dg.p_max, opts.cfl_max, opts.res_ref)


def vcycle(dg, u, n, opts=None):
    """One FAS V-cycle p_max -> 0 -> p_max (Sec. 2.3), returns (new state, CycleInfo)."""
    opts = opts or Options()
    P = dg.p_max
    R0, res, cfl = vcycle_entry(dg, u, n, opts)
    fac = opts.exp_dt_factor if opts.exp_dt_factor > 0 else P + 1
    dt = fac * dtau(dg, P, u, cfl)
    if opts.exp_dt_global:
        dt = np.full_like(dt, dt.min())
    frozen = opts.jac_freeze > 1 and len(opts.frozen) > 0 and (n - 1) % opts.jac_freeze != 0
    v = {P: u}
    v0 = {}
    tau = {P: np.zeros_like(u)}
    for p in range(P, 0, -1):
        def resid(w, p=p):
            return dg.residual(p, w) + tau[p]
        for _ in range(opts.pre_smooth):
            if frozen:
                Pm = opts.frozen[p]       # the factors of the last cycle that evaluated them
            else:
                # P(u^n) is re-evaluated at the state entering every PRK step
                D = dg.diag_blocks(p, v[p])
                dt_p = dtau(dg, p, v[p], cfl)
                b = D.shape[-1]
                Pm = np.eye(b)[None, :, :] / dt_p[:, None, None] - D
                if opts.jac_freeze > 1:
                    opts.frozen[p] = Pm
            v[p] = prk_step(resid, Pm, v[p], opts.rk_stages)
        nc = dg.N(p - 1)
        v0[p - 1] = restrict(v[p], nc)
        rbar = restrict(resid(v[p]), nc)
        tau[p - 1] = rbar - dg.residual(p - 1, v0[p - 1])
        v[p - 1] = v0[p - 1].copy()
    if P == 0:
        v0[0] = u
    v[0], k = exp1_step(dg, v0[0], tau[0], dt, opts)
    for p in range(1, P + 1):
        v[p] = prolong_add(v[p], v[p - 1] - v0[p - 1])
    res5 = np.sqrt(np.sum(R0 ** 2, axis=2).sum(axis=0)) / dg.mesh.domain_volume
    return v[P], CycleInfo(n, res, cfl, k, res5)


def solve_steady(dg, u, drop=1e-10, max_cycles=200, opts=None, history=None):
    """V-cycles until ||R(rho)|| <= drop * ||R(rho)|| of the initial state."""
    opts = opts or Options()
    r0 = None
    for n in range(1, max_cycles + 1):
        _, res, _ = vcycle_entry(dg, u, n, opts)
        if r0 is None:
            r0 = res
        if history is not None:
            history.append(res)
        if res <= drop * r0:
            return u, n - 1, True
        u, _ = vcycle(dg, u, n, opts)
    return u, max_cycles, False
