"""Euler flux, Roe flux and boundary ghost states (oracle; test infrastructure).

All functions take conservative states U[..., 5] = (rho, rho u, rho v, rho w, rho E)
and unit normals n[..., 3].  They accept complex arrays so that the oracle can
differentiate them by complex step: |.| is the analytic continuation z*sign(Re z)
and every branch tests the real part.

* Eq. euler: F_k = (rho v_k, rho v v_k + p e_k, rho H v_k) - (v_r)_k U in a frame rotating
  with angular velocity omega (v_r = omega x x; v the absolute velocity), i.e. mass and
  momentum carried by the relative velocity v - v_r and the energy flux
  rho E (v - v_r) + p v, which is what the Appendix's Jacobian (its B_2 terms) differentiates;
  p = (gamma-1)(rho E - rho|v|^2/2), gamma = 7/5.  The source -rho omega x v is added by the
  caller (dg.DG).
* Moving faces (v_r . n = v_rn != 0): the Roe flux of the same waves with speeds shifted by
  -v_rn; walls mirror the relative velocity; the far field is the stationary-frame condition
  applied to relative velocities.
* Roe flux (Sec. 3.1, Roe 1981): F~ = (F_n(U_L)+F_n(U_R))/2 - |A^|(U_R-U_L)/2 with
  A^ the flux Jacobian at the Roe average; no entropy fix (subsonic cases only).
* Boundary faces (Sec. 3.3): F~(U_L, U_ghost(U_L)) with the same Roe solver.  Slip
  wall: mirrored normal velocity.  Far field: subsonic 1-D Riemann invariants
  normal to the face, entropy and tangential velocity taken upwind.
"""
import numpy as np

GAMMA = 1.4


def cabs(z):
    if np.iscomplexobj(z):
        return np.where(z.real >= 0, z, -z)
    return np.abs(z)


def primitives(U, gamma=GAMMA):
    rho = U[..., 0]
    v = U[..., 1:4] / rho[..., None]
    p = (gamma - 1.0) * (U[..., 4] - 0.5 * rho * np.sum(v * v, axis=-1))
    return rho, v, p


def flux(U, gamma=GAMMA, vr=None):
    """F[..., k, a]: flux of variable a in direction k (k = 0, 1, 2); vr[..., 3] the frame
    velocity omega x x at the points (None: a stationary frame)."""
    rho, v, p = primitives(U, gamma)
    H = (U[..., 4] + p) / rho
    F = np.empty(U.shape[:-1] + (3, 5), dtype=np.result_type(U, vr) if vr is not None else U.dtype)
    for k in range(3):
        F[..., k, 0] = rho * v[..., k]
        for m in range(3):
            F[..., k, 1 + m] = rho * v[..., m] * v[..., k] + (p if m == k else 0.0)
        F[..., k, 4] = rho * H * v[..., k]
    if vr is not None:
        F = F - vr[..., :, None] * U[..., None, :]
    return F


def flux_n(U, n, gamma=GAMMA, vrn=None):
    F = np.einsum('...ka,...k->...a', flux(U, gamma), n)
    return F if vrn is None else F - vrn[..., None] * U


def roe(UL, UR, n, gamma=GAMMA, vrn=None):
    """Roe flux through a face moving with normal speed vrn (None: at rest)."""
    rL, vL, pL = primitives(UL, gamma)
    rR, vR, pR = primitives(UR, gamma)
    HL = (UL[..., 4] + pL) / rL
    HR = (UR[..., 4] + pR) / rR
    sL, sR = np.sqrt(rL), np.sqrt(rR)
    den = sL + sR
    u = (sL[..., None] * vL + sR[..., None] * vR) / den[..., None]
    H = (sL * HL + sR * HR) / den
    rho = sL * sR
    q2 = np.sum(u * u, axis=-1)
    c2 = (gamma - 1.0) * (H - 0.5 * q2)
    c = np.sqrt(c2)
    qn = np.sum(u * n, axis=-1)
    drho = rR - rL
    dp = pR - pL
    dv = vR - vL
    dqn = np.sum(dv * n, axis=-1)
    a1 = (dp - rho * c * dqn) / (2.0 * c2)
    a5 = (dp + rho * c * dqn) / (2.0 * c2)
    a2 = drho - dp / c2
    dvt = dv - dqn[..., None] * n
    qr = qn if vrn is None else qn - vrn          # wave speeds relative to the face
    l1, l2, l5 = cabs(qr - c), cabs(qr), cabs(qr + c)
    diss = np.empty(UL.shape, dtype=np.result_type(UL, UR, n))
    diss[..., 0] = l1 * a1 + l2 * a2 + l5 * a5
    diss[..., 1:4] = ((l1 * a1)[..., None] * (u - c[..., None] * n)
                      + (l2 * a2)[..., None] * u
                      + (l2 * rho)[..., None] * dvt
                      + (l5 * a5)[..., None] * (u + c[..., None] * n))
    diss[..., 4] = (l1 * a1 * (H - c * qn) + l2 * a2 * 0.5 * q2
                    + l2 * rho * np.sum(u * dvt, axis=-1) + l5 * a5 * (H + c * qn))
    return 0.5 * (flux_n(UL, n, gamma, vrn) + flux_n(UR, n, gamma, vrn)) - 0.5 * diss


def wall_ghost(UL, n, vr=None, gamma=GAMMA):
    """Mirror image about n of the velocity relative to the wall (vr: the wall's velocity)."""
    if vr is None:
        m = UL[..., 1:4]
        mn = np.sum(m * n, axis=-1)
        G = UL.copy()
        G[..., 1:4] = m - 2.0 * mn[..., None] * n
        return G
    rho, v, p = primitives(UL, gamma)
    wn = np.sum((v - vr) * n, axis=-1)
    return conservative(rho, v - 2.0 * wn[..., None] * n, p, gamma)


def conservative(rho, v, p, gamma=GAMMA):
    U = np.empty(np.shape(rho) + (5,), dtype=np.result_type(rho, v, p))
    U[..., 0] = rho
    U[..., 1:4] = rho[..., None] * v
    U[..., 4] = p / (gamma - 1.0) + 0.5 * rho * np.sum(v * v, axis=-1)
    return U


def farfield_ghost(UL, n, Uinf, gamma=GAMMA, vr=None):
    """Characteristic far field; in a rotating frame the same condition on the velocities
    relative to the frame (vr at the face points; Uinf in the absolute frame)."""
    if vr is not None:
        rL, vL, pL = primitives(UL, gamma)
        ri, vi, pi = primitives(np.broadcast_to(Uinf, UL.shape).astype(UL.dtype), gamma)
        G = farfield_ghost(conservative(rL, vL - vr, pL, gamma), n,
                           conservative(ri, vi - vr, pi, gamma), gamma)
        rb, vb, pb = primitives(G, gamma)
        return conservative(rb, vb + vr, pb, gamma)
    rL, vL, pL = primitives(UL, gamma)
    ri, vi, pi = primitives(np.broadcast_to(Uinf, UL.shape).astype(UL.dtype), gamma)
    cL = np.sqrt(gamma * pL / rL)
    ci = np.sqrt(gamma * pi / ri)
    qnL = np.sum(vL * n, axis=-1)
    qni = np.sum(vi * n, axis=-1)
    Rp = qnL + 2.0 * cL / (gamma - 1.0)
    Rm = qni - 2.0 * ci / (gamma - 1.0)
    qnb = 0.5 * (Rp + Rm)
    cb = 0.25 * (gamma - 1.0) * (Rp - Rm)
    inflow = (qnb.real < 0.0)
    s = np.where(inflow, pi / ri ** gamma, pL / rL ** gamma)
    vb = np.where(inflow[..., None], vi + (qnb - qni)[..., None] * n,
                  vL + (qnb - qnL)[..., None] * n)
    rb = (cb * cb / (gamma * s)) ** (1.0 / (gamma - 1.0))
    pb = rb * cb * cb / gamma
    return conservative(rb, vb, pb, gamma)


def freestream(mach, alpha_deg=0.0, gamma=GAMMA):
    """rho = 1, p = 1/gamma (c = 1), |v| = Ma at angle alpha in the x-y plane."""
    a = np.deg2rad(alpha_deg)
    v = np.array([mach * np.cos(a), mach * np.sin(a), 0.0])
    return conservative(np.array(1.0), v, np.array(1.0 / gamma), gamma)
