"""Modal DG residual and its Jacobian blocks (oracle; test infrastructure).

Eq. euler3 with the orthonormal basis (mass matrix = I):

  R_{e,a,i} = sum_q sum_k W_q d_k psi_i(x_q) F_{k,a}(U_h(x_q))
              - sum_{faces of e} sum_{face pts} |n dS| psi_i F~_a(U_in, U_out, n)

with U_h = sum_j u_{a,j} psi_j (Eq. uexp), F~ the Roe flux on interior faces and
F~(U_L, U_ghost(U_L)) on boundary faces (Sec. 3.3).  Level p uses the first N_p
basis functions and q = p + 2 Gauss points per direction.

Jacobians (Eqs. jac1, jac2) are computed here as what they are by definition, the
derivative of R_p, using complex-step differentiation (exact to rounding for the
analytic continuation of R_p): the element-diagonal blocks with a distance-1
colouring, the p = 0 off-diagonal blocks with a distance-2 colouring, and
Jacobian-vector products J x = Im R(u + i h x) / h.
"""
import numpy as np

from . import euler
from .basis import Basis, n_modes
from .geometry import Mesh, volume_rule
from workloads import BC_WALL, BC_FARFIELD, BC_SYMMETRY, BC_EXACT

CSTEP = 1e-30


class Level:
    pass


class DG:
    def __init__(self, desc, p_max, mach=0.3, alpha_deg=0.0, gamma=euler.GAMMA,
                 exact_state=None, source=None, omega=None):
        """exact_state(x[..., d]) -> U[..., 5] feeds BC_EXACT ghosts; source(x) -> S[..., 5]
        is added as int psi_i S dx (both only for manufactured-solution tests).  omega: the
        angular velocity of the rotating frame (Eq. euler; None or 0: a stationary frame;
        in 2-D only its z component)."""
        self.dim = desc.dim
        self.p_max = p_max
        self.gamma = gamma
        self.mesh = Mesh(desc, q_geom=p_max + 2)
        self.basis = Basis(self.mesh, p_max, q=p_max + 2)
        self.Uinf = euler.freestream(mach, alpha_deg, gamma)
        self.exact_state = exact_state
        self.source = source
        om = None if omega is None else np.asarray(omega, dtype=float)
        if om is not None and not np.any(om):
            om = None
        if om is not None and desc.dim == 2 and (om[0] != 0.0 or om[1] != 0.0):
            raise ValueError("in 2-D the rotation axis must be z")
        self.omega = om
        self.E = self.mesh.E
        self.levels = [self._build_level(p) for p in range(p_max + 1)]

    def N(self, p):
        return n_modes(self.dim, p)

    def _build_level(self, p):
        m, b, d = self.mesh, self.basis, self.dim
        q = p + 2
        n = self.N(p)
        L = Level()
        L.p, L.N, L.q = p, n, q
        xi, w = volume_rule(d, q)
        x, _, detJ = m.map_points(xi)
        W = detJ * w[None, :]
        ei = np.arange(self.E)
        psi, grad = b.evaluate(x, ei, n)
        L.x, L.W = x, W
        L.psi = psi                                               # [E][Q][N]
        L.wgrad = W[:, :, None, None] * grad                      # [E][Q][N][d]
        # interior faces: points from the L element's map; R's basis at the same points
        xf, af = m.face_points(m.int_L, m.int_fL, q)
        L.int_amag = np.linalg.norm(af, axis=-1)
        L.int_n = af / L.int_amag[..., None]
        L.int_psiL, _ = b.evaluate(xf, m.int_L, n)
        L.int_psiR, _ = b.evaluate(xf, m.int_R, n)
        xb, ab = m.face_points(m.bnd_L, m.bnd_f, q)
        L.bnd_x = xb
        L.bnd_amag = np.linalg.norm(ab, axis=-1)
        L.bnd_n = ab / L.bnd_amag[..., None] if ab.size else ab
        wn = m.face_wall_normals(m.bnd_L, m.bnd_f, q) if len(m.bnd_L) else None
        # slip-wall reflection normal: the true body normal when given, else the facet's
        if wn is None:
            L.bnd_wn = L.bnd_n
        else:
            have = np.linalg.norm(wn, axis=-1, keepdims=True) > 0
            L.bnd_wn = np.where(have, wn, L.bnd_n)
        L.bnd_psi, _ = b.evaluate(xb, m.bnd_L, n) if len(m.bnd_L) else (np.zeros((0, 1, n)), None)
        L.bnd_code = m.bnd_code
        if self.source is not None:
            L.src = np.einsum('eq,eqi,eqa->eai', W, psi, self.source(x))
        if self.omega is not None:
            # frame velocity v_r = omega x x at volume and face points
            L.vr = self.frame_velocity(x)
            L.int_vrn = np.sum(self.frame_velocity(xf) * L.int_n, axis=-1)
            L.bnd_vr = self.frame_velocity(xb)
            L.bnd_vrn = np.sum(L.bnd_vr * L.bnd_n, axis=-1) if xb.size else np.zeros(xb.shape[:2])
        return L

    def frame_velocity(self, x):
        """omega x x at points x[..., d] (3 components)."""
        x3 = np.zeros(x.shape[:-1] + (3,))
        x3[..., :x.shape[-1]] = x
        return np.cross(self.omega, x3)

    # -- states ---------------------------------------------------------------
    def freestream_state(self, p=None):
        p = self.p_max if p is None else p
        u = np.zeros((self.E, 5, self.N(p)))
        u[:, :, 0] = self.Uinf[None, :] * np.sqrt(self.mesh.vol)[:, None]
        return u

    def evaluate_at(self, p, u, x, elem_idx):
        psi, _ = self.basis.evaluate(x, elem_idx, self.N(p))
        return np.einsum('eai,epi->epa', u[elem_idx], psi)

    def centroid_state(self, p, u):
        x = self.mesh.xc[:, None, :]
        return self.evaluate_at(p, u, x, np.arange(self.E))[:, 0, :]

    # -- residual -------------------------------------------------------------
    def ghost(self, UL, n, x, code, wn=None, vr=None):
        """Ghost states; the slip wall mirrors the velocity about wn (body normal), a
        symmetry plane (Sec. 5, sphere case) about the face's own normal n; in a rotating
        frame (vr: the frame velocity at the points) the velocity relative to the frame."""
        G = np.empty_like(UL)
        wall = code == BC_WALL
        far = code == BC_FARFIELD
        sym = code == BC_SYMMETRY
        exact = code == BC_EXACT
        sel = (lambda m: None) if vr is None else (lambda m: vr[m])
        if wall.any():
            G[wall] = euler.wall_ghost(UL[wall], (n if wn is None else wn)[wall], sel(wall), self.gamma)
        if sym.any():
            G[sym] = euler.wall_ghost(UL[sym], n[sym], sel(sym), self.gamma)
        if far.any():
            G[far] = euler.farfield_ghost(UL[far], n[far], self.Uinf, self.gamma, sel(far))
        if exact.any():
            G[exact] = self.exact_state(x[exact]).astype(UL.dtype)
        return G

    def residual(self, p, u):
        """R_p(u), u [E][5][N_p] (real or complex) -> [E][5][N_p]."""
        L = self.levels[p]
        d = self.dim
        rot = self.omega is not None
        Uq = np.einsum('eai,eqi->eqa', u, L.psi)
        F = euler.flux(Uq, self.gamma, L.vr if rot else None)[..., :d, :]
        R = np.einsum('eqik,eqka->eai', L.wgrad, F)
        m = self.mesh
        if len(m.int_L):
            UL = np.einsum('fai,fqi->fqa', u[m.int_L], L.int_psiL)
            UR = np.einsum('fai,fqi->fqa', u[m.int_R], L.int_psiR)
            Fh = L.int_amag[..., None] * euler.roe(UL, UR, L.int_n, self.gamma, L.int_vrn if rot else None)
            np.add.at(R, m.int_L, -np.einsum('fqi,fqa->fai', L.int_psiL, Fh))
            np.add.at(R, m.int_R, np.einsum('fqi,fqa->fai', L.int_psiR, Fh))
        if len(m.bnd_L):
            UL = np.einsum('fai,fqi->fqa', u[m.bnd_L], L.bnd_psi)
            code = np.broadcast_to(L.bnd_code[:, None], UL.shape[:2])
            G = self.ghost(UL, L.bnd_n, L.bnd_x, code, L.bnd_wn, L.bnd_vr if rot else None)
            Fh = L.bnd_amag[..., None] * euler.roe(UL, G, L.bnd_n, self.gamma, L.bnd_vrn if rot else None)
            np.add.at(R, m.bnd_L, -np.einsum('fqi,fqa->fai', L.bnd_psi, Fh))
        if self.source is not None:
            R = R + L.src
        if rot:
            # Eq. euler's source S = (0, -rho omega x v, 0) = (0, -omega x (rho v), 0), as int psi_i S
            S = np.zeros(Uq.shape, dtype=Uq.dtype)
            S[..., 1:4] = -np.cross(np.broadcast_to(self.omega, Uq[..., 1:4].shape), Uq[..., 1:4])
            R = R + np.einsum('eq,eqi,eqa->eai', L.W, L.psi, S)
        return R

    # -- derivatives ----------------------------------------------------------
    def jvp(self, p, u, x):
        """J_p x = dR_p/du . x, exact to rounding (complex step)."""
        return self.residual(p, u + 1j * CSTEP * x).imag / CSTEP

    def diag_blocks(self, p, u):
        """D_e = dR_{p,e}/du_e, [E][5N][5N] with row/col index a*N + i (Eq. jac1)."""
        n = self.N(p)
        b = 5 * n
        D = np.zeros((self.E, b, b))
        col = self.mesh.coloring(1)
        for c in range(col.max() + 1):
            mask = col == c
            for a in range(5):
                for j in range(n):
                    uc = u.astype(complex)
                    uc[mask, a, j] += 1j * CSTEP
                    Ri = self.residual(p, uc).imag / CSTEP
                    D[mask, :, a * n + j] = Ri[mask].reshape(-1, b)
        return D

    def full_jacobian(self, p, u):
        """Dense dR_p/du [K][K] (K = E*5*N_p) from a distance-2 colouring (small meshes)."""
        n = self.N(p)
        b = 5 * n
        K = self.E * b
        J = np.zeros((K, K))
        m = self.mesh
        col = m.coloring(2)
        owner = np.full(self.E, -1)
        for c in range(col.max() + 1):
            mask = col == c
            # every element is itself perturbed or has at most one perturbed neighbour
            owner[:] = -1
            owner[mask] = np.nonzero(mask)[0]
            for e in np.nonzero(~mask)[0]:
                for nb in m.neighbours[e]:
                    if mask[nb]:
                        owner[e] = nb
            for a in range(5):
                for j in range(n):
                    uc = u.astype(complex)
                    uc[mask, a, j] += 1j * CSTEP
                    Ri = self.residual(p, uc).imag.reshape(self.E, b) / CSTEP
                    for e in np.nonzero(owner >= 0)[0]:
                        J[e * b:(e + 1) * b, owner[e] * b + a * n + j] = Ri[e]
        return J

    def p0_blocks(self, u0):
        """p = 0 Jacobian in block form (Eqs. jac1, jac2).

        Returns diag [E][5][5] and off [E][2d][5][5], off[e, f] = dR_e/du_nb for the
        neighbour across local face f (zero on boundary faces).
        """
        m = self.mesh
        diag = np.zeros((self.E, 5, 5))
        off = np.zeros((self.E, m.nf, 5, 5))
        nb = -np.ones((self.E, m.nf), dtype=np.int64)
        nb[m.int_L, m.int_fL] = m.int_R
        nb[m.int_R, m.int_fR] = m.int_L
        col = m.coloring(2)
        for c in range(col.max() + 1):
            mask = col == c
            for bvar in range(5):
                uc = u0.astype(complex)
                uc[mask, bvar, 0] += 1j * CSTEP
                Ri = self.residual(0, uc).imag[:, :, 0] / CSTEP      # [E][5]
                diag[mask, :, bvar] = Ri[mask]
                for f in range(m.nf):
                    has = nb[:, f] >= 0
                    tgt = has.copy()
                    tgt[has] = mask[nb[has, f]]
                    off[tgt, f, :, bvar] = Ri[tgt]
        return diag, off, nb
