"""Orthonormal Cartesian modal basis (oracle; test infrastructure).

Sec. 3.2, Eqs. basis2 and basis: normalised monomials
chi = ((x-x_c)/L_x)^p1 ((y-y_c)/L_y)^p2 ((z-z_c)/L_z)^p3 in graded order, made
orthonormal on each element with modified Gram-Schmidt, so that
psi_i = s_i [chi_i + sum_{j<i} c_ij chi_j] with s_i > 0.

Reading of the garbled index set of Eq. basis2: the monomials are ordered by total
degree 0, 1, ..., p and, within one degree, lexicographically with the x exponent
descending, then y (then z).  The basis is hierarchical: level p uses the first
N_p = C(p+d, d) functions of the p_max basis.
"""
import numpy as np


def n_modes(dim, p):
    if dim == 2:
        return (p + 1) * (p + 2) // 2
    return (p + 1) * (p + 2) * (p + 3) // 6


def exponents(dim, p):
    out = []
    for k in range(p + 1):
        if dim == 2:
            for a in range(k, -1, -1):
                out.append((a, k - a))
        else:
            for a in range(k, -1, -1):
                for b in range(k - a, -1, -1):
                    out.append((a, b, k - a - b))
    return np.array(out, dtype=np.int64)


def degrees(dim, p):
    return exponents(dim, p).sum(axis=1)


def monomials(x, xc, L, exps):
    """chi_k and grad chi_k at points.

    x: [E][P][d], xc, L: [E][d], exps: [N][d] -> chi [E][P][N], grad [E][P][N][d].
    """
    s = (x - xc[:, None, :]) / L[:, None, :]                       # [E][P][d]
    d = x.shape[-1]
    N = exps.shape[0]
    chi = np.ones(x.shape[:2] + (N,))
    for k in range(d):
        chi = chi * s[..., k:k + 1] ** exps[None, None, :, k]
    grad = np.zeros(x.shape[:2] + (N, d))
    for k in range(d):
        g = np.ones(x.shape[:2] + (N,))
        for j in range(d):
            if j == k:
                e = exps[:, j]
                pw = np.where(e[None, None, :] > 0, s[..., j:j + 1] ** np.maximum(e - 1, 0)[None, None, :], 0.0)
                g = g * e[None, None, :] * pw / L[:, None, k:k + 1]
            else:
                g = g * s[..., j:j + 1] ** exps[None, None, :, j]
        grad[..., k] = g
    return chi, grad


def mgs_coefficients(chi, W):
    """Modified Gram-Schmidt on the sampled monomials with <f,g> = sum_q W_q f_q g_q.

    chi: [E][Q][N], W: [E][Q].  Returns C [E][N][N] (lower triangular, positive
    diagonal) with psi_i = sum_k C[i, k] chi_k.
    """
    E, Q, N = chi.shape
    C = np.zeros((E, N, N))
    psi = np.zeros((E, Q, N))
    for i in range(N):
        v = chi[:, :, i].copy()
        c = np.zeros((E, N))
        c[:, i] = 1.0
        for j in range(i):
            r = np.sum(W * v * psi[:, :, j], axis=1)
            v -= r[:, None] * psi[:, :, j]
            c -= r[:, None] * C[:, j, :]
        s = np.sqrt(np.sum(W * v * v, axis=1))
        psi[:, :, i] = v / s[:, None]
        C[:, i, :] = c / s[:, None]
    return C


class Basis:
    """Per-element orthonormal basis at p_max, built on the q = p_max + 2 volume rule."""

    def __init__(self, mesh, p_max, q):
        from .geometry import volume_rule
        self.dim = mesh.dim
        self.p_max = p_max
        self.exps = exponents(mesh.dim, p_max)
        self.N = len(self.exps)
        xi, w = volume_rule(mesh.dim, q)
        x, _, detJ = mesh.map_points(xi)
        W = detJ * w[None, :]
        chi, _ = monomials(x, mesh.xc, mesh.half_extent, self.exps)
        self.C = mgs_coefficients(chi, W)
        self.xc = mesh.xc
        self.L = mesh.half_extent

    def evaluate(self, x, elem_idx, n):
        """psi_i and grad psi_i, i < n, of elements elem_idx at their points x [k][P][d]."""
        chi, g = monomials(x, self.xc[elem_idx], self.L[elem_idx], self.exps[:n])
        C = self.C[elem_idx][:, :n, :n]
        psi = np.einsum('ik,epk->epi', C, chi) if C.ndim == 2 else np.einsum('eik,epk->epi', C, chi)
        grad = np.einsum('eik,epkd->epid', C, g)
        return psi, grad
