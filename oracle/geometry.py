"""Mesh connectivity, reference maps and element geometry (oracle; test infrastructure).

Follows Sec. 3.2 (x_c, L_x, L_y, L_z of the basis definition) and Eq. x3d
(h_3D = 2 d |E| / |dE|).  Quadrature is tensor Gauss-Legendre with q points per
direction (the paper does not name its rule; q = p + 2 integrates psi_i psi_j det J
exactly on bilinear quads and trilinear hexes, so the discrete and exact inner
products agree).
"""
import itertools

import numpy as np


def ref_nodes(dim):
    quad = [(-1.0, -1.0), (1.0, -1.0), (1.0, 1.0), (-1.0, 1.0)]
    if dim == 2:
        return np.array(quad)
    return np.array([q + (-1.0,) for q in quad] + [q + (1.0,) for q in quad])


def gauss_legendre(q):
    """Nodes and weights on [-1, 1] (numpy's Golub-Welsch implementation)."""
    x, w = np.polynomial.legendre.leggauss(q)
    return x, w


def shape_functions(dim, xi):
    """Multilinear shape functions and their reference gradients.

    xi: [..., dim].  Returns N [..., 2**dim] and dN [..., 2**dim, dim].
    """
    rn = ref_nodes(dim)
    fac = 0.5 * (1.0 + xi[..., None, :] * rn)            # [..., a, d]
    N = np.prod(fac, axis=-1)
    dN = np.empty(fac.shape)
    for k in range(dim):
        others = np.prod(np.delete(fac, k, axis=-1), axis=-1)
        dN[..., k] = 0.5 * rn[:, k] * others
    return N, dN


def volume_rule(dim, q):
    x, w = gauss_legendre(q)
    pts = np.array(list(itertools.product(x, repeat=dim)))[:, ::-1]
    wts = np.array([np.prod(c) for c in itertools.product(w, repeat=dim)])
    return pts.copy(), wts


def face_rule(dim, q, f):
    """Reference points/weights on local face f = 2*axis + (side > 0)."""
    axis, side = f // 2, (1.0 if f % 2 else -1.0)
    x, w = gauss_legendre(q)
    others = [k for k in range(dim) if k != axis]
    sub = list(itertools.product(x, repeat=dim - 1))
    subw = [np.prod(c) for c in itertools.product(w, repeat=dim - 1)]
    pts = np.zeros((len(sub), dim))
    pts[:, axis] = side
    for n, c in enumerate(sub):
        for j, k in enumerate(others):
            pts[n, k] = c[::-1][j] if dim == 3 else c[0]
    return pts, np.array(subw), axis, side


def face_nodes(dim, f):
    rn = ref_nodes(dim)
    axis, side = f // 2, (1.0 if f % 2 else -1.0)
    return [a for a in range(len(rn)) if rn[a, axis] == side]


class Mesh:
    """Connectivity and per-element geometry of a MeshDesc (see workloads.meshes)."""

    def __init__(self, desc, q_geom):
        self.dim = d = desc.dim
        self.nodes = np.ascontiguousarray(desc.xyz.T)          # [n_nodes][d]
        self.elems = np.asarray(desc.elem_nodes, dtype=np.int64)
        self.face_bc = np.asarray(desc.face_bc, dtype=np.int64)
        wn = getattr(desc, "wall_normal", None)
        self.node_wall_normal = None if wn is None else np.ascontiguousarray(np.asarray(wn).T)
        self.E = self.elems.shape[0]
        self.nf = 2 * d
        self._match_faces()
        self._geometry(q_geom)

    # -- connectivity ---------------------------------------------------------
    def _match_faces(self):
        seen = {}
        iL, fL, iR, fR = [], [], [], []
        bE, bF, bC = [], [], []
        for e in range(self.E):
            for f in range(self.nf):
                bc = self.face_bc[e, f]
                if bc >= 0:
                    bE.append(e), bF.append(f), bC.append(bc)
                    continue
                key = frozenset(self.elems[e, face_nodes(self.dim, f)].tolist())
                if key in seen:
                    e0, f0 = seen.pop(key)
                    iL.append(e0), fL.append(f0), iR.append(e), fR.append(f)
                else:
                    seen[key] = (e, f)
        if seen:
            raise ValueError(f"{len(seen)} interior faces without a neighbour")
        self.int_L = np.array(iL, dtype=np.int64)
        self.int_fL = np.array(fL, dtype=np.int64)
        self.int_R = np.array(iR, dtype=np.int64)
        self.int_fR = np.array(fR, dtype=np.int64)
        self.bnd_L = np.array(bE, dtype=np.int64)
        self.bnd_f = np.array(bF, dtype=np.int64)
        self.bnd_code = np.array(bC, dtype=np.int64)
        nbrs = [set() for _ in range(self.E)]
        for a, b in zip(iL, iR):
            nbrs[a].add(b)
            nbrs[b].add(a)
        self.neighbours = [sorted(s) for s in nbrs]

    def coloring(self, distance=1):
        """Greedy colouring: no two elements within `distance` face hops share a colour."""
        col = -np.ones(self.E, dtype=np.int64)
        for e in range(self.E):
            near = set(self.neighbours[e])
            if distance >= 2:
                for n in self.neighbours[e]:
                    near.update(self.neighbours[n])
            near.discard(e)
            used = {col[n] for n in near if col[n] >= 0}
            c = 0
            while c in used:
                c += 1
            col[e] = c
        return col

    # -- maps -----------------------------------------------------------------
    def map_points(self, xi):
        """Physical points, Jacobians and det J of every element at reference points.

        xi: [P][d] -> x [E][P][d], J [E][P][d][d] (J[i][k] = dx_i/dxi_k), detJ [E][P].
        """
        N, dN = shape_functions(self.dim, xi)
        X = self.nodes[self.elems]                                  # [E][a][d]
        x = np.einsum('pa,ead->epd', N, X)
        J = np.einsum('pak,eai->epik', dN, X)
        return x, J, np.linalg.det(J)

    def face_points(self, elem_idx, f_idx, q):
        """Physical points and area vectors (w * outward n dS, 3 components) on faces.

        The outward area element of face xi_k = s is s * cof(J)[:, k] dA_ref with
        cof(J) = det(J) J^{-T}.
        """
        d = self.dim
        P = q ** (d - 1)
        x = np.empty((len(elem_idx), P, d))
        a = np.zeros((len(elem_idx), P, 3))
        for f in range(self.nf):
            sel = np.nonzero(f_idx == f)[0]
            if len(sel) == 0:
                continue
            pts, w, axis, side = face_rule(d, q, f)
            N, dN = shape_functions(d, pts)
            X = self.nodes[self.elems[elem_idx[sel]]]
            x[sel] = np.einsum('pa,ead->epd', N, X)
            J = np.einsum('pak,eai->epik', dN, X)
            cof = np.linalg.det(J)[..., None, None] * np.swapaxes(np.linalg.inv(J), -1, -2)
            a[sel, :, :d] = side * cof[..., :, axis] * w[None, :, None]
        return x, a

    def face_wall_normals(self, elem_idx, f_idx, q):
        """Unit normal of the true wall at face points: the node normals interpolated with
        the face's shape functions and normalised (for a circle or sphere centred at the
        origin this is exactly the radial direction of the point).  None without normals."""
        if self.node_wall_normal is None:
            return None
        d = self.dim
        out = np.zeros((len(elem_idx), q ** (d - 1), 3))
        for f in range(self.nf):
            sel = np.nonzero(f_idx == f)[0]
            if len(sel) == 0:
                continue
            pts, _, _, _ = face_rule(d, q, f)
            N, _ = shape_functions(d, pts)
            nn = self.node_wall_normal[self.elems[elem_idx[sel]]]        # [k][a][d]
            v = np.einsum('pa,ead->epd', N, nn)
            nv = np.linalg.norm(v, axis=-1, keepdims=True)
            out[sel, :, :d] = np.divide(v, nv, out=np.zeros_like(v), where=nv > 0)
        return out

    def _geometry(self, q):
        xi, w = volume_rule(self.dim, q)
        x, J, detJ = self.map_points(xi)
        if np.any(detJ <= 0):
            raise ValueError("element with non-positive Jacobian determinant")
        W = detJ * w[None, :]
        self.vol = W.sum(axis=1)
        self.xc = np.einsum('ep,epd->ed', W, x) / self.vol[:, None]
        X = self.nodes[self.elems]
        self.half_extent = 0.5 * (X.max(axis=1) - X.min(axis=1))
        surf = np.zeros(self.E)
        for f in range(self.nf):
            ei = np.arange(self.E)
            _, a = self.face_points(ei, np.full(self.E, f), q)
            surf += np.linalg.norm(a, axis=-1).sum(axis=1)
        self.surf = surf
        self.h = 2.0 * self.dim * self.vol / self.surf
        self.domain_volume = self.vol.sum()
