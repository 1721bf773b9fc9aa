"""Deterministic mesh generators for the synthetic cylinder / sphere / box workloads.

Conventions shared by every consumer (they are the interface, not the method):

* ``xyz``         float64 [dim][n_nodes] (structure of arrays).
* ``elem_nodes``  int64 [n_elems][2**dim], node order of the reference element
                  (-1,-1),(1,-1),(1,1),(-1,1) for quads; the same four at zeta=-1
                  followed by the same four at zeta=+1 for hexes.
* ``face_bc``     int32 [n_elems][2*dim]; local face f = 2*axis + (side > 0), i.e.
                  xi=-1, xi=+1, eta=-1, eta=+1, zeta=-1, zeta=+1.  Value -1 marks an
                  interior face (its neighbour is found by matching nodes), otherwise a
                  boundary code below.

* ``wall_normal``  optional float64 [dim][n_nodes]: unit normal of the true (curved)
                  wall at wall nodes (other entries unused).  Straight-sided elements
                  only approximate a curved body; the slip-wall condition reflects the
                  velocity about this normal.

The paper's meshes (896 curved hexes around a cylinder, 14026 curved tets/prisms
around a sphere, Sec. 5) are not available; these straight-sided O-grids and
cubed-sphere shells with geometric radial stretching stand in for them.
"""
from dataclasses import dataclass
import math

import numpy as np

BC_INTERIOR = -1
BC_WALL = 1        # inviscid slip wall (mirror ghost state)
BC_FARFIELD = 2    # characteristic far field built from Riemann invariants
BC_SYMMETRY = 3    # symmetry plane: mirror ghost about the (flat) face normal
BC_EXACT = 9       # ghost = prescribed exact state (manufactured-solution tests only)


@dataclass
class MeshDesc:
    dim: int
    xyz: np.ndarray         # [dim][n_nodes] float64
    elem_nodes: np.ndarray  # [n_elems][2**dim] int64
    face_bc: np.ndarray     # [n_elems][2*dim] int32
    name: str = ""
    wall_normal: np.ndarray = None   # [dim][n_nodes] unit normal of the true wall at wall nodes

    @property
    def n_elems(self):
        return int(self.elem_nodes.shape[0])

    @property
    def n_nodes(self):
        return int(self.xyz.shape[1])


def _radii(n_r, r0, r1):
    return np.array([r0 * (r1 / r0) ** (l / n_r) for l in range(n_r + 1)], dtype=np.float64)


def ogrid(n_theta, n_r, r0=0.5, r1=20.0, inner_bc=BC_WALL, outer_bc=BC_FARFIELD):
    """O-grid annulus around a circular cylinder.

    Nodes sit at theta_k = 2*pi*k/n_theta (symmetric about the x axis) and
    r_l = r0*(r1/r0)**(l/n_r) (geometric stretching).  Element (k, l) is
    e = l*n_theta + k; its reference xi axis runs outward in r, eta in theta.
    """
    if n_theta < 3 or n_r < 1:
        raise ValueError("ogrid needs n_theta >= 3 and n_r >= 1")
    r = _radii(n_r, r0, r1)
    th = 2.0 * np.pi * np.arange(n_theta) / n_theta
    xyz = np.empty((2, n_theta * (n_r + 1)), dtype=np.float64)
    for l in range(n_r + 1):
        xyz[0, l * n_theta:(l + 1) * n_theta] = r[l] * np.cos(th)
        xyz[1, l * n_theta:(l + 1) * n_theta] = r[l] * np.sin(th)

    def node(k, l):
        return l * n_theta + (k % n_theta)

    E = n_theta * n_r
    en = np.empty((E, 4), dtype=np.int64)
    fb = np.full((E, 4), BC_INTERIOR, dtype=np.int32)
    for l in range(n_r):
        for k in range(n_theta):
            e = l * n_theta + k
            en[e] = [node(k, l), node(k, l + 1), node(k + 1, l + 1), node(k + 1, l)]
            if l == 0:
                fb[e, 0] = inner_bc
            if l == n_r - 1:
                fb[e, 1] = outer_bc
    # the wall is the circle r = r0: its normal at a wall node is the radial direction
    wn = np.zeros_like(xyz)
    wn[0, :n_theta] = np.cos(th)
    wn[1, :n_theta] = np.sin(th)
    return MeshDesc(2, xyz, en, fb, name=f"ogrid{n_theta}x{n_r}", wall_normal=wn)


def box(nx, ny, x0=0.0, x1=1.0, y0=0.0, y1=1.0, bc=BC_EXACT, jitter=0.0, seed=0):
    """Structured quad mesh of a rectangle; interior nodes optionally jittered.

    ``jitter`` is a fraction of the local spacing; the displacement is a seeded
    uniform draw, small enough (< 0.25) to keep every quad convex.
    """
    xs = np.linspace(x0, x1, nx + 1)
    ys = np.linspace(y0, y1, ny + 1)
    X, Y = np.meshgrid(xs, ys)  # [ny+1][nx+1]
    X = X.copy()
    Y = Y.copy()
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        hx = (x1 - x0) / nx
        hy = (y1 - y0) / ny
        dx = rng.uniform(-jitter, jitter, X.shape) * hx
        dy = rng.uniform(-jitter, jitter, Y.shape) * hy
        dx[0, :] = dx[-1, :] = 0.0
        dx[:, 0] = dx[:, -1] = 0.0
        dy[0, :] = dy[-1, :] = 0.0
        dy[:, 0] = dy[:, -1] = 0.0
        X += dx
        Y += dy
    xyz = np.stack([X.ravel(), Y.ravel()]).astype(np.float64)

    def node(i, j):
        return j * (nx + 1) + i

    E = nx * ny
    en = np.empty((E, 4), dtype=np.int64)
    fb = np.full((E, 4), BC_INTERIOR, dtype=np.int32)
    for j in range(ny):
        for i in range(nx):
            e = j * nx + i
            en[e] = [node(i, j), node(i + 1, j), node(i + 1, j + 1), node(i, j + 1)]
            if i == 0:
                fb[e, 0] = bc
            if i == nx - 1:
                fb[e, 1] = bc
            if j == 0:
                fb[e, 2] = bc
            if j == ny - 1:
                fb[e, 3] = bc
    return MeshDesc(2, xyz, en, fb, name=f"box{nx}x{ny}")


def cubed_sphere_shell(n, n_r, r0=0.5, r1=20.0, inner_bc=BC_WALL, outer_bc=BC_FARFIELD):
    """Equiangular gnomonic cubed-sphere shell: 6 panels x n x n x n_r trilinear hexes.

    Surface nodes are keyed by their integer lattice point on the cube surface so
    that panel seams share nodes.  Reference axes: xi, eta tangential, zeta radial.
    """
    if n < 1 or n_r < 1:
        raise ValueError("cubed_sphere_shell needs n >= 1 and n_r >= 1")
    r = _radii(n_r, r0, r1)
    t = np.array([math.tan(-math.pi / 4 + i * math.pi / (2 * n)) for i in range(n + 1)])
    t[0], t[-1] = -1.0, 1.0
    key_index = {}
    unit = []

    def surf_node(key):
        idx = key_index.get(key)
        if idx is None:
            idx = len(unit)
            key_index[key] = idx
            p = np.array([t[key[0]], t[key[1]], t[key[2]]])
            unit.append(p / np.linalg.norm(p))
        return idx

    panels = []
    for a in range(3):
        for s in (-1, 1):
            ua, va = ((a + 1) % 3, (a + 2) % 3) if s > 0 else ((a + 2) % 3, (a + 1) % 3)
            panels.append((a, s, ua, va))
    quads = []
    for (a, s, ua, va) in panels:
        for j in range(n):
            for i in range(n):
                q = []
                for (ii, jj) in ((i, j), (i + 1, j), (i + 1, j + 1), (i, j + 1)):
                    key = [0, 0, 0]
                    key[a] = 0 if s < 0 else n
                    key[ua] = ii
                    key[va] = jj
                    q.append(surf_node(tuple(key)))
                quads.append(q)
    ns = len(unit)
    unit = np.array(unit)
    xyz = np.empty((3, ns * (n_r + 1)), dtype=np.float64)
    for l in range(n_r + 1):
        xyz[:, l * ns:(l + 1) * ns] = (r[l] * unit).T
    E = len(quads) * n_r
    en = np.empty((E, 8), dtype=np.int64)
    fb = np.full((E, 6), BC_INTERIOR, dtype=np.int32)
    e = 0
    for l in range(n_r):
        for q in quads:
            en[e, :4] = [l * ns + v for v in q]
            en[e, 4:] = [(l + 1) * ns + v for v in q]
            if l == 0:
                fb[e, 4] = inner_bc
            if l == n_r - 1:
                fb[e, 5] = outer_bc
            e += 1
    wn = np.zeros_like(xyz)
    wn[:, :ns] = unit.T          # sphere r = r0: radial unit vectors at the wall nodes
    return MeshDesc(3, xyz, en, fb, name=f"cubedsphere6x{n}x{n}x{n_r}", wall_normal=wn)


def half_mesh(desc, axis=1, tol=1e-9):
    """The part of a mesh on the positive side of the plane x_axis = 0, with the faces that lie
    on the plane tagged as symmetry planes (the paper's sphere mesh respects the flow's planes
    of symmetry and imposes a symmetry condition on them, Sec. 5).

    Elements are kept when the mean of their nodes is on the positive side, in their original
    order; nodes are renumbered in order of first use.  A face is on the plane when all of its
    nodes are within tol * (largest node coordinate) of it.  Returns (MeshDesc, kept element
    indices of the input mesh).
    """
    dim = desc.dim
    nn = 1 << dim
    X = desc.xyz
    cen = X[:, desc.elem_nodes].mean(axis=2)              # [dim][E]
    keep = np.nonzero(cen[axis] > 0.0)[0]
    en = desc.elem_nodes[keep]
    new_id = {}
    for nd in en.ravel():
        if int(nd) not in new_id:
            new_id[int(nd)] = len(new_id)
    old_of_new = np.array(list(new_id.keys()), dtype=np.int64)
    en_new = np.array([new_id[int(nd)] for nd in en.ravel()], dtype=np.int64).reshape(en.shape)
    xyz = X[:, old_of_new].copy()
    fb = desc.face_bc[keep].copy()
    scale = np.abs(X).max()
    ref = np.array([[(a & 1) ^ ((a >> 1) & 1), (a >> 1) & 1, (a >> 2) & 1] for a in range(nn)])
    for e in range(len(keep)):
        for f in range(2 * dim):
            ax, side = f >> 1, f & 1
            loc = [a for a in range(nn) if ref[a][ax] == side]
            if np.all(np.abs(xyz[axis, en_new[e, loc]]) <= tol * scale):
                fb[e, f] = BC_SYMMETRY
    wn = None if desc.wall_normal is None else desc.wall_normal[:, old_of_new].copy()
    return MeshDesc(dim, xyz, en_new, fb, name=desc.name + f"_half{axis}", wall_normal=wn), keep


# The synthetic stand-ins for the paper's cylinder and sphere cases.
NAMED = {
    "cyl32x16": dict(kind="ogrid", n_theta=32, n_r=16, p_max=2),
    "cyl64x32": dict(kind="ogrid", n_theta=64, n_r=32, p_max=4),
    "cyl128x64": dict(kind="ogrid", n_theta=128, n_r=64, p_max=4),
    "cyl256x128": dict(kind="ogrid", n_theta=256, n_r=128, p_max=4),
    "sphere6x16x16x24": dict(kind="sphere", n=16, n_r=24, p_max=3),
    "sphere6x24x24x32": dict(kind="sphere", n=24, n_r=32, p_max=4),
}


def named_config(name):
    """Return (MeshDesc, p_max) for one of the named synthetic workloads."""
    c = NAMED[name]
    if c["kind"] == "ogrid":
        return ogrid(c["n_theta"], c["n_r"]), c["p_max"]
    return cubed_sphere_shell(c["n"], c["n_r"]), c["p_max"]
