"""Pins of the oracle's geometry and basis against closed forms (Sec. 3.2, Eqs. x3d, x2d)."""
import numpy as np
import pytest

from oracle.basis import Basis, exponents, monomials, n_modes
from oracle.geometry import Mesh, volume_rule
from workloads import BC_EXACT, BC_FARFIELD, MeshDesc, box, cubed_sphere_shell, ogrid


def shoelace(P):
    x, y = P[:, 0], P[:, 1]
    return 0.5 * np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y)


def test_annulus_area_closed_form():
    for nt, nr in [(8, 4), (32, 16)]:
        m = Mesh(ogrid(nt, nr, inner_bc=BC_FARFIELD), q_geom=4)
        exact = 0.5 * nt * np.sin(2 * np.pi / nt) * (20.0 ** 2 - 0.5 ** 2)
        assert abs(m.vol.sum() - exact) < 1e-12 * exact


def test_quad_area_perimeter_h_centroid():
    m = Mesh(box(5, 4, jitter=0.2, seed=3), q_geom=3)
    for e in range(m.E):
        P = m.nodes[m.elems[e]]
        A = shoelace(P)
        per = np.sum(np.linalg.norm(P - np.roll(P, -1, axis=0), axis=1))
        assert abs(m.vol[e] - A) < 1e-14
        assert abs(m.surf[e] - per) < 1e-13
        assert abs(m.h[e] - 4 * A / per) < 1e-13          # h_2D = 4A/P (d = 2)
        # polygon centroid formula
        x, y = P[:, 0], P[:, 1]
        cr = x * np.roll(y, -1) - np.roll(x, -1) * y
        cx = np.sum((x + np.roll(x, -1)) * cr) / (6 * A)
        cy = np.sum((y + np.roll(y, -1)) * cr) / (6 * A)
        assert np.allclose(m.xc[e], [cx, cy], atol=1e-14)


def extrude(desc2, dz):
    """One layer of hexes over a quad mesh (the quasi-2-D meshes of Sec. 4)."""
    n = desc2.xyz.shape[1]
    xyz = np.zeros((3, 2 * n))
    xyz[:2, :n] = desc2.xyz
    xyz[:2, n:] = desc2.xyz
    xyz[2, n:] = dz
    en = np.concatenate([desc2.elem_nodes, desc2.elem_nodes + n], axis=1)
    fb = np.full((desc2.n_elems, 6), BC_EXACT, dtype=np.int32)
    fb[:, :4] = desc2.face_bc
    return MeshDesc(3, xyz, en, fb)


def test_eq_x2d_recovers_true_2d_length():
    """Eq. x2d applied to the extruded mesh gives the true 2-D h = 4A/P."""
    d2 = box(4, 3, jitter=0.15, seed=5)
    dz = 0.37
    m2 = Mesh(d2, q_geom=3)
    m3 = Mesh(extrude(d2, dz), q_geom=3)
    h2 = 2.0 / (3.0 / m3.h - 1.0 / dz)
    assert np.allclose(h2, m2.h, rtol=1e-13)
    assert np.allclose(m3.vol, m2.vol * dz, rtol=1e-13)


def test_cubed_sphere_volume_converges_to_shell():
    vols = []
    for n in (4, 8):
        m = Mesh(cubed_sphere_shell(n, 2, r0=1.0, r1=2.0), q_geom=3)
        vols.append(m.vol.sum())
    exact = 4.0 / 3.0 * np.pi * (2.0 ** 3 - 1.0)
    e4, e8 = exact - vols[0], exact - vols[1]
    assert 0 < e8 < e4                      # faceted shell is inscribed
    assert 3.5 < np.log2(e4 / e8) < 4.5 or e8 / exact < 2e-2


@pytest.mark.parametrize("desc,p", [(ogrid(6, 3), 3), (box(3, 2, jitter=0.2, seed=1), 4),
                                    (cubed_sphere_shell(2, 1), 3)])
def test_basis_orthonormal_and_hierarchical(desc, p):
    m = Mesh(desc, q_geom=p + 2)
    b = Basis(m, p, q=p + 2)
    # Gram matrix on a finer, independent rule
    xi, w = volume_rule(m.dim, p + 4)
    x, _, detJ = m.map_points(xi)
    W = detJ * w[None, :]
    psi, _ = b.evaluate(x, np.arange(m.E), b.N)
    G = np.einsum('eq,eqi,eqj->eij', W, psi, psi)
    assert np.abs(G - np.eye(b.N)).max() < 1e-11
    # psi_1 = 1/sqrt|E|, lower-triangular C with positive diagonal (Eq. basis)
    assert np.allclose(psi[:, :, 0], 1.0 / np.sqrt(m.vol)[:, None], rtol=1e-13)
    assert np.all(np.triu(b.C, 1) == 0.0)
    assert np.all(np.diagonal(b.C, axis1=1, axis2=2) > 0)
    # every monomial of degree <= p lies in the span (projection is exact)
    chi, _ = monomials(x, m.xc, m.half_extent, exponents(m.dim, p))
    coef = np.einsum('eq,eqk,eqi->eki', W, chi, psi)
    recon = np.einsum('eki,eqi->eqk', coef, psi)
    assert np.abs(recon - chi).max() < 1e-10
    assert b.N == n_modes(m.dim, p)


def test_face_matching_and_normals_close_the_element():
    """sum of outward area vectors over an element's faces is zero (closed surface)."""
    for desc in (ogrid(5, 2), cubed_sphere_shell(2, 2), box(3, 3, jitter=0.2)):
        m = Mesh(desc, q_geom=3)
        tot = np.zeros((m.E, 3))
        for f in range(m.nf):
            _, a = m.face_points(np.arange(m.E), np.full(m.E, f), 3)
            tot += a.sum(axis=1)
        assert np.abs(tot).max() < 1e-12 * m.surf.max()
        n_int = len(m.int_L)
        n_bnd = len(m.bnd_L)
        assert 2 * n_int + n_bnd == m.E * m.nf


def test_gauss_legendre_rule():
    """q-point Gauss-Legendre on [-1, 1]: the two-point rule +-1/sqrt(3) with unit weights, and
    every rule integrates x^k exactly for k <= 2q - 1 (2/(k + 1) for even k, 0 for odd) but
    not x^(2q)."""
    from oracle.geometry import gauss_legendre
    x, w = gauss_legendre(2)
    assert np.allclose(np.sort(x), [-1 / np.sqrt(3), 1 / np.sqrt(3)], rtol=0, atol=1e-15)
    assert np.allclose(w, [1.0, 1.0], rtol=0, atol=1e-15)
    for q in range(1, 8):
        x, w = gauss_legendre(q)
        for k in range(2 * q):
            exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
            assert abs(np.sum(w * x ** k) - exact) < 1e-14
        assert abs(np.sum(w * x ** (2 * q)) - 2.0 / (2 * q + 1)) > 1e-6


@pytest.mark.parametrize("mk", [lambda: ogrid(8, 3), lambda: cubed_sphere_shell(2, 1)])
def test_wall_normals_are_radial_on_circle_and_sphere(mk):
    """The slip-wall reflection normal (node normals of the true wall, interpolated with the
    face's shape functions and normalised): for a circle or a sphere about the origin the
    interpolated node normals are the face point over the radius, so the normal is the point's
    radial direction exactly, not the facet normal; far-field faces keep the facet normal."""
    from oracle.dg import DG
    from workloads import BC_WALL
    dg = DG(mk(), 1)
    m, L = dg.mesh, dg.levels[1]
    wall = m.bnd_code == BC_WALL
    assert wall.any()
    x = L.bnd_x[wall]
    radial = np.zeros(x.shape[:-1] + (3,))
    radial[..., :dg.dim] = x / np.linalg.norm(x, axis=-1, keepdims=True)
    wn = L.bnd_wn[wall]
    assert np.abs(np.abs(np.sum(wn * radial, axis=-1)) - 1.0).max() < 1e-13
    facet = L.bnd_n[wall]
    assert np.abs(np.abs(np.sum(facet * radial, axis=-1)) - 1.0).max() > 1e-4
    assert np.array_equal(L.bnd_wn[~wall], L.bnd_n[~wall])
