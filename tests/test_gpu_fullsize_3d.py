"""Full-size sphere workloads (cubed-sphere shells 6x16x16x24 at p = 3 and 6x24x24x32 at
p = 4): the CUDA residual on the whole mesh against the oracle on sampled elements.

An element's residual depends only on its own state and on its face neighbours' states,
so the oracle evaluates it on a patch (the sampled elements and their neighbours, faces
cut off by the patch tagged far-field).  Only the sampled elements are compared: their
faces are all inside the patch or on the true boundary.
"""
import numpy as np
import pytest

from oracle.dg import DG
from oracle.geometry import Mesh, face_nodes
from tests.helpers import rel_err
from workloads import BC_FARFIELD, BC_INTERIOR, MeshDesc, cubed_sphere_shell, standard_normal_modes

TOL = 1e-12   # the residual is FP64 on both sides; only the summation order differs


@pytest.fixture(scope="module")
def lib():
    import paper_1807_01151_gb300 as pkg
    return pkg


def _state(desc, mesh, p, seed=1807, amp=1e-2, mach=0.3):
    """U_inf + seeded draws on every mode (decaying as 1/(1+deg)^2), modal coefficients."""
    from oracle.basis import degrees
    g = 1.4
    uinf = np.array([1.0, mach, 0.0, 0.0, (1.0 / g) / (g - 1.0) + 0.5 * mach * mach])
    n = degrees(desc.dim, p).size
    xi = standard_normal_modes(mesh.E, 5, n, seed)
    scale = np.array([1.0, 0.3, 0.3, 0.3, 1.0])
    w = amp * scale[None, :, None] * xi / (1.0 + degrees(desc.dim, p)[None, None, :]) ** 2
    w[:, :, 0] += uinf[None, :]
    return np.ascontiguousarray(w * np.sqrt(mesh.vol)[:, None, None])


def _patch(desc, mesh, samples):
    elems = sorted(set(samples).union(*[mesh.neighbours[e] for e in samples]))
    en = desc.elem_nodes[elems]
    fb = desc.face_bc[elems].copy()
    keys = {}
    for k in range(len(elems)):
        for f in range(2 * desc.dim):
            if fb[k, f] == BC_INTERIOR:
                key = tuple(sorted(en[k, face_nodes(desc.dim, f)]))
                keys.setdefault(key, []).append((k, f))
    for lst in keys.values():
        if len(lst) == 1:                       # the neighbour across this face is outside
            fb[lst[0]] = BC_FARFIELD
    return MeshDesc(desc.dim, desc.xyz, np.ascontiguousarray(en), np.ascontiguousarray(fb),
                    name="patch", wall_normal=getattr(desc, "wall_normal", None)), elems


def _check(lib, n, n_r, p, levels, n_samples=40):
    desc = cubed_sphere_shell(n, n_r)
    mesh = Mesh(desc, q_geom=2)
    u = _state(desc, mesh, p)
    s = lib.Solver(desc, p_max=p, prec=1)
    rng = np.random.default_rng(7)
    E = mesh.E
    per_layer = 6 * n * n
    # wall layer, outer layer and the interior
    samples = sorted(set(rng.choice(per_layer, 8, replace=False).tolist()
                         + (E - per_layer + rng.choice(per_layer, 8, replace=False)).tolist()
                         + rng.choice(E, n_samples - 16, replace=False).tolist()))
    pdesc, elems = _patch(desc, mesh, samples)
    pos = [elems.index(e) for e in samples]
    dg = DG(pdesc, p)
    for lev in levels:
        nl = dg.N(lev)
        ul = np.ascontiguousarray(u[:, :, :nl])
        Rg = s.residual(lev, ul)[samples]
        Ro = dg.residual(lev, np.ascontiguousarray(ul[elems]))[pos]
        assert rel_err(Rg, Ro) < TOL, (lev, rel_err(Rg, Ro))
    s.close()


def test_patch_residual_equals_full_mesh_residual_in_the_oracle():
    """The patch reduction itself, checked oracle against oracle on a small shell."""
    desc = cubed_sphere_shell(3, 3)
    mesh = Mesh(desc, q_geom=2)
    u = _state(desc, mesh, 2)
    full = DG(desc, 2).residual(2, u)
    samples = [0, 7, 30, 54, 100, 161]
    pdesc, elems = _patch(desc, mesh, samples)
    assert len(elems) < mesh.E
    part = DG(pdesc, 2).residual(2, np.ascontiguousarray(u[elems]))
    pos = [elems.index(e) for e in samples]
    assert rel_err(part[pos], full[samples]) < 1e-14
    others = [k for k, e in enumerate(elems) if e not in samples and len(mesh.neighbours[e]) > 0]
    assert rel_err(part[others], full[[elems[k] for k in others]]) > 1e-8   # cut faces differ


@pytest.mark.gpu
def test_sphere_6x16x16x24_p3_sampled_residual(lib):
    _check(lib, 16, 24, 3, (3, 1, 0))


@pytest.mark.gpu
def test_sphere_6x24x24x32_p4_sampled_residual(lib):
    _check(lib, 24, 32, 4, (4, 2))


@pytest.mark.gpu
def test_sphere_6x24x24x32_p4_free_stream_preserved(lib):
    """With far-field conditions on both spheres the free stream is an exact discrete
    steady state: R(U_inf) = 0 to rounding on the full mesh."""
    desc = cubed_sphere_shell(24, 32, inner_bc=BC_FARFIELD)
    s = lib.Solver(desc, p_max=4, prec=1)
    u = s.get_state()                      # the free stream set at creation
    R = s.residual(4, u)
    mesh = Mesh(desc, q_geom=2)
    assert np.isfinite(R).all()
    assert np.abs(R).max() < 1e-12 * mesh.surf.max(), np.abs(R).max() / mesh.surf.max()
    s.close()
