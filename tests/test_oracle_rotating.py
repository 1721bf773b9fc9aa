"""Pins of the oracle's rotating frame (Eq. euler with omega != 0): closed forms for the source
term, states that the rotating-frame equations leave steady, the relative-velocity wall and far
field, and the Jacobians against finite differences."""
import numpy as np
import pytest

from oracle import euler
from oracle.dg import DG
from tests.helpers import perturbed_state
from workloads import BC_EXACT, BC_WALL, box, cubed_sphere_shell, ogrid

OMEGA_2D = (0.0, 0.0, 0.37)
OMEGA_3D = (0.11, -0.23, 0.31)


def uniform(dg, U0, p):
    u = np.zeros((dg.E, 5, dg.N(p)))
    u[:, :, 0] = U0[None, :] * np.sqrt(dg.mesh.vol)[:, None]
    return u


def test_source_of_a_uniform_state_is_minus_omega_cross_momentum():
    """A uniform state (its flux F - v_r U has zero divergence: div(omega x x) = 0) leaves only
    the source: R_{e,m,0} = -(omega x rho v)_m sqrt|E| on the momentum rows of mode 0 and zero
    elsewhere (Eq. euler's S as written; the printed dS/dU of the Appendix has the other sign)."""
    U0 = euler.freestream(0.3, 30.0)
    dg = DG(box(4, 3, jitter=0.2, seed=2, bc=BC_EXACT), 3, omega=OMEGA_2D,
            exact_state=lambda x: np.broadcast_to(U0, x.shape[:-1] + (5,)))
    R = dg.residual(3, uniform(dg, U0, 3))
    exp = np.zeros_like(R)
    exp[:, 1:4, 0] = -np.cross(OMEGA_2D, U0[1:4])[None, :] * np.sqrt(dg.mesh.vol)[:, None]
    assert np.abs(exp).max() > 1e-2
    assert np.abs(R - exp).max() < 1e-12 * np.abs(exp).max() + 1e-14


@pytest.mark.parametrize("case", ["rest", "axial"])
def test_states_left_steady_by_the_rotating_frame(case):
    """Fluid at rest in the absolute frame and a uniform stream along the rotation axis are
    steady in the rotating frame (zero flux divergence, zero source): R = 0 at every level on a
    3-D shell.  At rest with the shell's own boundaries: the slip wall (v_r is tangential to a
    sphere about the origin, so the relative-velocity mirror keeps the state) and the far field
    of a Ma = 0 free stream taken in relative velocities; the axial stream with exact-state
    boundaries."""
    om = np.array(OMEGA_3D)
    if case == "rest":
        U0 = euler.conservative(np.array(1.0), np.zeros(3), np.array(1.0 / 1.4))
        dg = DG(cubed_sphere_shell(2, 1), 2, mach=0.0, omega=om)
    else:
        U0 = euler.conservative(np.array(1.0), 0.2 * om / np.linalg.norm(om), np.array(1.0 / 1.4))
        dg = DG(cubed_sphere_shell(2, 1, inner_bc=BC_EXACT, outer_bc=BC_EXACT), 2, omega=om,
                exact_state=lambda x: np.broadcast_to(U0, x.shape[:-1] + (5,)))
    for p in range(3):
        R = dg.residual(p, uniform(dg, U0, p))
        assert np.abs(R).max() < 1e-13, (p, np.abs(R).max())


def test_walls_at_rest_in_the_rotating_frame_conserve_mass():
    """Slip walls fixed in the rotating frame pass no mass (the velocity relative to the wall is
    mirrored, so the Roe mass flux through the wall vanishes): the cell-mean mass residuals of a
    closed box sum to zero for any state."""
    dg = DG(box(4, 3, jitter=0.2, seed=4, bc=BC_WALL), 2, omega=OMEGA_2D)
    u = perturbed_state(dg, amp=0.1)
    R = dg.residual(2, u)
    total = np.sqrt(dg.mesh.vol) @ R[:, 0, 0]
    assert abs(total) < 1e-13 * np.abs(R[:, 0, 0]).max() * dg.E
    # the relative normal velocity of the ghost is minus the interior one
    n = np.array([[0.6, 0.8, 0.0]])
    vr = np.array([[0.3, -0.1, 0.0]])
    UL = euler.conservative(np.array([1.1]), np.array([[0.2, 0.4, 0.0]]), np.array([0.8]))
    G = euler.wall_ghost(UL, n, vr)
    wl = np.sum((UL[:, 1:4] / UL[:, :1] - vr) * n, axis=-1)
    wg = np.sum((G[:, 1:4] / G[:, :1] - vr) * n, axis=-1)
    assert np.allclose(wg, -wl, rtol=0, atol=1e-15) and abs(wl[0]) > 0.1
    assert np.allclose(euler.primitives(G)[2], euler.primitives(UL)[2], rtol=1e-15)


def test_far_field_of_the_free_stream_is_the_free_stream_in_a_rotating_frame():
    Ui = euler.freestream(0.3, 10.0)
    n = np.array([[0.6, 0.8, 0.0], [-1.0, 0.0, 0.0]])
    vr = np.array([[0.05, -0.02, 0.0], [0.0, 0.07, 0.0]])
    G = euler.farfield_ghost(np.broadcast_to(Ui, (2, 5)).copy(), n, Ui, vr=vr)
    assert np.abs(G - Ui[None, :]).max() < 1e-14


def test_rotating_jacobians_against_finite_differences():
    dg = DG(ogrid(5, 2), 2, omega=OMEGA_2D)
    u = perturbed_state(dg, amp=0.05)
    rng = np.random.default_rng(3)
    for p in (2, 0):
        up = u[:, :, :dg.N(p)]
        x = rng.standard_normal(up.shape)
        eps = 1e-6
        fd = (dg.residual(p, up + eps * x) - dg.residual(p, up - eps * x)) / (2 * eps)
        jv = dg.jvp(p, up, x)
        assert np.abs(fd - jv).max() < 1e-7 * np.abs(jv).max()


def test_rotation_axis_must_be_z_in_2d():
    with pytest.raises(ValueError):
        DG(ogrid(4, 2), 1, omega=(0.1, 0.0, 0.0))


def test_frame_velocity_is_omega_cross_x():
    """v_r = omega x x: about z in 2-D, (-w y, w x, 0); in 3-D the three components of the
    cross product (its sign decides the direction of the relative fluxes)."""
    dg = DG(ogrid(4, 2), 1, omega=(0.0, 0.0, 0.5))
    x = np.array([[1.0, 2.0], [-3.0, 0.5]])
    assert np.allclose(dg.frame_velocity(x), [[-1.0, 0.5, 0.0], [-0.25, -1.5, 0.0]], rtol=0, atol=1e-15)
    dg3 = DG(cubed_sphere_shell(1, 1), 1, omega=(1.0, 2.0, 3.0))
    assert np.allclose(dg3.frame_velocity(np.array([[4.0, 5.0, 6.0]])), [[2 * 6 - 3 * 5, 3 * 4 - 1 * 6, 1 * 5 - 2 * 4]],
                       rtol=0, atol=1e-15)
