"""Pins of the oracle's coupled LB/IB step: conservation and the exact mirror
symmetries of the swimmer problem (Sec. 2.2, Sec. 3.3).  CPU only."""
import math

import numpy as np
import pytest

import oracle
from workloads import BoxSpec, SwimmerSpec, single_swimmer_48


def _momentum(sim):
    return (sim.f @ sim.c).sum(0)


def test_single_swimmer_conserves_and_stays_on_axis():
    """Net external force is zero (drive and springs both sum to zero, membrane
    forces are internal), so the total fluid momentum stays zero; the problem
    is mirror-symmetric in y and z about the swimmer axis, so x_cm drifts only
    along x."""
    box = single_swimmer_48()
    sim = oracle.OracleSim(box)
    m0 = sim.f.sum()
    x0 = sim.swimmer_centres()[0].copy()
    for _ in range(4):
        sim.step(10)
        assert sim.f.sum() == pytest.approx(m0, rel=1e-13)
        np.testing.assert_allclose(_momentum(sim), 0.0, atol=1e-13)
    x1 = sim.swimmer_centres()[0]
    assert abs(x1[1] - x0[1]) < 1e-12 and abs(x1[2] - x0[2]) < 1e-12
    # the node forces balance: sum over all nodes is zero at every step
    np.testing.assert_allclose(sim.node_force.sum(0), 0.0, atol=1e-15)
    # the beads have moved along x (the drive is on)
    R = oracle.bead_centres(sim.r, sim.asm["beads"])
    R0 = oracle.bead_centres(sim.rest, sim.asm["beads"])
    assert np.abs(R[:, 0] - R0[:, 0]).max() > 1e-5


def test_side_by_side_pair_moves_identically():
    """Two swimmers placed mirror-symmetrically about the y mid-plane move with
    identical x_cm (the paper's side-by-side observation, Sec. 3.3, holds
    exactly by symmetry)."""
    s1 = SwimmerSpec(center=(24.0, 17.0, 24.0), radius=4.0, subdiv=1, spacing=12.0).with_drive(1e-3, 1e-3, math.pi / 2)
    s2 = SwimmerSpec(center=(24.0, 31.0, 24.0), radius=4.0, subdiv=1, spacing=12.0).with_drive(1e-3, 1e-3, math.pi / 2)
    box = BoxSpec(dims=(48, 48, 48), swimmers=(s1, s2))
    sim = oracle.OracleSim(box).step(30)
    c = sim.swimmer_centres()
    assert c[0, 0] == pytest.approx(c[1, 0], abs=1e-12)
    assert c[0, 2] == pytest.approx(c[1, 2], abs=1e-12)
    assert (c[0, 1] - 17.0) == pytest.approx(-(c[1, 1] - 31.0), abs=1e-12)


def test_zero_drive_rest_state_is_fixed_point():
    """Without drive, a resting fluid with undeformed beads stays exactly at rest."""
    s = SwimmerSpec(center=(12.0, 12.0, 12.0), radius=3.0, subdiv=1, spacing=8.0, amp=(0.0, 0.0, 0.0))
    box = BoxSpec(dims=(24, 24, 24), swimmers=(s,))
    sim = oracle.OracleSim(box)
    f0 = sim.f.copy()
    r0 = sim.r.copy()
    sim.step(5)
    np.testing.assert_allclose(sim.f, f0, atol=1e-17)
    np.testing.assert_allclose(sim.r, r0, atol=1e-15)


def _rectified(A, alpha, steps=100):
    """Even-in-amplitude part [D(A) + D(-A)]/2 of the x displacement over one
    drive period from rest (the rectified drift; the odd part holds the
    linear response, including the start-up transient)."""
    from workloads import assemble  # noqa: F401
    out = []
    for sgn in (1.0, -1.0):
        s = SwimmerSpec(center=(16.0, 12.0, 12.0), radius=3.0, subdiv=1, spacing=9.0,
                        period=float(steps)).with_drive(sgn * A, sgn * A, alpha)
        out.append(oracle.displacement(BoxSpec(dims=(32, 24, 24), swimmers=(s,)), steps)[0, 0])
    return 0.5 * (out[0] + out[1]), 0.5 * (out[0] - out[1])


def test_reciprocal_forcing_gives_no_net_displacement():
    """Reciprocal drive (alpha = 0: f1 = f3, f2 = -2 f1, Sec. 2.2) is its own
    mirror image with the amplitude reversed, so the displacement is odd in the
    amplitude: no rectified drift, and in the periodic state zero net
    displacement per period (Purcell's scallop theorem, cited in Sec. 1).  The
    non-reciprocal drive (alpha = pi/2) rectifies a drift that is quadratic in
    the amplitude."""
    even0, odd0 = _rectified(1e-3, 0.0)
    even1, _ = _rectified(1e-3, math.pi / 2)
    even2, _ = _rectified(2e-3, math.pi / 2)
    assert abs(odd0) > 1e-5            # the beads do move
    assert abs(even1) > 1e-9           # a non-reciprocal stroke swims
    assert abs(even0) < 1e-4 * abs(even1)
    assert even2 / even1 == pytest.approx(4.0, rel=1e-3)


def _sphere_drag_velocity(L, steps, a=3.0, Fx=5e-4, Gs=0.1, tau=1.0):
    """Steady velocity of one bead (icosphere, subdivision 2) pulled by a total
    force Fx spread evenly over its nodes, in a periodic L^3 box whose fluid
    carries the opposite uniform force density -Fx/L^3 (zero net force)."""
    from workloads import icosphere
    unit, tris = icosphere(2)
    X = unit * a + L / 2.0
    r = X.copy()
    N = L ** 3
    _, w = oracle.lattice()
    f = np.tile(w, (N, 1))
    g = np.array([-Fx / N, 0.0, 0.0])
    fext = np.zeros_like(r)
    fext[:, 0] = Fx / len(r)
    xs = []
    for _ in range(steps):
        fn = oracle.membrane_forces(X, r, tris, Gs) + fext
        F = oracle.spread(r, fn, (L, L, L))
        f, _, u = oracle.lb_step(f, (L, L, L), tau, F, g)
        r = r + oracle.interpolate(r, u, (L, L, L))
        xs.append(r[:, 0].mean())
    U = (xs[-1] - xs[-101]) / 100.0
    U_prev = (xs[-101] - xs[-201]) / 100.0
    return U, U_prev


def _hasimoto_velocity(F, mu, a, L):
    """Velocity of a simple cubic array of spheres under force F (Hasimoto,
    J. Fluid Mech. 5 (1959) 317): F = 6 pi mu a U / K(c),
    K = 1 - 1.7601 c^(1/3) + c - 1.5593 c^2, c = (4 pi / 3) a^3 / L^3."""
    c = 4.0 * math.pi / 3.0 * a ** 3 / L ** 3
    K = 1.0 - 1.7601 * c ** (1.0 / 3.0) + c - 1.5593 * c * c
    return F * K / (6.0 * math.pi * mu * a)


@pytest.mark.slow
def test_hasimoto_drag_of_periodic_sphere_array():
    """Stokes drag on a periodic array of beads (one per box) follows
    Hasimoto's correction: the hydrodynamic radius fitted at L = 20 predicts
    the velocity at L = 28, where the periodic images weigh 30 % less, and it
    lies within a lattice unit or so of the nominal radius, as usual for a
    4-point delta kernel.  Viscosity mu = rho nu = (tau - 1/2)/3 (Sec. 2.1)."""
    F, mu, a = 5e-4, 1.0 / 6.0, 3.0
    U20, U20p = _sphere_drag_velocity(20, 800)
    U28, U28p = _sphere_drag_velocity(28, 1500)
    assert abs(U20 - U20p) < 2e-3 * U20 and abs(U28 - U28p) < 2e-3 * U28  # steady
    lo, hi = a, a + 2.0
    for _ in range(60):  # bisection: U_Hasimoto(a_h, L = 20) = U20 (decreasing in a_h)
        mid = 0.5 * (lo + hi)
        if _hasimoto_velocity(F, mu, mid, 20) > U20:
            lo = mid
        else:
            hi = mid
    a_h = 0.5 * (lo + hi)
    assert a < a_h < a + 1.5
    assert U28 == pytest.approx(_hasimoto_velocity(F, mu, a_h, 28), rel=5e-3)
