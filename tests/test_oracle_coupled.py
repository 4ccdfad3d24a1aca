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
