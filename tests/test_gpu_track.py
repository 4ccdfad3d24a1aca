"""Per-step trajectory points (lb_track) against the oracle and against the
library's other observables.

Every coupled step writes, for every swimmer, the bead centres R_b, the mean
node velocity V_b of each bead in that step and x_cm (Fig. 1 caption: a bead
centre is the mean of its nodes; Sec. 3, Eq. vel_swim: x_cm is the mean of
the three centres).  The oracle gives R_b(t) as the mean of its FP64 node
positions after t steps, and V_b(t) = R_b(t) - R_b(t - 1) (each node moves by
its interpolated velocity, dt = 1).
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import gpu_sim
from workloads import adjoint_small, assemble, single_swimmer_48

pytestmark = pytest.mark.gpu


def _oracle_track(box, asm, steps):
    osim = oracle.OracleSim(box, asm)
    beads = np.asarray(asm["beads"])
    sw = [s["beads"] for s in asm["swimmers"]]
    R = [oracle.bead_centres(osim.r, beads)]
    for _ in range(steps):
        osim.step(1)
        R.append(oracle.bead_centres(osim.r, beads))
    R = np.array(R)  # (steps + 1, n_beads, 3)
    Rs = np.stack([R[:, b] for b in sw], axis=1)  # (steps + 1, n_swimmers, 3, 3)
    return Rs[1:], Rs[1:] - Rs[:-1]


def test_track_matches_oracle_every_step(gpu_lib):
    """24 steps (one 16-step graph replay, then eight single steps of
    alternating parity): every step's bead centres, bead velocities and x_cm."""
    box = adjoint_small()
    asm = assemble(box)
    steps = 24
    R_o, V_o = _oracle_track(box, asm, steps)
    sim = gpu_sim(box, asm)
    sim.lb_step(steps)
    tr = sim.track(steps)
    assert tr.shape == (steps, 1)
    assert (tr["step"][:, 0] == np.arange(1, steps + 1)).all()
    R0 = R_o[0] - V_o[0]
    disp = np.abs(R_o - R0[None]).max()
    assert disp > 1e-4  # the beads have moved
    assert np.abs(tr["R"] - R_o).max() < 1e-3 * disp
    assert np.abs(tr["V"] - V_o).max() < 1e-3 * np.abs(V_o).max()
    np.testing.assert_allclose(tr["x_cm"], tr["R"].mean(axis=2), rtol=0, atol=1e-12)
    # the last point against swimmer_state (mean of the FP64 node positions)
    st = sim.swimmer_state(0)
    assert np.abs(tr["x_cm"][-1, 0] - st["x_cm"]).max() < 1e-9
    assert np.abs(tr["V"][-1, 0] - st["V"]).max() < 1e-7
    sim.close()


def test_track_same_for_every_launch_path(gpu_lib, monkeypatch):
    """Deterministic spreading: one call of 40 steps (graph replays), 40 calls
    of one step (direct launches) and LBIB_GRAPHS=0 give bitwise equal
    trajectories."""
    box = adjoint_small()
    asm = assemble(box)
    out = []
    for mode in ("whole", "single", "direct"):
        monkeypatch.setenv("LBIB_GRAPHS", "0" if mode == "direct" else "1")
        sim = gpu_sim(box, asm, deterministic=True)
        if mode == "whole":
            sim.lb_step(40)
        else:
            for _ in range(40):
                sim.lb_step(1)
        out.append((sim.track(40), sim.get_nodes()))
        sim.close()
    for tr, nodes in out[1:]:
        assert (tr == out[0][0]).all()
        assert (nodes == out[0][1]).all()


def test_track_ring_wraps_and_validates(gpu_lib):
    from paper_2202_12147_gb300._lib import TRACK_STEPS, LbibError
    box = adjoint_small()
    sim = gpu_sim(box, deterministic=True)
    with pytest.raises(LbibError):
        sim.track(1)  # no step taken yet
    sim.lb_step(60)
    early = sim.track(60)
    sim.lb_step(TRACK_STEPS + 3)  # the ring wraps; the copy comes in two runs
    n_total = 60 + TRACK_STEPS + 3
    full = sim.track(TRACK_STEPS)
    assert (full["step"][:, 0] == np.arange(n_total - TRACK_STEPS + 1, n_total + 1)).all()
    tail = sim.track(17)
    assert (tail == full[-17:]).all()
    for bad in (0, TRACK_STEPS + 1):
        with pytest.raises(LbibError):
            sim.track(bad)
    assert (np.diff(full["x_cm"][:, 0, 0]) != 0).any()
    assert early["step"][-1, 0] == 60
    sim.close()


def test_track_in_a_batch(gpu_lib):
    """Boxes advanced by a batch write their own trajectory points; in
    deterministic mode they equal the standalone boxes' bitwise."""
    from paper_2202_12147_gb300 import Batch
    box = single_swimmer_48(period=200.0)
    small = adjoint_small()
    specs = [box, small, box]
    alone = []
    for b in specs:
        s = gpu_sim(b, deterministic=True)
        s.lb_step(20)
        alone.append(s.track(20))
        s.close()
    sims = [gpu_sim(b, deterministic=True) for b in specs]
    batch = Batch(sims)
    batch.lb_step(20)
    for s, ref in zip(sims, alone):
        assert (s.track(20) == ref).all()
    batch.close()
    for s in sims:
        s.close()


def test_profiled_steps_match_plain_steps(gpu_lib):
    """The timing hook (lb_profile): 16-step graph replays with event-record
    nodes around the main fluid kernel, one-by-one launches for the rest.
    Deterministic spreading: the state equals an unprofiled run's bitwise,
    and every main-kernel launch is timed once."""
    box = adjoint_small()
    asm = assemble(box)
    ref = gpu_sim(box, asm, deterministic=True)
    ref.lb_step(37)
    sim = gpu_sim(box, asm, deterministic=True)
    sim.profile(True)
    sim.lb_step(37)  # two timed replays, five single steps
    ms, n = sim.profile_read()
    assert n == 37 and ms > 0.0
    sim.profile(True)  # discards the earlier measurements
    sim.lb_step(16)
    ms2, n2 = sim.profile_read()
    assert n2 == 16 and 0.0 < ms2 < ms
    sim.profile(False)
    ref.lb_step(16)
    assert (sim.get_nodes() == ref.get_nodes()).all()
    assert (sim.get_populations() == ref.get_populations()).all()
    assert (sim.track(53) == ref.track(53)).all()
    ref.close()
    sim.close()
