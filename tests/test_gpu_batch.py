"""Batched boxes: each box of a batch (one set of launches per step for all
boxes) must evolve exactly as it does alone.  With deterministic spreading
every kernel does the same arithmetic per box in both modes, so the states
agree bitwise."""
import math

import numpy as np
import pytest

import oracle
from gpu_helpers import gpu_f_to_oracle, gpu_sim, lattice_perm, rel_l2
from workloads import BoxSpec, SwimmerSpec, assemble, fluid_box, single_swimmer_48

pytestmark = pytest.mark.gpu


def _small(center, a=3.0, L=9.0, alpha=math.pi / 2, amp=1e-3):
    return SwimmerSpec(center=center, radius=a, subdiv=1, spacing=L, period=60.0).with_drive(amp, amp, alpha)


def _boxes():
    return [
        BoxSpec(dims=(32, 24, 20), swimmers=(_small((16.0, 12.0, 10.0)),)),
        BoxSpec(dims=(40, 32, 28), swimmers=(_small((20.0, 10.0, 14.0), alpha=1.1), _small((20.0, 22.0, 14.0), alpha=1.1))),
        fluid_box((24, 20, 16), tau=0.8, g=(1e-6, 0.0, 0.0)),
        single_swimmer_48(period=200.0),
    ]


@pytest.fixture(scope="module")
def perm(gpu_lib):
    return lattice_perm()


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_batch_matches_boxes_alone(perm, storage):
    from paper_2202_12147_gb300 import Batch
    boxes = _boxes()
    asms = [assemble(b) for b in boxes]
    steps = (3, 34)  # single steps, then graph replays and a tail
    alone = []
    for b, a in zip(boxes, asms):
        s = gpu_sim(b, a, deterministic=True, storage=storage)
        for n in steps:
            s.lb_step(n)
        alone.append((s.get_populations(), s.get_nodes() if s.n_nodes else None,
                      s.swimmer_state(0) if s.n_swimmers else None))
        s.close()
    sims = [gpu_sim(b, a, deterministic=True, storage=storage) for b, a in zip(boxes, asms)]
    batch = Batch(sims)
    for n in steps:
        batch.lb_step(n)
    for k, s in enumerate(sims):
        f_ref, r_ref, st_ref = alone[k]
        assert np.array_equal(s.get_populations(), f_ref), f"box {k} populations differ"
        if r_ref is not None:
            assert np.array_equal(s.get_nodes(), r_ref), f"box {k} nodes differ"
            st = s.swimmer_state(0)
            assert st["step"] == sum(steps)
            assert np.array_equal(st["x_cm"], st_ref["x_cm"])
    with pytest.raises(Exception):
        sims[0].lb_step(1)  # batched contexts step only through the batch
    batch.close()
    sims[0].lb_step(1)      # free again once the batch is gone
    for s in sims:
        s.close()


def test_batched_box_against_oracle(perm):
    """One batched box against the FP64 oracle (velocity field within 1e-5)."""
    from paper_2202_12147_gb300 import Batch
    boxes = _boxes()
    asms = [assemble(b) for b in boxes]
    sims = [gpu_sim(b, a) for b, a in zip(boxes, asms)]
    batch = Batch(sims)
    batch.lb_step(40)
    k = 1
    fg = gpu_f_to_oracle(sims[k].get_populations(), perm)
    osim = oracle.OracleSim(boxes[k], asms[k]).step(40)
    _, ug = oracle.macros(fg)
    _, uo = oracle.macros(osim.f)
    assert rel_l2(ug, uo) < 1e-5
    assert np.abs(sims[k].get_nodes() - osim.r).max() < 1e-7
    batch.close()
    for s in sims:
        s.close()


def test_autotuned_batch_against_oracle(perm):
    """lb_batch_autotune times the launch-shape candidates on real steps, keeps
    the fastest and re-captures the graph; the tuning steps are ordinary steps,
    and the tuned batch still matches the oracle."""
    from paper_2202_12147_gb300 import Batch
    boxes = _boxes()
    asms = [assemble(b) for b in boxes]
    sims = [gpu_sim(b, a) for b, a in zip(boxes, asms)]
    batch = Batch(sims)
    rep = batch.autotune(steps_per_trial=2)
    assert len(rep["classes"]) == 4
    assert rep["steps_taken"] >= 4 and rep["steps_taken"] % 2 == 0
    for c in rep["classes"]:
        assert c["cells_per_thread"] in (1, 2)
        assert str(c["cells_per_thread"]) in c["us_by_cells_per_thread"]
        assert c["dims"][0] % c["cells_per_thread"] == 0
    assert rep["marked_blocks"] >= 1
    n = 40 - rep["steps_taken"] % 16
    batch.lb_step(n)  # graph replays from the tuned capture plus single steps
    total = rep["steps_taken"] + n
    k = 1
    assert sims[k].swimmer_state(0)["step"] == total
    fg = gpu_f_to_oracle(sims[k].get_populations(), perm)
    osim = oracle.OracleSim(boxes[k], asms[k]).step(total)
    _, ug = oracle.macros(fg)
    _, uo = oracle.macros(osim.f)
    assert rel_l2(ug, uo) < 1e-5
    assert np.abs(sims[k].get_nodes() - osim.r).max() < 1e-7
    batch.close()
    for s in sims:
        s.close()


def test_checkpoint_resume_is_bitwise(perm, tmp_path):
    """A run checkpointed at step 13 and resumed in a fresh context (from a
    file) continues bitwise like the uninterrupted run (deterministic
    spreading); a corrupted or mismatched blob is refused."""
    from paper_2202_12147_gb300._lib import LbibError
    box = _boxes()[1]
    asm = assemble(box)
    a = gpu_sim(box, asm, deterministic=True)
    a.lb_step(13)
    blob = a.checkpoint()
    path = tmp_path / "state.lbib"
    blob.tofile(path)
    a.lb_step(21)
    ref = (a.get_populations(), a.get_nodes(), a.swimmer_state(1))
    a.close()
    b = gpu_sim(box, asm, deterministic=True)
    b.restore(np.fromfile(path, dtype=np.uint8))
    assert b.swimmer_state(0)["step"] == 13
    b.lb_step(21)
    assert np.array_equal(b.get_populations(), ref[0])
    assert np.array_equal(b.get_nodes(), ref[1])
    st = b.swimmer_state(1)
    assert st["step"] == 34 and np.array_equal(st["disp"], ref[2]["disp"])
    bad = blob.copy()
    bad[len(bad) // 2] ^= 1
    with pytest.raises(LbibError):
        b.restore(bad)
    other = gpu_sim(_boxes()[0], assemble(_boxes()[0]), deterministic=True)
    with pytest.raises(LbibError):
        other.restore(blob)
    other.close()
    b.close()
