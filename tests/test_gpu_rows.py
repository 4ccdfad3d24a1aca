"""The staged-rows main-fluid kernel for 16-bit storage
(LBIB_MAIN_KERNEL=rows) against the tile kernel.  Both run the same
four-cell update on the same stored words (the rows kernel may read them
from shared-memory copies of the 19 source row-planes, and may stage its
results in shared memory before writing them as aligned words: modes 1, 2,
3), so whole runs agree bitwise: both AA parities, rows stamped around a swimmer (skipped and left
to the marked-tile kernel), periodic seams, and row counts that R does not
divide."""
import math

import numpy as np
import pytest

from gpu_helpers import gpu_sim
from workloads import BoxSpec, SwimmerSpec, assemble, fluid_box

pytestmark = pytest.mark.gpu


def _sim(box, asm, kernel, monkeypatch, R=None, mode=None, **kw):
    monkeypatch.setenv("LBIB_MAIN_KERNEL", kernel)
    if R is not None:
        monkeypatch.setenv("LBIB_ROWS_PER_BLOCK", str(R))
    if mode is not None:
        monkeypatch.setenv("LBIB_ROWS_MODE", str(mode))
    s = gpu_sim(box, asm, **kw)
    for v in ("LBIB_MAIN_KERNEL", "LBIB_ROWS_PER_BLOCK", "LBIB_ROWS_MODE"):
        monkeypatch.delenv(v, raising=False)
    return s


def _swimmer_box():
    sw = SwimmerSpec(center=(64.0, 16.0, 12.0), radius=4.0, subdiv=2, spacing=12.0, period=60.0).with_drive(
        2e-3, 2e-3, math.pi / 2)
    return BoxSpec(dims=(128, 32, 24), swimmers=(sw,))


def _run(box, asm, kernel, monkeypatch, storage, R=None, mode=None):
    s = _sim(box, asm, kernel, monkeypatch, R=R, mode=mode, storage=storage, deterministic=True)
    s.lb_step(3)   # single steps of both parities
    s.lb_step(32)  # graph replays
    out = (s.get_populations(), s.get_nodes(), s.lb_get_macros()[1].cpu().numpy())
    s.close()
    return out


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("R,mode", [(1, 3), (4, 3), (5, 3), (4, 1), (5, 2), (1, 2)])
def test_rows_kernel_matches_tile_kernel_with_swimmer(gpu_lib, monkeypatch, storage, R, mode):
    box = _swimmer_box()
    asm = assemble(box)
    ref = _run(box, asm, "tiles", monkeypatch, storage)
    got = _run(box, asm, "rows", monkeypatch, storage, R=R, mode=mode)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_rows_kernel_matches_tile_kernel_fluid_only(gpu_lib, monkeypatch, mode):
    """No immersed boundary (the main kernel advances the step counter), a
    uniform body force, 64-cell rows, 7 x 9 rows."""
    box = fluid_box((64, 7, 9), tau=0.7, g=(2e-6, -1e-6, 5e-7))
    ref = _run(box, None, "tiles", monkeypatch, "f16")
    got = _run(box, None, "rows", monkeypatch, "f16", R=4, mode=mode)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


def test_rows_kernel_on_the_benchmark_box(gpu_lib, monkeypatch):
    """One 256 x 128 x 128 box of the six-box benchmark workload."""
    from workloads import pair_boxes_256x128x128
    box = pair_boxes_256x128x128()[0]
    asm = assemble(box)
    out = []
    for k in ("tiles", "rows"):
        s = _sim(box, asm, k, monkeypatch, storage="f16", deterministic=True)
        s.lb_step(18)
        out.append((s.get_nodes(), s.lb_get_macros()[1].cpu().numpy()))
        s.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("kernel", ["rows2", "rows4"])
def test_adjacent_rows_kernel_matches_tile_kernel(gpu_lib, monkeypatch, storage, kernel):
    """Two or four adjacent rows per block (30 rows per plane: the last block
    of four holds two), rows stamped around a swimmer skipped per row."""
    sw = SwimmerSpec(center=(64.0, 15.0, 12.0), radius=4.0, subdiv=2, spacing=12.0, period=60.0).with_drive(
        2e-3, 2e-3, math.pi / 2)
    box = BoxSpec(dims=(128, 30, 24), swimmers=(sw,))
    asm = assemble(box)
    ref = _run(box, asm, "tiles", monkeypatch, storage)
    got = _run(box, asm, kernel, monkeypatch, storage)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
