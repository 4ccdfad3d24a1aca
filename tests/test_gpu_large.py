"""A box at the large end of what one GPU holds: 1024 x 512 x 448 cells
(235 M cells, 19 x 235 M = 4.5e9 population values, past 32-bit element
offsets; 18 GB of FP32 populations), with a swimmer straddling the periodic
x seam at the far end of the box.

No oracle runs at this size.  The check uses a property that holds at any
size: the lattice Boltzmann update moves information one cell per step, so
for the first steps the flow around a swimmer does not depend on the box
around it.  The same swimmer is run in a 96 x 64 x 64 box, and after 12
steps the node positions, shifted, and the velocity field in the region the
disturbance can have reached must agree (deterministic spreading, so the
force sums do not depend on the order of atomics; the only differences come
from the FP64 rounding of positions of larger magnitude).
"""
import math

import numpy as np
import pytest

from gpu_helpers import gpu_sim
from workloads import BoxSpec, SwimmerSpec, assemble, perturbed_nodes

pytestmark = pytest.mark.gpu

BIG = (1024, 512, 448)
SMALL = (96, 64, 64)
STEPS = 12


def _box(dims, center):
    sw = SwimmerSpec(center=center, radius=4.0, subdiv=2, spacing=12.0, period=40.0).with_drive(
        2e-3, 2e-3, math.pi / 2)
    return BoxSpec(dims=dims, swimmers=(sw,))


def test_large_box_matches_small_box(gpu_lib):
    import torch
    free, _ = torch.cuda.mem_get_info()
    need = BIG[0] * BIG[1] * BIG[2] * (19 * 4 + 16 + 16 + 12) + (4 << 30)
    assert free > need, f"needs {need / 2**30:.0f} GiB of device memory, {free / 2**30:.0f} GiB free"
    c_small = (48.0, 32.0, 32.0)
    shift = np.array([BIG[0] - 4.0 - c_small[0], BIG[1] - 40.0 - c_small[1], BIG[2] - 40.0 - c_small[2]])
    c_big = tuple(float(v) for v in np.array(c_small) + shift)  # x centre 1020: the swimmer straddles x = 0
    small, big = _box(SMALL, c_small), _box(BIG, c_big)
    a_small, a_big = assemble(small), assemble(big)
    r0 = perturbed_nodes(a_small["nodes"], seed=21, amp=0.05)
    assert np.abs(a_big["nodes"] - (a_small["nodes"] + shift)).max() < 1e-12

    out = []
    for box, asm, r in ((small, a_small, r0), (big, a_big, r0 + shift)):
        sim = gpu_sim(box, asm, deterministic=True)
        sim.set_nodes(r)
        sim.lb_step(STEPS)
        nodes = sim.get_nodes()
        _, u = sim.lb_get_macros()
        # the region around the swimmer the disturbance can reach: the
        # swimmer's extent plus the stencil reach and one cell per step
        lo = np.floor(r.min(0)).astype(int) - 2 - STEPS
        hi = np.floor(r.max(0)).astype(int) + 3 + STEPS
        idx = [np.arange(lo[a], hi[a] + 1) % box.dims[a] for a in range(3)]
        cells = (idx[0][:, None, None] + box.dims[0] * (idx[1][None, :, None] + box.dims[1] * idx[2][None, None, :]))
        ureg = u[torch.as_tensor(cells.ravel(), dtype=torch.long, device=u.device)].cpu().numpy().astype(np.float64)
        out.append((nodes, ureg))
        del u
        sim.close()
        torch.cuda.empty_cache()
    (n_s, u_s), (n_b, u_b) = out
    assert np.abs((n_b - shift) - n_s).max() < 1e-10
    assert np.abs(n_s - r0).max() > 1e-5  # the nodes have moved
    assert np.abs(u_s).max() > 1e-6      # the fluid moves in the region
    assert np.abs(u_b - u_s).max() < 1e-6 * np.abs(u_s).max()
