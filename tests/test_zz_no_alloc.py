"""The allocation-free spreading entry point.

Some callers cannot allocate device memory: code inside a framework whose
caching allocator owns all device memory, or loops that must keep their
memory footprint fixed after start-up.
ib_spread_fixed_noalloc serves them with a scratch grid the library owns.
This file is collected last on purpose: it checks the new entry point
against the context path's deterministic spreading, on two calls in a row
(the second call must not see the first call's sums)."""
import ctypes
import math

import numpy as np
import pytest

from workloads import BoxSpec, SwimmerSpec, assemble, perturbed_nodes


def _box():
    s = SwimmerSpec(center=(20.3, 18.6, 17.2), radius=4.0, subdiv=2, spacing=12.0).with_drive(1e-3, 1e-3, math.pi / 2)
    return BoxSpec(dims=(40, 36, 34), swimmers=(s,))


def test_no_alloc_rejects_boxes_above_the_limit():
    from paper_2202_12147_gb300 import _lib
    L = _lib.load()
    out = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    rc = L.ib_spread_fixed_noalloc(None, None, 0, 65, 64, 64, _lib.PESKIN4, out, None)
    assert rc == _lib.LBIB_ESIZE
    assert "maximum" in L.lbib_last_error().decode()


@pytest.mark.gpu
@pytest.mark.parametrize("kernel", ["peskin4", "linear2"])
def test_no_alloc_spread_matches_context_path(kernel):
    import torch
    from paper_2202_12147_gb300 import Simulation, _lib
    assert torch.cuda.is_available()
    box = _box()
    asm = assemble(box)
    r = perturbed_nodes(asm["nodes"], seed=5, amp=0.05)
    sim = Simulation(box.dims, asm, deterministic=True, kernel=kernel)
    sim.set_nodes(r)
    sim.ib_spread()
    F_ref = sim.get_force_field()
    fn = sim.get_node_forces()
    sim.close()
    assert np.abs(F_ref).max() > 0
    L = _lib.load()
    r_d = torch.from_numpy(np.ascontiguousarray(r)).cuda()
    f_d = torch.from_numpy(np.ascontiguousarray(fn)).cuda()
    N = box.n_cells
    stream = torch.cuda.current_stream()
    for call in range(2):
        out = torch.full((N, 3), float("nan"), dtype=torch.float32, device="cuda")
        rc = L.ib_spread_fixed_noalloc(ctypes.c_void_p(r_d.data_ptr()), ctypes.c_void_p(f_d.data_ptr()), r.shape[0],
                                       *box.dims, _lib.LINEAR2 if kernel == "linear2" else _lib.PESKIN4,
                                       ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == _lib.LBIB_OK, L.lbib_last_error().decode()
        torch.cuda.synchronize()
        F = out.cpu().numpy()
        assert np.isfinite(F).all()
        # the same integers summed exactly and converted with one rounding:
        # bitwise equal to the context path, on the second call as on the first
        np.testing.assert_array_equal(F, F_ref, err_msg=f"call {call}")
