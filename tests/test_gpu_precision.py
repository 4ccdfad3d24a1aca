"""Reduced-precision population storage (FP16 / BF16 of the scaled shifted
deviations d_i / w_i * S, collided in FP32) against the FP64 oracle.

Tolerance: velocity field relative L2 <= 2e-3 after the stated step counts
and swimmer displacement within 1 %, for both 16-bit formats.  A 16-bit
float keeps 11 (FP16) or 8 (BF16) significant bits, so each stored deviation
carries a relative rounding error of up to 2^-12 or 2^-9 per step.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import gpu_f_to_oracle, gpu_sim, lattice_perm, oracle_f_to_gpu, rel_l2
from workloads import assemble, fluid_box, random_populations, single_swimmer_48

pytestmark = pytest.mark.gpu

BOUND = {"f16": 2e-3, "bf16": 2e-3}


@pytest.fixture(scope="module")
def perm(gpu_lib):
    return lattice_perm()


@pytest.fixture(scope="module")
def oracle_48():
    box = single_swimmer_48()
    asm = assemble(box)
    osim = oracle.OracleSim(box, asm).step(500)
    return box, asm, osim


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_fluid_step_reduced_storage(perm, storage):
    box = fluid_box((32, 20, 18), tau=0.8, g=(1e-6, 0.0, 0.0))
    c, w = oracle.lattice()
    f0 = random_populations(box.n_cells, w, seed=21, rho_amp=1e-3, u_amp=1e-3)
    sim = gpu_sim(box, storage=storage)
    sim.set_populations(oracle_f_to_gpu(f0, perm))
    sim.lb_step(20)
    fg = gpu_f_to_oracle(sim.get_populations(), perm)
    fo = f0
    for _ in range(20):
        fo, _, _ = oracle.lb_step(fo, box.dims, box.tau, g=box.g)
    _, ug = oracle.macros(fg)
    _, uo = oracle.macros(fo)
    err = rel_l2(ug, uo)
    print(f"{storage}: velocity rel L2 after 20 steps {err:.3e}")
    assert err < BOUND[storage], err
    sim.close()


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_single_swimmer_48_reduced_storage(perm, oracle_48, storage):
    """The 48^3 single-swimmer workload for a full drive period (500 steps)."""
    box, asm, osim = oracle_48
    sim = gpu_sim(box, asm, storage=storage)
    sim.lb_step(500)
    st = sim.swimmer_state(0)
    fg = gpu_f_to_oracle(sim.get_populations(), perm)
    _, ug = oracle.macros(fg)
    _, uo = oracle.macros(osim.f)
    err = rel_l2(ug, uo)
    x0 = asm["nodes"].reshape(3, -1, 3).mean(axis=(0, 1))
    dx_o = osim.swimmer_centres()[0][0] - x0[0]
    print(f"{storage}: velocity rel L2 {err:.3e}, displacement {st['disp'][0]:.6e} vs {dx_o:.6e}")
    assert err < BOUND[storage], err
    assert abs(st["disp"][0] - dx_o) < 0.01 * abs(dx_o)
    sim.close()
