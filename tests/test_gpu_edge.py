"""Degenerate and corner cases of the coupled step against the FP64 oracle
(or against what the method fixes exactly).

* a swimmer with zero drive at its rest shape: every force is zero to
  rounding, so the fluid stays at rest and the nodes do not move;
* 16-bit storage on a box whose rows cannot be split into 2- or 4-cell
  groups (odd nx: one cell per thread), both AA parities;
* relaxation times near the stability limit (tau = 0.51) and large (tau = 3);
* Shan-Chen forcing with FP16 storage and a body force.
"""
import math

import numpy as np
import pytest

import oracle
from gpu_helpers import gpu_f_to_oracle, gpu_sim, lattice_perm, oracle_f_to_gpu, rel_l2
from workloads import BoxSpec, SwimmerSpec, assemble, fluid_box, random_populations

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def perm(gpu_lib):
    return lattice_perm()


def test_zero_drive_is_a_fixed_point(perm):
    sw = SwimmerSpec(center=(24.0, 16.0, 16.0), radius=4.0, subdiv=2, spacing=12.0, period=100.0).with_drive(
        0.0, 0.0, math.pi / 2)
    box = BoxSpec(dims=(48, 32, 32), swimmers=(sw,))
    asm = assemble(box)
    sim = gpu_sim(box, asm)
    r0 = sim.get_nodes()
    sim.lb_step(40)
    _, w = oracle.lattice()
    f = gpu_f_to_oracle(sim.get_populations(), perm)
    assert np.abs(f - w[None, :] * box.rho0).max() < 1e-12
    assert np.abs(sim.get_nodes() - r0).max() < 1e-12
    st = sim.swimmer_state(0)
    assert np.abs(st["disp"]).max() < 1e-12
    sim.close()


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_reduced_storage_odd_rows(perm, storage):
    """nx = 27: no 2- or 4-cell grouping; 9 steps (both parities)."""
    box = fluid_box((27, 13, 11), tau=0.8, g=(1e-6, -5e-7, 0.0))
    _, w = oracle.lattice()
    f0 = random_populations(box.n_cells, w, seed=31, rho_amp=1e-3, u_amp=1e-3)
    sim = gpu_sim(box, storage=storage)
    sim.set_populations(oracle_f_to_gpu(f0, perm))
    sim.lb_step(9)
    fo = f0
    for _ in range(9):
        fo, _, _ = oracle.lb_step(fo, box.dims, box.tau, g=box.g)
    _, ug = oracle.macros(gpu_f_to_oracle(sim.get_populations(), perm))
    _, uo = oracle.macros(fo)
    err = rel_l2(ug, uo)
    print(f"{storage}, nx = 27, 9 steps: velocity rel L2 {err:.2e}")
    # random deviations as large as the velocity they carry: each stored value
    # is rounded at up to 2^-p relative (p = 12 FP16, 9 BF16), and the error
    # of the velocity, a signed sum of them, stays within twice that
    assert err < 2.0 * 2.0 ** -(12 if storage == "f16" else 9)
    sim.close()


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("dims", [(264, 6, 5), (200, 7, 5), (36, 9, 7)])
def test_multi_cell_lanes_partial_warps(perm, storage, dims):
    """Two (FP32) or four (16-bit) cells per lane, with the x-shifted values of
    odd steps passed between lanes: rows of two tiles (264 = 256 + 8 cells),
    a row whose last warp is partly idle (200 cells), a row shorter than a
    warp's cells (36); 1, 2 and 5 steps (both parities).  A value moved to
    the wrong cell shows as an O(1) error of the deviations."""
    box = fluid_box(dims, tau=0.9, g=(1e-6, 0.0, -5e-7))
    _, w = oracle.lattice()
    f0 = random_populations(box.n_cells, w, seed=sum(dims), rho_amp=1e-3, u_amp=1e-3)
    dev_o = []
    fo = f0
    for n in range(1, 6):
        fo, _, _ = oracle.lb_step(fo, box.dims, box.tau, g=box.g)
        dev_o.append(fo - w[None, :] * box.rho0)
    for steps in (1, 2, 5):
        sim = gpu_sim(box, storage=storage)
        sim.set_populations(oracle_f_to_gpu(f0, perm))
        sim.lb_step(steps)
        dg = gpu_f_to_oracle(sim.get_populations(), perm) - w[None, :] * box.rho0
        sim.close()
        do = dev_o[steps - 1]
        err = np.abs(dg - do).max() / np.abs(do).max()
        bound = {"f32": 1e-5, "f16": 5e-3, "bf16": 3e-2}[storage]
        assert err < bound, (steps, err)


@pytest.mark.parametrize("tau", [0.51, 3.0])
def test_extreme_relaxation_times(perm, tau):
    box = fluid_box((40, 24, 20), tau=tau, g=(1e-6, 0.0, 2e-7))
    _, w = oracle.lattice()
    f0 = random_populations(box.n_cells, w, seed=41, rho_amp=1e-3, u_amp=1e-3)
    sim = gpu_sim(box)
    sim.set_populations(oracle_f_to_gpu(f0, perm))
    sim.lb_step(12)
    fo = f0
    for _ in range(12):
        fo, _, _ = oracle.lb_step(fo, box.dims, box.tau, g=box.g)
    _, ug = oracle.macros(gpu_f_to_oracle(sim.get_populations(), perm))
    _, uo = oracle.macros(fo)
    assert rel_l2(ug, uo) < 1e-5
    sim.close()


def test_shan_chen_with_fp16_storage(perm):
    box = fluid_box((32, 16, 12), tau=0.9, g=(2e-6, 0.0, -1e-6), forcing="shan_chen")
    _, w = oracle.lattice()
    f0 = random_populations(box.n_cells, w, seed=51, rho_amp=1e-3, u_amp=1e-3)
    sim = gpu_sim(box, storage="f16")
    sim.set_populations(oracle_f_to_gpu(f0, perm))
    sim.lb_step(10)
    fo = f0
    for _ in range(10):
        fo, _, _ = oracle.lb_step(fo, box.dims, box.tau, g=box.g, forcing=oracle.SHAN_CHEN)
    _, ug = oracle.macros(gpu_f_to_oracle(sim.get_populations(), perm))
    _, uo = oracle.macros(fo)
    assert rel_l2(ug, uo) < 2e-3
    sim.close()
