"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element
by element on seeded inputs.

Tolerances.  The CUDA path stores FP32 deviations f_i - w_i rho0 and
collides in FP32; each step rounds every deviation at ~6e-8 relative, so
deviation fields agree to ~1e-6 relative after tens of steps; the velocity
field criterion is a relative L2 error <= 1e-5 after the stated step count.
"""
import math

import numpy as np
import pytest

import oracle
from gpu_helpers import gpu_f_to_oracle, gpu_sim, lattice_perm, oracle_f_to_gpu, rel_l2
from workloads import BoxSpec, SwimmerSpec, assemble, fluid_box, random_populations, single_swimmer_48, perturbed_nodes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def perm(gpu_lib):
    return lattice_perm()


def _dev(f, w, rho0=1.0):
    return f - w[None, :] * rho0


@pytest.mark.parametrize("steps", [1, 2, 5])
@pytest.mark.parametrize("forcing", ["guo", "shan_chen"])
def test_fluid_random_state_ragged_box(perm, steps, forcing):
    """Random populations, uniform force, a box whose cell count (2717) leaves
    a ragged last tile; both AA parities."""
    box = fluid_box((19, 13, 11), tau=0.8, g=(2e-6, -1e-6, 5e-7), forcing=forcing)
    c, w = oracle.lattice()
    f0 = random_populations(box.n_cells, w, seed=steps, rho_amp=1e-3, u_amp=1e-3)
    sim = gpu_sim(box)
    sim.set_populations(oracle_f_to_gpu(f0, perm))
    sim.lb_step(steps)
    fg = gpu_f_to_oracle(sim.get_populations(), perm)
    fo = f0
    for _ in range(steps):
        fo, _, _ = oracle.lb_step(fo, box.dims, box.tau, g=box.g, forcing=oracle.SHAN_CHEN if forcing == "shan_chen" else oracle.GUO)
    assert rel_l2(_dev(fg, w), _dev(fo, w)) < 1e-6
    assert np.abs(fg - fo).max() < 1e-9
    rho, u = sim.lb_get_macros()
    ro, uo = oracle.macros(fo)
    assert rel_l2(u.cpu().numpy(), uo) < 1e-5
    np.testing.assert_allclose(rho.cpu().numpy(), ro, rtol=1e-6)
    sim.close()


def test_fluid_many_steps_graph_path(perm):
    """37 steps: graph replays (16 steps each) plus single-step tails."""
    box = fluid_box((32, 24, 20), tau=0.7)
    c, w = oracle.lattice()
    f0 = random_populations(box.n_cells, w, seed=9, rho_amp=1e-3, u_amp=1e-3)
    sim = gpu_sim(box)
    sim.set_populations(oracle_f_to_gpu(f0, perm))
    sim.lb_step(3)
    sim.lb_step(34)
    fg = gpu_f_to_oracle(sim.get_populations(), perm)
    fo = f0
    for _ in range(37):
        fo, _, _ = oracle.lb_step(fo, box.dims, box.tau)
    assert rel_l2(_dev(fg, w), _dev(fo, w)) < 2e-6
    # mass and momentum conserved on the GPU itself
    assert fg.sum() == pytest.approx(f0.sum(), rel=1e-7)
    np.testing.assert_allclose((fg @ c).sum(0), (f0 @ c).sum(0), atol=1e-6)
    sim.close()


def test_uniform_force_closed_form_gpu(perm):
    """Resting fluid under uniform g: after n steps every cell has momentum n g."""
    g = np.array([1e-5, -2e-6, 3e-6])
    box = fluid_box((16, 8, 8), tau=0.9, g=g)
    sim = gpu_sim(box)
    sim.lb_step(20)
    rho, u = sim.lb_get_macros()
    np.testing.assert_allclose(u.cpu().numpy(), np.tile(20 * g, (box.n_cells, 1)), rtol=2e-5, atol=1e-12)
    sim.close()


def _perturbed_swimmer_box(kernel="peskin4", dims=(40, 36, 34), center=(20.3, 18.6, 17.2)):
    s = SwimmerSpec(center=center, radius=4.0, subdiv=2, spacing=12.0).with_drive(1e-3, 1e-3, math.pi / 2)
    return BoxSpec(dims=dims, swimmers=(s,), kernel=kernel)


@pytest.mark.parametrize("kernel", ["peskin4", "linear2"])
def test_node_forces_and_spread(perm, kernel):
    box = _perturbed_swimmer_box(kernel)
    asm = assemble(box)
    sim = gpu_sim(box, asm)
    r = perturbed_nodes(asm["nodes"], seed=1, amp=0.05)
    sim.set_nodes(r)
    sim.ib_spread()
    fg = sim.get_node_forces().astype(np.float64)
    osim = oracle.OracleSim(box, asm)
    osim.r = r.copy()
    fo = osim.node_forces()
    assert np.abs(fg - fo).max() < 1e-5 * np.abs(fo).max()
    Fg = sim.get_force_field().astype(np.float64)
    Fo = oracle.spread(r, fg, box.dims, oracle.LINEAR2 if kernel == "linear2" else oracle.PESKIN4)
    assert np.abs(Fg - Fo).max() < 1e-6 * np.abs(Fo).max()
    # FP32 atomics round each of ~25 contributions per cell; the sums agree to rounding
    np.testing.assert_allclose(Fg.sum(0), fg.sum(0), atol=1e-6 * np.abs(fg).sum())
    sim.close()


def test_swimmer_state_forces_and_torques(perm):
    """Per-bead observables after ib_spread at perturbed positions (t = 0).
    F_b is the sum of the oracle's node forces over bead b; the membrane part
    cancels (translation invariance of the energy), leaving the drive plus the
    spring force of Sec. 2.2 from the oracle's own drive and springs
    functions.  T_b = sum_j (r_j - R_b) x f_j vanishes up to rounding
    (rotation invariance; the drive and spring shares are uniform over the
    nodes and R_b is their mean).

    The GPU sums F_b and T_b in FP64.  F_b is a small remainder of much
    larger node forces (here, with nodes displaced by 0.05 lattice units, the
    undriven bead's F_b is 1.5e-5 of sum |f_j|), so the reduction is checked
    relative to |F_b| itself, against the FP64 sum of the GPU's own FP32 node
    forces (an FP32 sum misses this bound by orders of magnitude).  Against
    the oracle the FP32 rounding of the node forces themselves sets the
    error, so that comparison is relative to sum |f_j|; the physical run of
    test_coupled_single_swimmer_48 checks F_b against the oracle relative to
    |F_b|."""
    box = _perturbed_swimmer_box()
    asm = assemble(box)
    sim = gpu_sim(box, asm)
    r = perturbed_nodes(asm["nodes"], seed=4, amp=0.05)
    sim.set_nodes(r)
    sim.ib_spread()
    st = sim.swimmer_state(0)
    fg = sim.get_node_forces().astype(np.float64)
    rg = sim.get_nodes()
    osim = oracle.OracleSim(box, asm)
    osim.r = r.copy()
    fo = osim.node_forces()
    beads = asm["beads"]
    sw = asm["swimmers"][0]
    R = oracle.bead_centres(r, beads)
    fd = oracle.drive(osim.drive[0, 0:3], osim.drive[0, 3:6], sw["balance"], sw["period"], 0.0)
    fs = oracle.springs(sw["k"], sw["L"], R[sw["beads"]])
    for q, b in enumerate(sw["beads"]):
        n0, nn = beads[b][0], beads[b][1]
        rj, fj = r[n0:n0 + nn], fo[n0:n0 + nn]
        F_ref = fj.sum(0)
        f_scale = np.abs(fj).sum()
        assert np.abs(F_ref - (fd[q] + fs[q])).max() < 1e-12 * f_scale
        assert np.linalg.norm(F_ref) < 0.05 * f_scale  # the remainder is small against the node forces
        T_ref = np.cross(rj - R[b], fj).sum(0)
        t_scale = (np.linalg.norm(rj - R[b], axis=1) * np.linalg.norm(fj, axis=1)).sum()
        assert np.abs(T_ref).max() < 1e-12 * t_scale
        assert np.abs(np.asarray(st["R"][q]) - R[b]).max() < 1e-12
        F_gpu, T_gpu = np.asarray(st["F"][q]), np.asarray(st["T"][q])
        # the reduction: FP64 sums of the GPU's own node data
        gj, gr = fg[n0:n0 + nn], rg[n0:n0 + nn]
        F_own = gj.sum(0)
        T_own = np.cross(gr - gr.mean(0), gj).sum(0)
        red_f = np.abs(F_gpu - F_own).max() / np.linalg.norm(F_own)
        red_t = np.abs(T_gpu - T_own).max() / t_scale
        err_f = np.abs(F_gpu - F_ref).max() / f_scale
        print(f"bead {q}: |F_b| {np.linalg.norm(F_ref):.3e} (sum |f_j| {f_scale:.3e}); reduction error "
              f"{red_f:.1e} of |F_b|, torque {red_t:.1e} of its scale; F_b against the oracle {err_f:.1e} "
              f"of sum |f_j|")
        assert red_f < 1e-8
        assert red_t < 1e-12
        assert err_f < 1e-5
        assert np.abs(T_gpu - T_ref).max() < 1e-5 * t_scale
    np.testing.assert_allclose(st["x_cm"], R[sw["beads"]].mean(0), rtol=0, atol=1e-12)
    sim.close()


@pytest.mark.parametrize("kernel", ["peskin4", "linear2"])
def test_interpolate(perm, kernel):
    import torch
    box = _perturbed_swimmer_box(kernel, center=(1.4, 18.6, 33.5))  # straddles the periodic seams
    asm = assemble(box)
    sim = gpu_sim(box, asm)
    rng = np.random.default_rng(3)
    u = rng.normal(size=(box.n_cells, 3)).astype(np.float32)
    sim.set_velocity(u)
    v = sim.ib_interpolate().cpu().numpy()
    vo = oracle.interpolate(asm["nodes"], u.astype(np.float64), box.dims,
                            oracle.LINEAR2 if kernel == "linear2" else oracle.PESKIN4)
    assert np.abs(v - vo).max() < 2e-6 * np.abs(vo).max()
    sim.close()


def test_deterministic_spread_is_bitwise_reproducible(perm):
    box = _perturbed_swimmer_box()
    asm = assemble(box)
    r = perturbed_nodes(asm["nodes"], seed=2, amp=0.05)
    outs = []
    for _ in range(2):
        sim = gpu_sim(box, asm, deterministic=True)
        sim.set_nodes(r)
        sim.ib_spread()
        outs.append(sim.get_force_field())
        sim.close()
    assert np.array_equal(outs[0], outs[1])
    sim = gpu_sim(box, asm)
    sim.set_nodes(r)
    sim.ib_spread()
    Fa = sim.get_force_field()
    assert np.abs(outs[0] - Fa).max() < 1e-6 * np.abs(Fa).max()
    sim.close()


def test_deterministic_spread_with_scattered_nodes(perm):
    """Nodes scattered at random over a 48^3 box: the 32 nodes a spreading
    block holds touch up to 2048 distinct cells, more than its shared table
    of 1024, so contributions also take the direct path to the global
    fixed-point field.  The field is still bitwise reproducible, and equal to
    the float-atomic field and to the oracle's spreading of the same node
    forces to FP32 rounding."""
    from workloads import single_swimmer_48
    box = single_swimmer_48()
    asm = assemble(box)
    rng = np.random.default_rng(8)
    r = rng.uniform(0.0, 48.0, size=asm["nodes"].shape)
    outs = []
    for det in (True, True, False):
        sim = gpu_sim(box, asm, deterministic=det)
        sim.set_nodes(r)
        sim.ib_spread()
        outs.append((sim.get_force_field().astype(np.float64), sim.get_node_forces().astype(np.float64)))
        sim.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    scale = np.abs(outs[0][0]).max()
    assert np.abs(outs[0][0] - outs[2][0]).max() < 1e-6 * scale
    Fo = oracle.spread(r, outs[0][1], box.dims)
    assert np.abs(outs[0][0] - Fo).max() < 1e-6 * np.abs(Fo).max()


@pytest.mark.parametrize("deterministic", [False, True])
def test_coupled_single_swimmer_48(perm, deterministic):
    """The 48^3 single-swimmer workload (beads of radius 4 at subdivision 2,
    k = 0.005, Gs = 0.01, drive 1e-3, period 500, phase pi/2), a full period
    of 500 steps: velocity field within 1e-5 relative L2, swimmer
    displacement within 1%."""
    box = single_swimmer_48()
    asm = assemble(box)
    sim = gpu_sim(box, asm, deterministic=deterministic)
    sim.lb_step(500)
    st = sim.swimmer_state(0)
    osim = oracle.OracleSim(box, asm).step(500)
    fg = gpu_f_to_oracle(sim.get_populations(), perm)
    _, ug = oracle.macros(fg)
    _, uo = oracle.macros(osim.f)
    err = rel_l2(ug, uo)
    assert err < 1e-5, err
    rg = sim.get_nodes()
    assert np.abs(rg - osim.r).max() < 1e-6
    xo = osim.swimmer_centres()[0]
    dx_o = xo - asm["nodes"].reshape(3, -1, 3).mean(axis=(0, 1))
    assert st["step"] == 500
    assert abs(st["disp"][0] - dx_o[0]) < 0.01 * abs(dx_o[0]) + 1e-9
    np.testing.assert_allclose(st["x_cm"], xo, atol=1e-6)
    # per-bead force of the last step (drive plus springs; the membrane part
    # cancels) against the oracle's node forces of the same step, relative to
    # |F_b|: FP64 bead sums keep the remainder (an FP32 sum of these node
    # forces alone errs by up to 7e-7 of |F_b|)
    for q, b in enumerate(asm["swimmers"][0]["beads"]):
        n0, nn = asm["beads"][b][0], asm["beads"][b][1]
        F_ref = osim.node_force[n0:n0 + nn].sum(0)
        e = np.abs(np.asarray(st["F"][q]) - F_ref).max() / np.linalg.norm(F_ref)
        print(f"bead {q}: |F_b| {np.linalg.norm(F_ref):.3e}, GPU against the oracle {e:.1e} of |F_b|")
        assert e < 1e-3
    sim.close()


def test_empty_structure_and_tiny_box(perm):
    """No swimmers, a box smaller than one tile (5^3 = 125 cells)."""
    box = fluid_box((5, 5, 5), tau=1.3)
    c, w = oracle.lattice()
    f0 = random_populations(box.n_cells, w, seed=4, rho_amp=1e-3, u_amp=1e-3)
    sim = gpu_sim(box)
    sim.set_populations(oracle_f_to_gpu(f0, perm))
    sim.lb_step(7)
    fo = f0
    for _ in range(7):
        fo, _, _ = oracle.lb_step(fo, box.dims, box.tau)
    fg = gpu_f_to_oracle(sim.get_populations(), perm)
    assert rel_l2(_dev(fg, w), _dev(fo, w)) < 1e-6
    sim.close()


def test_swimmer_state_async_matches_sync(gpu_lib):
    """swimmer_state_async queues the same records swimmer_state returns."""
    import ctypes

    import torch

    from paper_2202_12147_gb300 import _lib
    from workloads import BoxSpec, SwimmerSpec
    sw = tuple(SwimmerSpec(center=(24.0, y, 12.0), radius=3.0, subdiv=1, spacing=9.0, period=40.0).with_drive(
        1e-3, 1e-3, 1.0) for y in (8.0, 20.0))
    box = BoxSpec(dims=(48, 28, 24), swimmers=sw)
    s = gpu_sim(box)
    rec = ctypes.sizeof(_lib.SwimmerState)
    ring = torch.zeros((3, 2 * rec), dtype=torch.uint8, pin_memory=True)
    for k in range(3):
        s.lb_step(5)
        s.swimmer_state_async(ring[k])
    s.sync()
    last = _lib.SwimmerState.from_buffer_copy(bytes(ring[2, rec:2 * rec].numpy()))
    ref = s.swimmer_state(1)
    assert last.step == ref["step"] == 15
    assert list(last.x_cm) == list(ref["x_cm"])
    first = _lib.SwimmerState.from_buffer_copy(bytes(ring[0, :rec].numpy()))
    assert first.step == 5
    s.close()


def test_coupled_paper_scheme_shan_chen_linear2(perm):
    """The paper's own choices (Sec. 2.1 Eq. sc velocity shift, Sec. 2.3
    two-point kernel) in a coupled swimmer run against the oracle."""
    from workloads import BoxSpec, SwimmerSpec
    sw = SwimmerSpec(center=(20.0, 14.0, 12.0), radius=3.0, subdiv=2, spacing=9.0, period=60.0).with_drive(
        2e-3, 2e-3, 1.0)
    box = BoxSpec(dims=(40, 28, 24), swimmers=(sw,), forcing="shan_chen", kernel="linear2")
    asm = assemble(box)
    sim = gpu_sim(box, asm)
    sim.lb_step(3)
    sim.lb_step(40)
    osim = oracle.OracleSim(box, asm).step(43)
    _, ug = oracle.macros(gpu_f_to_oracle(sim.get_populations(), perm))
    _, uo = oracle.macros(osim.f)
    assert rel_l2(ug, uo) < 1e-5
    assert np.abs(sim.get_nodes() - osim.r).max() < 1e-6
    np.testing.assert_allclose(sim.swimmer_state(0)["x_cm"], osim.swimmer_centres()[0], atol=1e-6)
    sim.close()


@pytest.mark.parametrize("storage,tol", [("f32", 1e-5), ("f16", 2e-3)])
def test_benchmark_box_full_size(perm, storage, tol):
    """One box of the benchmark at its full size (256 x 128 x 128, two
    side-by-side swimmers of 642-node beads, gap 3 radii), advanced the way
    bench.py does (two streams, 16-step graph replays), against the oracle's
    full field after 32 steps."""
    from workloads import swimmer_pair
    box = swimmer_pair("side", 3)
    asm = assemble(box)
    sim = gpu_sim(box, asm, storage=storage)
    sim.lb_step(32)
    osim = oracle.OracleSim(box, asm).step(32)
    _, ug = oracle.macros(gpu_f_to_oracle(sim.get_populations(), perm))
    _, uo = oracle.macros(osim.f)
    err = rel_l2(ug, uo)
    print(f"{storage}: velocity rel. L2 after 32 steps {err:.2e}")
    assert err < tol
    assert np.abs(sim.get_nodes() - osim.r).max() < (1e-6 if storage == "f32" else 1e-5)
    sim.close()


def test_period_velocity_and_reynolds_numbers(perm):
    """The mean swimming velocity over each completed drive period (Sec. 3,
    Eq. vel_swim), recorded on the device at period boundaries, against the
    oracle's x_cm at the same steps (within 1 %, the net-velocity bound), and
    the Reynolds numbers against their definitions."""
    from workloads import BoxSpec, SwimmerSpec
    T = 40
    sw = SwimmerSpec(center=(24.0, 14.0, 12.0), radius=3.0, subdiv=1, spacing=9.0, period=float(T)).with_drive(
        2e-3, 2e-3, math.pi / 2)
    box = BoxSpec(dims=(48, 28, 24), swimmers=(sw,))
    asm = assemble(box)
    sim = gpu_sim(box, asm)
    assert sim.swimmer_state(0)["periods"] == 0
    sim.lb_step(T - 1)
    st = sim.swimmer_state(0)
    assert st["periods"] == 0 and np.all(st["v_period"] == 0.0)
    sim.lb_step(T + 5)  # 2T + 4 steps: inside the third period
    st = sim.swimmer_state(0)
    assert st["periods"] == 2
    osim = oracle.OracleSim(box, asm).step(T)
    x1 = osim.swimmer_centres()[0]
    osim.step(T)
    x2 = osim.swimmer_centres()[0]
    v_ref = (x2 - x1) / T
    assert abs(st["v_period"][0] - v_ref[0]) < 1e-2 * abs(v_ref[0])
    nu = (box.tau - 0.5) / 3.0
    L_swim = np.linalg.norm(st["R"][2] - st["R"][0]) + 2 * 3.0
    assert st["re_swim"] == pytest.approx(np.linalg.norm(st["v_period"]) * L_swim / nu, rel=1e-6)
    v_bead = max(np.linalg.norm(st["V"][q]) for q in range(3))
    assert st["re_bead"] == pytest.approx(v_bead * 3.0 / nu, rel=1e-6)
    sim.close()
