"""The hand-written reverse sweep (lb_adjoint_*) against the oracle.

* its forward sweep reproduces the oracle's coupled step;
* dD/dtheta (D = x displacement of the swimmer over one drive period, theta
  the per-bead amplitudes and phases) agrees with the oracle's exact discrete
  derivative (complex step) and with central finite differences;
* the adjoint of the whole multi-step map passes the dot-product test
  <J v, w> = <v, J^T w> against central differences of the FP64 forward;
* checkpoint intervals and the autograd wrapper do not change the result.
"""
import json
import os

import numpy as np
import pytest

import oracle
from gpu_helpers import gpu_f_to_oracle, lattice_perm, oracle_f_to_gpu, rel_l2
from workloads import adjoint_small, assemble, perturbed_nodes, random_populations

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
PARAMS = [(0, 0), (0, 1), (0, 2), (0, 4), (0, 5)]  # A1, A2, A3, phi2, phi3
IDX = [0, 1, 2, 4, 5]


def _engine(box, asm, n_steps, K, precision):
    from paper_2202_12147_gb300 import Adjoint
    return Adjoint(box.dims, asm, n_steps=n_steps, K=K, precision=precision, tau=box.tau, rho0=box.rho0, g=box.g)


@pytest.fixture(scope="module")
def small():
    box = adjoint_small()
    asm = assemble(box)
    steps = int(box.swimmers[0].period)
    cs = oracle.displacement_jacobian_cs(box, steps, PARAMS, asm=asm)[:, 0, 0]
    D = oracle.displacement(box, steps, asm=asm)[0, 0]
    return box, asm, steps, cs, D


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_forward_sweep_matches_oracle(gpu_lib, precision):
    box = adjoint_small()
    asm = assemble(box)
    eng = _engine(box, asm, 60, 25, precision)
    disp = eng.forward()
    osim = oracle.OracleSim(box, asm)
    x0 = osim.swimmer_centres()
    osim.step(60)
    f, r = eng.final_state()
    perm = lattice_perm()
    _, ug = oracle.macros(gpu_f_to_oracle(f, perm))
    _, uo = oracle.macros(osim.f)
    tol_u, tol_r = (1e-10, 1e-12) if precision == "f64" else (1e-5, 1e-7)
    assert rel_l2(ug, uo) < tol_u
    assert np.abs(r - osim.r).max() < tol_r
    # the oracle's x_cm(T) - x_cm(0) is rounded at |x_cm| * 2^-52 (about 4e-15 here)
    d_ref = (osim.swimmer_centres() - x0)[0]
    assert abs(disp[0, 0] - d_ref[0]) < (1e-13 if precision == "f64" else 1e-3 * abs(d_ref[0]))
    eng.close()


def test_gradient_fp64_matches_complex_step(gpu_lib, small):
    box, asm, steps, cs, D = small
    eng = _engine(box, asm, steps, 30, "f64")  # segments 30, 30, 30, 10
    d = eng.forward()
    assert d[0, 0] == pytest.approx(D, abs=1e-13)
    g = eng.backward(np.array([[1.0, 0.0, 0.0]]))[0, IDX]
    assert np.abs(g - cs).max() < 1e-9 * np.abs(cs).max(), (g, cs)
    eng.close()


def test_gradient_fp32(gpu_lib, small):
    """FP32 fluid state, FP64 node-level work: the gradient's error against the
    exact derivative stays at the level of the forward sweep's FP32 error."""
    box, asm, steps, cs, D = small
    eng = _engine(box, asm, steps, 30, "f32")
    eng.forward()
    g = eng.backward(np.array([[1.0, 0.0, 0.0]]))[0, IDX]
    err = np.abs(g - cs).max() / np.abs(cs).max()
    print(f"FP32 adjoint max relative gradient error {err:.2e}")
    assert err < 1e-4
    eng.close()


def test_checkpoint_interval_does_not_change_the_gradient(gpu_lib, small):
    box, asm, steps, cs, D = small
    out = []
    for K in (7, steps, 1000):
        eng = _engine(box, asm, steps, K, "f64")
        eng.forward()
        out.append(eng.backward(np.array([[1.0, 0.0, 0.0]]))[0])
        eng.close()
    for g in out[1:]:
        assert np.abs(g - out[0]).max() < 1e-12 * np.abs(out[0]).max()


def test_backward_twice_and_error_paths(gpu_lib, small):
    from paper_2202_12147_gb300._lib import LbibError
    box, asm, steps, cs, D = small
    eng = _engine(box, asm, 40, 16, "f64")
    with pytest.raises(LbibError):
        eng.backward(np.array([[1.0, 0.0, 0.0]]))  # no forward sweep yet
    eng.forward()
    g1 = eng.backward(np.array([[1.0, 0.0, 0.0]]))
    g2 = eng.backward(np.array([[1.0, 0.0, 0.0]]))  # slots now hold segment 0: recomputes the last one
    assert np.abs(g1 - g2).max() < 1e-12 * np.abs(g1).max()
    g3 = eng.backward(np.array([[2.0, 0.0, 0.0]]))  # linear in the seed
    assert np.abs(g3 - 2 * g1).max() < 1e-12 * np.abs(g1).max()
    # a second forward sweep records into slot sets the reverse sweeps used
    # (their row tags and lists start afresh): the same gradient again
    eng.forward()
    g4 = eng.backward(np.array([[1.0, 0.0, 0.0]]))
    assert np.abs(g4 - g1).max() < 1e-12 * np.abs(g1).max()
    eng.set_drive(eng.theta0)
    with pytest.raises(LbibError):
        eng.backward(np.array([[1.0, 0.0, 0.0]]))  # the drive changed: forward first
    eng.close()


def test_dot_product_whole_step(gpu_lib):
    """<dL/dx0, v> equals the central difference of L(x0 +- e v) for
    L = <w_f, f(T)> + <w_r, r(T)> over three coupled steps from a perturbed
    state (every kernel of the reverse sweep enters)."""
    box = adjoint_small()
    asm = assemble(box)
    perm = lattice_perm()
    c, w = oracle.lattice()
    N = box.n_cells
    f0 = oracle_f_to_gpu(random_populations(N, w, seed=11, rho_amp=2e-3, u_amp=2e-3), perm)
    r0 = perturbed_nodes(asm["nodes"], seed=12, amp=0.05)
    rng = np.random.default_rng(13)
    wf = rng.standard_normal((19, N))
    wr = rng.standard_normal(r0.shape)
    vf = 1e-4 * rng.standard_normal((19, N)) * w[perm][:, None]
    vr = 1e-3 * rng.standard_normal(r0.shape)
    eng = _engine(box, asm, 3, 2, "f64")

    def L(f, r):
        eng.set_initial(f, r)
        eng.forward()
        fT, rT = eng.final_state()
        return float(np.sum(wf * fT) + np.sum(wr * rT))

    eng.set_initial(f0, r0)
    eng.forward()
    _, gf, gr = eng.backward(np.zeros((1, 3)), seed_f=wf, seed_r=wr, state_grads=True)
    lhs = float(np.sum(gf * vf) + np.sum(gr * vr))
    fd = (L(f0 + vf, r0 + vr) - L(f0 - vf, r0 - vr)) / 2.0
    assert lhs == pytest.approx(fd, rel=1e-6)
    eng.close()


def test_autograd_function(gpu_lib, small):
    import torch
    from paper_2202_12147_gb300 import displacement
    box, asm, steps, cs, D = small
    eng = _engine(box, asm, steps, 25, "f64")
    theta = torch.tensor(eng.theta0, dtype=torch.float64, requires_grad=True)
    disp = displacement(theta, eng)
    assert disp.shape == (1, 3)
    assert float(disp[0, 0]) == pytest.approx(D, abs=1e-13)
    disp[0, 0].backward()
    g = theta.grad.numpy()[0, IDX]
    assert np.abs(g - cs).max() < 1e-9 * np.abs(cs).max()
    eng.close()


def _golden():
    with open(os.path.join(HERE, "golden", "adjoint_single_96.json")) as fh:
        return json.load(fh)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_adjoint_single_96_against_stored_oracle_gradients(gpu_lib, precision):
    """The 96^3 workload, one period of 1000 steps, checkpoints every 100
    steps: the gradient against the oracle's stored central differences
    (h = 1e-6 relative) and exact discrete derivative."""
    from workloads import adjoint_single_96
    gold = _golden()
    box = adjoint_single_96()
    asm = assemble(box)
    eng = _engine(box, asm, gold["steps"], 100, precision)
    d = eng.forward()
    g = eng.backward(np.array([[1.0, 0.0, 0.0]]))[0, IDX]
    fd = np.array([v[0] for v in gold["grad_finite_difference"]])
    cs = np.array([v[0] for v in gold["grad_complex_step"]])
    scale = np.abs(cs).max()
    err_fd = np.abs(g - fd).max() / scale
    err_cs = np.abs(g - cs).max() / scale
    t = eng.timing()
    print(f"{precision}: D {d[0, 0]:.10e} (oracle {gold['displacement'][0]:.10e}); gradient error vs finite "
          f"differences {err_fd:.2e}, vs exact derivative {err_cs:.2e}; forward {t['forward_ms']:.1f} ms, "
          f"backward {t['backward_ms']:.1f} ms")
    if precision == "f64":
        assert d[0, 0] == pytest.approx(gold["displacement"][0], abs=1e-12)
        assert err_fd < 1e-4
        assert err_cs < 1e-8
    else:
        assert d[0, 0] == pytest.approx(gold["displacement"][0], rel=1e-3)
        assert err_cs < 1e-4
        assert err_fd < 1e-4
    eng.close()
