"""Pins of the oracle's exact discrete derivative (its complex-step twin).

The complex-step method (Squire & Trapp 1998) differentiates the oracle's
own discrete map: each function is evaluated over double complex with one
input perturbed by i*h, and Im(output)/h is its exact derivative.  These
tests tie that derivative to things that do not depend on it: central
finite differences of the real oracle, the energy-force relation of the
membrane (Sec. 2.2, virtual work), the symmetry of a Hessian, and the
equivalence of the free per-bead drive at the base point with the paper's
balanced protocol (Sec. 2.2, driving-force equation).
"""
import math

import numpy as np
import pytest

import oracle
from workloads import adjoint_small, assemble, icosphere, random_populations


def test_phi_complex_step_matches_finite_difference():
    h = 1e-30
    for r in (-1.7, -1.2, -0.6, -0.1, 0.05, 0.4, 0.9, 1.3, 1.95):
        cs = oracle.phi(complex(r, h)).imag / h
        e = 1e-6
        fd = (oracle.phi(r + e) - oracle.phi(r - e)) / (2 * e)
        assert abs(cs - fd) < 1e-9, (r, cs, fd)
        assert oracle.phi(complex(r, h)).real == pytest.approx(oracle.phi(r), abs=1e-16)


@pytest.mark.parametrize("law", [oracle.NEOHOOKE, oracle.SKALAK])
def test_membrane_energy_derivative_is_minus_force(law):
    """d/de W(x + e v) = -<f(x), v>: the complex-step derivative of the
    energy against the oracle's real virtual-work forces."""
    X, tris = icosphere(1)
    X = 4.0 * X
    rng = np.random.default_rng(3)
    x = X * np.array([1.08, 0.95, 1.01]) + 0.05 * rng.standard_normal(X.shape)
    v = rng.standard_normal(X.shape)
    p1, p2 = (0.01, 0.0) if law == oracle.NEOHOOKE else (0.01, 1.0)
    h = 1e-30
    dW = oracle.membrane_energy(X, x + 1j * h * v, tris, p1, p2, law).imag / h
    f = oracle.membrane_forces(X, x, tris, p1, p2, law)
    assert dW == pytest.approx(-np.sum(f * v), rel=1e-11)


def test_membrane_force_jacobian_is_symmetric():
    """The force is minus the gradient of an energy, so its Jacobian (minus
    the Hessian) is symmetric: <w, J v> = <v, J w>."""
    X, tris = icosphere(2)
    X = 4.0 * X
    rng = np.random.default_rng(4)
    x = X * np.array([1.1, 0.93, 1.0]) + 0.05 * rng.standard_normal(X.shape)
    v, w = rng.standard_normal(X.shape), rng.standard_normal(X.shape)
    h = 1e-30

    def jvp(d):
        return oracle.membrane_forces(X, x + 1j * h * d, tris, 0.01).imag / h

    a, b = np.sum(w * jvp(v)), np.sum(v * jvp(w))
    assert a == pytest.approx(b, rel=1e-10)
    # and J v against central differences of the real forces
    e = 1e-6
    fd = (oracle.membrane_forces(X, x + e * v, tris, 0.01) - oracle.membrane_forces(X, x - e * v, tris, 0.01)) / (2 * e)
    assert np.abs(jvp(v) - fd).max() < 1e-7 * np.abs(fd).max()


def test_lb_step_complex_step_matches_finite_difference():
    """Directional derivative of one collide-and-stream step (Sec. 2.1, Eq.
    lbe with Guo forcing) with respect to the populations and the force."""
    dims = (7, 5, 4)
    N = 7 * 5 * 4
    c, w = oracle.lattice()
    rng = np.random.default_rng(5)
    f = random_populations(N, w, seed=5, rho_amp=1e-2, u_amp=2e-2)
    F = 1e-3 * rng.standard_normal((N, 3))
    vf = 1e-2 * rng.standard_normal(f.shape)
    vF = 1e-3 * rng.standard_normal(F.shape)
    h = 1e-30
    out, _, u = oracle.lb_step(f + 1j * h * vf, dims, 0.8, F + 1j * h * vF)
    cs_f, cs_u = out.imag / h, u.imag / h
    e = 1e-6
    fp, _, up = oracle.lb_step(f + e * vf, dims, 0.8, F + e * vF)
    fm, _, um = oracle.lb_step(f - e * vf, dims, 0.8, F - e * vF)
    assert np.abs(cs_f - (fp - fm) / (2 * e)).max() < 1e-8 * np.abs(cs_f).max()
    assert np.abs(cs_u - (up - um) / (2 * e)).max() < 1e-8 * np.abs(cs_u).max()
    # the real part is the real oracle's step
    f_ref, _, _ = oracle.lb_step(f, dims, 0.8, F)
    assert np.abs(out.real - f_ref).max() < 1e-15


def test_free_drive_base_point_equals_balanced_protocol():
    """The per-bead drive (A, sqrt 2 A, A; 0, 5pi/4, pi/2) is the paper's
    f2 = -f1 - f3 with alpha = pi/2: both runs give the same displacement."""
    box = adjoint_small()
    asm = assemble(box)
    free = oracle.drive_parameters(asm)
    assert free[0, 1] == pytest.approx(math.sqrt(2) * 1e-3)
    assert free[0, 4] == pytest.approx(1.25 * math.pi)
    d_free = oracle.displacement(box, 60, asm=asm)
    asm_bal = dict(asm)
    asm_bal["swimmers"] = [dict(asm["swimmers"][0], balance=True)]
    d_bal = oracle.displacement(box, 60, asm=asm_bal)
    assert np.abs(d_free - d_bal).max() < 1e-12 * np.abs(d_bal).max() + 1e-18


def test_displacement_gradient_complex_step_matches_finite_difference():
    """dD/dtheta over one drive period, theta = (A1, A2, A3, phi2, phi3):
    the exact discrete derivative against central differences with
    h = 1e-6 |theta| (the finite differences carry rounding of about
    1e-15 / h in D)."""
    box = adjoint_small()
    asm = assemble(box)
    params = [(0, 0), (0, 1), (0, 2), (0, 4), (0, 5)]
    steps = int(box.swimmers[0].period)
    cs = oracle.displacement_jacobian_cs(box, steps, params, asm=asm)[:, 0, 0]
    fd = oracle.displacement_jacobian_fd(box, steps, params, asm=asm)[:, 0, 0]
    scale = np.abs(cs).max()
    assert scale > 1e-3
    assert np.abs(cs - fd).max() < 5e-5 * scale, (cs, fd)
